// Private definition of heat_ctx, shared by the translation units of libheat.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/heat.h"

namespace heat {
struct Surrogate;
void surrogate_free(Surrogate* s);
}

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T>
    T* as() const { return (T*)p; }
};

struct heat_ctx {
    int device = 0;
    int N = 0;
    std::vector<double> lam;
    std::string err;

    // grid
    DevBuf d_lam, d_dln, d_lam32, d_dln32;
    // grains
    int G = 0, nbt = 0;
    std::vector<int> bin_off;
    std::vector<double> w;
    bool has_w = false;
    long long band_per_cell = 0;
    int max_bins = 0;
    int band_max = 0;  // largest band (elements per cell) of one grain
    int wmax_all = 1;  // widest band row over the grains
    std::vector<int> grain_order, grain_order_build;  // task orders of the recursion and the build
    std::vector<long long> grain_band;                // band elements per cell of each grain
    std::vector<int> grain_rows;                      // bins of each grain
    int row_weight = 30;                              // recursion order: band + row_weight x rows
    DevBuf d_bin_off, d_cabs, d_T, d_E, d_Cf, d_invC, d_invdE, d_invdE32, d_Cact, d_sC, d_ca32, d_ce32, d_sC32,
        d_rowptr, d_wmax, d_seg_ptr, d_pat64, d_pat32, d_soft, d_soft_off, d_K, d_Kw, d_w, d_koff_all, d_cde,
        d_pent, d_pcol, d_kexp, d_rent, d_gl, d_Dtd, d_Dtd_off, d_Dtd_woff, d_Dtd_order;
    bool td_built = false;  // thermal-discrete downward rates computed
    // fields
    int n_cells = 0;
    const void* u_dev = nullptr;
    int u_dtype = 0;
    DevBuf d_u_own;
    // chunk task lists: (grain, group) pairs, the recursion's order then the build's (each
    // longest first); `full` for chunks of tasks_NG groups, `tail` for the last, shorter
    // chunk (tail_NG groups)
    DevBuf s_tasks, s_tasks_tail;
    int tasks_NG = -1, tail_NG = -1;
    // scratch of one chunk in flight; chunks go round-robin over the slots, each slot on
    // its own stream, so that the FP64 recursion of one chunk overlaps the build and the
    // tensor-core emissivity of the next
    static constexpr int kMaxSlots = 4;
    struct Slot {
        DevBuf ua64, su64, ua32, Bb64, Bb32, xs, ep, pabs, P, j, led, A, rowscale, work, phs, tdq;
        DevBuf P_alt, j_alt, led_alt;   // second staging set of asynchronous host I/O
        cudaStream_t stream = nullptr;  // created on first use
        cudaEvent_t done = nullptr;
        cudaStream_t copy = nullptr;    // asynchronous host I/O: copies to the host
        cudaEvent_t computed = nullptr; // a chunk's kernels are done (copy stream waits on it)
        cudaEvent_t copied[2] = {nullptr, nullptr};  // staging set k has been copied out
        bool copied_valid[2] = {false, false};
    } slots[kMaxSlots];
    cudaEvent_t ev_fork = nullptr;
    int tuned_streams = 0, tuned_chunk = 0;  // heat_autotune's choice (0: none)
    int tuned_recur_bps = 0;                 // its resident blocks per SM of the recursion (0: all)
    int tuned_emis_nt = 0;                   // its tensor-core tile width (0: 256)
    int tuned_fused = 0;                     // its choice of the fused mixed-path kernel
    int tuned_prefetch = 0;                  // its choice of the FP32 build's pattern prefetch (1 on, 2 off)
    int io_parity = 0;  // staging set of the next asynchronous host-I/O solve
    DevBuf d_status;
    long long wait_polls = HEAT_WAIT_POLLS_DEFAULT;  // give-up limit of the tcgen05 kernels' waits
    int sms = 0;
    std::vector<double> radius;
    heat::Surrogate* sur = nullptr;  // learned surrogate (heat_surrogate_init)
    // tensor-core emissivity operands, per mode (index = HEAT_EMIS_*)
    struct TcMode {
        bool built = false;
        DevBuf B, colscale, kp, boff, aoff;
        std::vector<int> kp_h;
        std::vector<long long> boff_h, aoff_h;
        int aoff_cells = -1;
        std::vector<int> order;  // grains by K extent, largest first
    } tc[5], tc_si[5];           // per-grain output; size-integrated output (one operand over all bins)
    // per-kernel event timing
    struct TimedLaunch {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event() {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    heat_status fail(heat_status s, const std::string& m) {
        err = m;
        return s;
    }
    heat_status cuda_fail(cudaError_t e, const char* where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return HEAT_ECUDA;
    }
};

