// The Guhathakurta-Draine recursion (Eq. xf) and renormalisation (Eq. renormalization) over
// the B band that the build wrote: a persistent lane-per-cell kernel (warp = grain x 32 cells,
// one FP64 FMA per band element and cell, no divergence, no cross-lane reductions) and a
// warp-per-spectrum column sweep for solves of few cells.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "pack.cuh"

namespace heat {

// Task loop of the persistent launches: with ch.work set, each warp takes the next task of
// the list from an atomic counter (dynamic scheduling per warp, in the list's order, as the
// paper's dynamic OpenMP schedule does per thread); without it, one warp per task.
template <typename F>
__device__ __forceinline__ void for_each_task(const ChunkDev& ch, int counter, F&& run) {
    const int lane = threadIdx.x & 31;
    if (!ch.work) {
        const int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (task < ch.n_tasks) run(task, lane);
        return;
    }
    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(ch.work + counter, 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= ch.n_tasks) return;
        run(task, lane);
    }
}

// ---------------------------------------------------------------------------
// k_recur: the recursion kernel.  X_0 = 1,
//   X_f = (sum_{j in band(f)} B_fj X_j) / T_{f-1,f}                              (Eq. xf)
// in FP64, where the band holds every j whose transition wavelength lies on the grid
// (all other B_fj are exactly zero) plus the diagonal j = f-1, which also carries the
// intra-bin term; then P = X / sum X (Eq. renormalization) is written to P[cell][off_g + i].
// Overflow guard: when X_f >= 2^800 every X is to be multiplied by 2^-800 (exact).  Only
// the values later rows still read (j >= the next row's band start), the register window
// and the running sum are scaled at once; each stored X keeps the epoch (count of
// rescales) it was last written in, and the normalisation applies the missing powers of
// two, so the work is O(band) per rescale instead of O(f) and the result is the same.
// B streams from the band storage in element order with evict-first loads (it is read
// once), eight elements per step, so that the X history stays in L2.
template <int BUILD>
__device__ __forceinline__ double band_b(const float* B32, const double* B64, int e) {
    if (BUILD) return widen_pos(__ldcs(B32 + (size_t)e * 32));
    return __ldcs(B64 + (size_t)e * 32);
}

// B in its stored type (kept in registers ahead of use), and its FP64 value
template <int BUILD>
struct BandRaw {
    using T = double;
    static __device__ __forceinline__ T load(const float*, const double* B64, int e) {
        return __ldcs(B64 + (size_t)e * 32);
    }
    static __device__ __forceinline__ double wide(T v) { return v; }
};
template <>
struct BandRaw<1> {
    using T = float;
    static __device__ __forceinline__ T load(const float* B32, const double*, int e) {
        return __ldcs(B32 + (size_t)e * 32);
    }
    static __device__ __forceinline__ double wide(T v) { return widen_pos(v); }
};

// x * 2^(-800 d) for x >= 0 and d >= 0 on the integer pipe (the exponent field lowered), zero
// where the result would fall below the normal range (values under 2^-1022 of the current
// scale, far below anything an output resolves).  The recursion's rescales and the
// normalisation's epoch corrections use it: a multiply or the library ldexp would put every
// one of them on the FP64 unit, which the band's FMAs already keep busy.
__device__ __forceinline__ double scale_down_800(double x, int d) {
    const long long bits = __double_as_longlong(x);
    const long long e = (bits >> 52) - 800LL * d;
    return (d == 0) ? x : (e > 0 ? __longlong_as_double(bits - ((800LL * d) << 52)) : 0.0);
}

// Window part of a row: element e1-1-k multiplies X_{f-1-k} = w[k] for k < nreg (<= W),
// accumulated into S in element order; a jump into the unrolled tail, so no predicated-off
// FMA occupies the FP64 pipe.
template <int BUILD, int W>
__device__ __forceinline__ void window_tail(int nreg, const typename BandRaw<BUILD>::T (&br)[W],
                                            const double (&w)[W], double& S) {
    using Raw = BandRaw<BUILD>;
    switch (nreg) {
        case 8: if constexpr (W > 7) S = fma(Raw::wide(br[7 % W]), w[7 % W], S);  // fallthrough
        case 7: if constexpr (W > 6) S = fma(Raw::wide(br[6 % W]), w[6 % W], S);  // fallthrough
        case 6: if constexpr (W > 5) S = fma(Raw::wide(br[5 % W]), w[5 % W], S);  // fallthrough
        case 5: if constexpr (W > 4) S = fma(Raw::wide(br[4 % W]), w[4 % W], S);  // fallthrough
        case 4: if constexpr (W > 3) S = fma(Raw::wide(br[3 % W]), w[3 % W], S);  // fallthrough
        case 3: if constexpr (W > 2) S = fma(Raw::wide(br[2 % W]), w[2 % W], S);  // fallthrough
        case 2: if constexpr (W > 1) S = fma(Raw::wide(br[1 % W]), w[1 % W], S);  // fallthrough
        case 1: S = fma(Raw::wide(br[0]), w[0], S);                               // fallthrough
        default: break;
    }
}

// Epilogue with the emissivity operand (ch.packA): P_i = X_i / sum X for i <= i_end (0 above,
// the pruned tail), written to P when requested and weighted by the bin's emitted power for
// the energy check (returned), and packed for the tensor cores exactly as k_pack_p packs a P
// row: row scale 2^e from the row's largest P (its running maximum, normalised), then each P
// divided by 2^e, rounded to FP32 and split into hi + lo, eight bins per 16-byte store (each
// lane writes its own cell's row).
__device__ __noinline__ double pack_epilogue(const GrainDev& gd, const ChunkDev& ch, int g, int cc, int M, int i_end,
                                             double inv, int epoch, long long xmaxb, const double* xl,
                                             const unsigned short* epl) {
    const int off = gd.bin_off[g];
    double* prow = ch.P ? ch.P + (size_t)cc * ch.ldP + off : nullptr;
    const double* cde = gd.cde + off;
    double emit = 0.0;
    const int e = row_scale_exp((unsigned)__double2hiint(__longlong_as_double(xmaxb) * inv));
    ch.pack_rowscale[(size_t)cc * gd.G + g] = ldexpf(1.0f, e);
    const int K = ch.pack_kp[g], half = ch.pack_split ? K / 2 : K;
    const bool ledger = ch.ledger != nullptr;
    auto p_of = [&](int i) {
        return i <= i_end ? scale_down_800(xl[i * 32], epoch - (int)epl[i * 32]) * inv : 0.0;
    };
    if (ch.pack_tf32) {
        float* row = (float*)ch.packA + ch.pack_aoff[g] + (size_t)cc * K;
        for (int i0 = 0; i0 < half; i0 += 4) {
            float4 h, l;
            float* hv = &h.x;
            float* lv = &l.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k;
                const double p = p_of(i);
                if (i <= M && prow) prow[i] = p;
                if (ledger && i <= i_end) emit = fma(p, cde[i], emit);
                const float v = scaled_to_f32(p, e);
                hv[k] = tf32_rn(v);
                lv[k] = tf32_rn(v - hv[k]);
            }
            *(float4*)(row + i0) = h;
            if (ch.pack_split) *(float4*)(row + half + i0) = l;
        }
    } else {
        uint16_t* row = (uint16_t*)ch.packA + ch.pack_aoff[g] + (size_t)cc * K;
        for (int i0 = 0; i0 < half; i0 += 8) {
            uint4 h, l;
            unsigned* hv = &h.x;
            unsigned* lv = &l.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                unsigned hp = 0, lp = 0;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int i = i0 + 2 * k + s;
                    const double p = p_of(i);
                    if (i <= M && prow) prow[i] = p;
                    if (ledger && i <= i_end) emit = fma(p, cde[i], emit);
                    const float v = scaled_to_f32(p, e);
                    const uint16_t hb = bf16_rn(v);
                    const uint16_t lb = bf16_rn(v - bf16_f(hb));
                    hp |= (unsigned)hb << (16 * s);
                    lp |= (unsigned)lb << (16 * s);
                }
                hv[k] = hp;
                lv[k] = lp;
            }
            *(uint4*)(row + i0) = h;
            if (ch.pack_split) *(uint4*)(row + half + i0) = l;
        }
    }
    return emit;
}

// One task: the recursion of grain g for the 32 cells of group grp (lane = cell).  W is
// the register window: the last W values of X, and the window part of each row's band
// (its last min(width, W) elements), prefetched one row ahead.  The row loop's fixed
// cost grows with W, so grains whose rows are all narrow (the large grains: nearly a
// chain) use a small W.
//
// PRUNE (heat_opts.prune_eps > 0, threshold 2^-L): a row f is "small" for a cell when both
// X_f < 2^-L max_{i<=f} X_i and X_f Kmax_f < 2^-L max_{i<=f} X_i Kmax_i (Kmax_i: the bin's
// largest emission kernel over the grid), tested on binary exponents.  Once every row of
// the band window [f - width_f, f] is small, the cell's X_f' for f' > f are set to zero:
// X_f' is a combination of the window's values only, so beyond this point the spectrum
// carries no more than a 2^-L share of the probability or of any wavelength's emission,
// unless it grows again (which a steady state past its mode does not).  The decision is per
// cell, so results do not depend on which cells share a warp; the warp leaves the row loop
// once all its cells have stopped.
template <int BUILD, int W, bool PRUNE>
__device__ __forceinline__ void recur_task(const GrainDev& gd, const ChunkDev& ch, int g, int grp, int lane) {
    using Raw = BandRaw<BUILD>;
    const int nbt = gd.nbt;
    const int off = gd.bin_off[g];
    const int M = gd.bin_off[g + 1] - off - 1;
    const int cc = grp * 32 + lane;
    const size_t xb = ((size_t)grp * nbt + off) * 32 + lane;
    const int* rp = gd.rowptr + off + g;
    const double* ic_row = gd.invC + off;
    double* xl = ch.xs + xb;
    const size_t bb = (size_t)grp * gd.band_total * 32 + lane;
    const float* __restrict__ B32 = ch.Bb32 + (BUILD ? bb : 0);
    const double* __restrict__ B64 = ch.Bb64 + (BUILD ? 0 : bb);
    bool numeric_bad = false;

    unsigned short* epl = ch.ep + xb;
    int epoch = 0;
    xl[0] = 1.0;
    epl[0] = 0;
    double total = 1.0;  // running sum of X, rescaled with it
    // running maximum of X (bit pattern: X >= 0 orders as its bits), rescaled with it; it
    // gives the row scale of the packed emissivity operand without another pass over X
    long long xmaxb = __double_as_longlong(1.0);
    // register window: w[k] = X_{f-1-k}; the band's last elements read it instead of
    // reloading what this thread just stored
    double w[W];
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = 0.0;
    w[0] = 1.0;
    // row pipeline: the band bounds, the cooling rate and the window-part B values of row
    // f+1 are loaded while row f is computed
    int e = rp[1];                       // band of row f: elements [e, e1)
    int e1 = rp[2];
    int e2 = M >= 2 ? rp[3] : e1;        // end of row f+1's band
    double ic = ic_row[1];
    typename Raw::T br[W];               // window part of row f: br[k] = B at element e1-1-k
    {
        const int nr = min(e1 - e, W);
#pragma unroll
        for (int k = 0; k < W; ++k) br[k] = (k < nr) ? Raw::load(B32, B64, e1 - 1 - k) : 0;
    }
    const int e_end = rp[M + 1];
    // L2 prefetch of the B stream, kept 16..48 elements ahead: lane k fetches the
    // 128-byte line of element pf + k (lines of all 32 lanes of one element).  Measured on the
    // batched workload: none 6.62 ms, 8 6.37, 16 6.36, 32 6.39, 64 6.47, 128 6.63, 256 6.98 ms
    // (further ahead, the stream pushes the X history out of L2)
    const size_t lane_base = bb - lane;
    int pf = e;
    // tail pruning state: running maxima of the true binary exponents (epoch included) of X
    // and of X Kmax, the last row that was not small, whether this cell has stopped
    const int* kx = gd.kexp + off;
    int xmax = 1023, cmax = 0, last_big = 0, f_last = M;
    bool stopped = false;
    if constexpr (PRUNE) cmax = 1023 + kx[0];
    for (int f = 1; f <= M; ++f) {
        int kf = 0;
        if constexpr (PRUNE) kf = kx[f];
        // next row's loads
        const bool more = f < M;
        const int e3 = f + 2 <= M ? rp[f + 3] : e2;
        const double ic_n = more ? ic_row[f + 1] : 0.0;
        const int nr_n = more ? min(e2 - e1, W) : 0;
        typename Raw::T br_n[W];
#pragma unroll
        for (int k = 0; k < W; ++k) br_n[k] = (k < nr_n) ? Raw::load(B32, B64, e2 - 1 - k) : 0;
        while (pf < e1 + 16 && pf < e_end) {
            int q = pf + lane;
            if (q < e_end) {
                const void* a = BUILD ? (const void*)(ch.Bb32 + lane_base + (size_t)q * 32)
                                      : (const void*)(ch.Bb64 + lane_base + (size_t)q * 32);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
            pf += 32;
        }
        const int width = e1 - e;          // band of row f: j in [f - width, f)
        const int nreg = min(width, W);    // its last nreg elements come from the window
        const int e_mem = e1 - nreg;       // elements before e_mem read X from memory
        // one accumulator, in element order: the SM sub-partition's FP64 unit, shared by the
        // warps on it, is the bound, not this warp's dependent FMA chain
        double S = 0.0;
        if (e < e_mem) {
            int j = f - width;
            // batches of 4 elements, two register sets: the loads of the next batch are in
            // flight while this batch's FMAs run (no register copy waits on a load).  Batches of
            // 4 leave room for 5 resident blocks per SM (20 warps): 6.36 -> 6.27 ms on the
            // batched workload against batches of 8 at 4 blocks (8 at 5 blocks spills: 7.45 ms)
            const int nb = (e_mem - e) >> 2;
            if (nb > 0) {
                typename Raw::T bA[4], bB[4];
                double xA[4], xB[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) bA[k] = Raw::load(B32, B64, e + k);
#pragma unroll
                for (int k = 0; k < 4; ++k) xA[k] = xl[(j + k) * 32];
                int i = 0;
                for (; i + 2 <= nb; i += 2) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) bB[k] = Raw::load(B32, B64, e + 4 + k);
#pragma unroll
                    for (int k = 0; k < 4; ++k) xB[k] = xl[(j + 4 + k) * 32];
#pragma unroll
                    for (int k = 0; k < 4; ++k) S = fma(Raw::wide(bA[k]), xA[k], S);
                    if (i + 2 < nb) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) bA[k] = Raw::load(B32, B64, e + 8 + k);
#pragma unroll
                        for (int k = 0; k < 4; ++k) xA[k] = xl[(j + 8 + k) * 32];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) S = fma(Raw::wide(bB[k]), xB[k], S);
                    e += 8;
                    j += 8;
                }
                if (i < nb) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) S = fma(Raw::wide(bA[k]), xA[k], S);
                    e += 4;
                    j += 4;
                }
            }
            for (; e < e_mem; ++e, ++j) S = fma(band_b<BUILD>(B32, B64, e), xl[j * 32], S);
        }
        window_tail<BUILD, W>(nreg, br, w, S);
        double X = S * ic;
        if (__double2hiint(ic) == 0 && __double2loint(ic) == 0) {  // zero cooling rate
            X = 0.0;
            // S >= 0: non-zero bits, tested on the integer pipe
            if (__double_as_longlong(S) != 0 && !(PRUNE && stopped)) numeric_bad = true;
        }
        if constexpr (PRUNE) {
            if (stopped) {
                X = 0.0;
            } else {
                const int L = ch.prune;
                const int xe = ((__double2hiint(X) >> 20) & 0x7ff) + 800 * epoch;
                const int ce = xe + kf;
                xmax = max(xmax, xe);
                cmax = max(cmax, ce);
                if (!(xe < xmax - L && ce < cmax - L)) last_big = f;
                stopped = last_big < f - width;
            }
        }
        xl[f * 32] = X;
        epl[f * 32] = (unsigned short)epoch;
        total += X;
        xmaxb = max(xmaxb, __double_as_longlong(X));
#pragma unroll
        for (int k = W - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = X;
        if (above_rescale(X)) {
            ++epoch;
            xmaxb = __double_as_longlong(scale_down_800(__longlong_as_double(xmaxb), 1));
            const int lo = more ? (f + 1) - (e2 - e1) : f + 1;  // next row's band start
            // exact power-of-two scaling on the integer pipe (the exponent field lowered by 800)
            for (int i = lo; i <= f; ++i) {
                xl[i * 32] = scale_down_800(xl[i * 32], 1);
                epl[i * 32] = (unsigned short)epoch;
            }
            total = scale_down_800(total, 1);
#pragma unroll
            for (int k = 0; k < W; ++k) w[k] = scale_down_800(w[k], 1);
        }
        if constexpr (PRUNE) {
            if (__all_sync(0xffffffffu, stopped)) {
                f_last = f;
                break;
            }
        }
        // rotate the row pipeline
        e = e1;
        e1 = e2;
        e2 = e3;
        ic = ic_n;
#pragma unroll
        for (int k = 0; k < W; ++k) br[k] = br_n[k];
    }
    if (cc < ch.cells && ch.packA) {
        const double inv = 1.0 / total;
        const double emit = pack_epilogue(gd, ch, g, cc, M, PRUNE ? f_last : M, inv, epoch, xmaxb, xl, epl);
        if (ch.ledger) {
            double* lg = ch.ledger + ((size_t)cc * gd.G + g) * 2;
            lg[0] = ch.pabs[(size_t)cc * gd.G + g];
            lg[1] = emit;
        }
    } else if (cc < ch.cells) {
        const double inv = 1.0 / total;
        double* prow = ch.P + (size_t)cc * ch.ldP + off;
        double emit = 0.0;
        const double* cde = gd.cde + off;
        const int i_end = PRUNE ? f_last : M;
        // scale X first (as the plain rescale would have), then normalise: the factor alone
        // could underflow where the product is still a normal number.  Two loops, so that
        // no predicated-off FMA of the energy check occupies the FP64 unit without a ledger
        if (ch.ledger) {
            for (int i = 0; i <= i_end; ++i) {
                const double p = scale_down_800(xl[i * 32], epoch - (int)epl[i * 32]) * inv;
                prow[i] = p;
                emit = fma(p, cde[i], emit);
            }
        } else {
            for (int i = 0; i <= i_end; ++i) prow[i] = scale_down_800(xl[i * 32], epoch - (int)epl[i * 32]) * inv;
        }
        if constexpr (PRUNE)
            for (int i = f_last + 1; i <= M; ++i) prow[i] = 0.0;  // rows past a pruned tail
        if (ch.ledger) {
            double* lg = ch.ledger + ((size_t)cc * gd.G + g) * 2;
            lg[0] = ch.pabs[(size_t)cc * gd.G + g];
            lg[1] = emit;
        }
    }
    if (numeric_bad) atomicOr(ch.status, kStatNumeric);
}

template <int BUILD, bool PRUNE>
__global__ void __launch_bounds__(128, 5) k_recur(GrainDev gd, ChunkDev ch) {
    for_each_task(ch, 1, [&](int task, int lane) {
        const int g = ch.tasks[task].x, grp = ch.tasks[task].y;
        // window classes 1, 2 and 4 (warp-uniform).  Measured on the batched workload: a class
        // of 8 for rows wider than 4 spilled at the 96 registers of 5 resident blocks (6.26 ms
        // against 6.04-6.10 with 4 the widest; widest 3 or 5 the same, 6 6.33, 7 7.25 ms)
        const int wm = gd.wmax[g];
        if (wm <= 1)
            recur_task<BUILD, 1, PRUNE>(gd, ch, g, grp, lane);
        else if (wm <= 2)
            recur_task<BUILD, 2, PRUNE>(gd, ch, g, grp, lane);
        else
            recur_task<BUILD, 4, PRUNE>(gd, ch, g, grp, lane);
    });
}

// ---------------------------------------------------------------------------
// Recursion for solves of few cells (ChunkDev::small), one block per spectrum: a column
// sweep.  Once X_j is final, every later row f whose band holds j takes B_fj X_j into its
// accumulator, so each row's sum runs in ascending j as in k_recur, and the chain from one X
// to the next is one FMA, the multiply by 1/T_{f-1,f} and a broadcast instead of a row's dot
// product and a cross-lane reduction.  Thread t of the T threads owns rows t, t + T, ...; a
// thread has up to K rows in progress (T above the grain's widest band row and K = 1, one warp
// needing no barrier; or T = 1024 and K = 4); each row in progress keeps in registers its accumulator, its band start
// and element offset, 1/T_{f-1,f} and the B value of the next column (loaded a step ahead),
// and the thread's following rows are loaded a run of 32 columns ahead (off the column chain).
// The thread that completes row j + 1 multiplies, stores X_{j+1} and broadcasts it (a shuffle
// when T = 32, else a shared slot, double-buffered, and one barrier per column).  Rescales
// apply at once to the history, the accumulators and the running sum (exact powers of two);
// normalisation, pruning and the energy check as in k_recur.  The band is staged in shared
// memory when the launch gives room for the largest grain's (`staged`).
template <int BUILD>
struct SmallRow {
    int f, jl, rs;  // row, band start, element of column j at rs + j
    double ic, acc, b;
};
struct SmallRowRaw {  // a row's loads, not yet used (so that nothing waits on them)
    int f, p0, p1;
    double ic;
};

template <int BUILD, bool PRUNE, int K, bool WARP>
__global__ void __launch_bounds__(WARP ? 32 : 1024, 1) k_recur_small(GrainDev gd, ChunkDev ch, int staged) {
    using Raw = BandRaw<BUILD>;
    extern __shared__ double smx[];
    __shared__ double bc[2];  // broadcast: X_{j+1} and the width of its row (double-buffered)
    __shared__ int bcw[2];
    const int T = WARP ? 32 : blockDim.x, tid = threadIdx.x;
    const bool one_warp = WARP;
    const int sp = blockIdx.x;
    const int cell = sp / gd.G, g = sp % gd.G;
    const int grp = cell >> 5, lc = cell & 31;
    const int off = gd.bin_off[g];
    const int M = gd.bin_off[g + 1] - off - 1;
    double* xs = smx;  // X history [max_bins]
    typename Raw::T* bs = (typename Raw::T*)(xs + gd.max_bins);
    const int* rp = gd.rowptr + off + g;
    const double* ic_row = gd.invC + off;
    const size_t bb = (size_t)grp * gd.band_total * 32 + lc;
    const float* B32 = ch.Bb32 + (BUILD ? bb : 0);
    const double* B64 = ch.Bb64 + (BUILD ? 0 : bb);
    const int ebeg = rp[1];
    if (staged) {  // eight independent loads in flight per thread
        const int nel = rp[M + 1] - ebeg;
        for (int e0 = tid; e0 < nel; e0 += 8 * T) {
            typename Raw::T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = e0 + u * T < nel ? Raw::load(B32, B64, ebeg + e0 + u * T) : 0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (e0 + u * T < nel) bs[e0 + u * T] = v[u];
        }
    }
    if (tid == 0) xs[0] = 1.0;
    __syncthreads();
    auto bval = [&](int e) -> double { return staged ? Raw::wide(bs[e]) : band_b<BUILD>(B32, B64, e); };
    auto load_row = [&](int f) {  // row f's loads (unconditional: rows past M load row M's, unused)
        SmallRowRaw r;
        const int fc = f <= M ? f : M;
        r.f = f;
        r.p0 = rp[fc];
        r.p1 = rp[fc + 1];
        r.ic = ic_row[fc];
        return r;
    };
    auto open_row = [&](const SmallRowRaw& q) {  // the row in progress, from its loads
        SmallRow<BUILD> r;
        r.f = q.f;
        r.acc = 0.0;
        r.b = 0.0;
        r.ic = q.f <= M ? q.ic : 0.0;
        r.jl = q.f <= M ? q.f - (q.p1 - q.p0) : 1 << 30;
        r.rs = q.p0 - (q.f - (q.p1 - q.p0)) - (staged ? ebeg : 0);
        return r;
    };
    // Rows: row[] in progress, nxt the one after them (opened), raw the one after that (its
    // loads in flight).  A warp completes rows in runs of 32 columns (lane 0 .. 31); at the end
    // of its run every lane opens raw as nxt and loads the next raw, so no lane reads a
    // register whose load another lane of the warp has just issued (the scoreboard is per warp).
    SmallRow<BUILD> row[K];
    int fnext = tid == 0 ? T : tid;  // row 0 is given (X_0 = 1)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        row[k] = open_row(load_row(fnext));
        fnext += T;
    }
    SmallRow<BUILD> nxt = open_row(load_row(fnext));
    fnext += T;
    SmallRowRaw raw = load_row(fnext);
    fnext += T;
    const int warp = tid >> 5;
    bool used = false;  // nxt was taken in this run
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (row[k].jl <= 0 && 0 < row[k].f) row[k].b = bval(row[k].rs);
    bool numeric_bad = false;
    // X = X_j, the value being spread (uniform); the running sum of X is kept by thread 0 alone
    // (the same additions in the same order as k_recur), off the other warps' FP64 units
    double total = 1.0, X = 1.0;
    const int* kx = gd.kexp + off;
    const int L = ch.prune;
    int xmax = 1023, cmax = PRUNE ? 1023 + kx[0] : 0, last_big = 0, f_last = M, shift = 0;
    for (int j = 0; j < M; ++j) {
        const int f1 = j + 1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            SmallRow<BUILD>& r = row[k];
            const bool act = r.jl <= j && j < r.f;
            const bool act_next = r.jl <= j + 1 && j + 1 < r.f;
            if (K == 1 || __any_sync(0xffffffffu, act || act_next)) {  // no predicated-off FMA on the FP64 unit
                if (act) r.acc = fma(r.b, X, r.acc);
                if (act_next) r.b = bval(r.rs + j + 1);
            }
        }
        double Xn = 0.0;
        int wn = 0;
        if (row[0].f == f1) {  // this thread completes row j + 1
            const double S = row[0].acc;
            Xn = S * row[0].ic;
            if (__double2hiint(row[0].ic) == 0 && __double2loint(row[0].ic) == 0) {
                Xn = 0.0;
                if (__double_as_longlong(S) != 0) numeric_bad = true;  // S >= 0
            }
            wn = f1 - row[0].jl;
            xs[f1] = Xn;
            if (!one_warp) {
                bc[j & 1] = Xn;
                bcw[j & 1] = wn;
            }
#pragma unroll
            for (int k = 0; k + 1 < K; ++k) row[k] = row[k + 1];
            row[K - 1] = nxt;
            used = true;
            if (row[K - 1].jl <= j + 1 && j + 1 < row[K - 1].f) row[K - 1].b = bval(row[K - 1].rs + j + 1);
        }
        if ((f1 & 31) == 31 && ((f1 % T) >> 5) == warp && used) {  // this warp's run ends: refresh
            nxt = open_row(raw);
            raw = load_row(fnext);
            fnext += T;
            used = false;
        }
        if (one_warp) {
            Xn = __shfl_sync(0xffffffffu, Xn, f1 & 31);
            wn = __shfl_sync(0xffffffffu, wn, f1 & 31);
        } else {
            __syncthreads();
            Xn = bc[j & 1];
            wn = bcw[j & 1];
        }
        if (tid == 0) total += Xn;
        bool stop = false;
        if (PRUNE) {  // the same test as k_recur, on uniform values
            const int xe = ((__double2hiint(Xn) >> 20) & 0x7ff) + shift;
            const int ce = xe + kx[f1];
            xmax = max(xmax, xe);
            cmax = max(cmax, ce);
            if (!(xe < xmax - L && ce < cmax - L)) last_big = f1;
            stop = last_big < f1 - wn;
        }
        if (above_rescale(Xn)) {
            if (one_warp) __syncwarp(); else __syncthreads();  // xs[f1] is stored
            for (int i = tid; i <= f1; i += T) xs[i] = scale_down_800(xs[i], 1);
#pragma unroll
            for (int k = 0; k < K; ++k) row[k].acc = scale_down_800(row[k].acc, 1);
            if (tid == 0) total = scale_down_800(total, 1);
            Xn = scale_down_800(Xn, 1);
            shift += 800;
        }
        X = Xn;
        if (stop) {
            f_last = f1;
            break;
        }
    }
    __shared__ double total_s;
    if (tid == 0) total_s = total;
    __syncthreads();
    const double inv = 1.0 / total_s;
    double* prow = ch.P + (size_t)cell * ch.ldP + off;
    double emit = 0.0;
    for (int i = tid; i <= M; i += T) {
        const double p = i <= f_last ? xs[i] * inv : 0.0;
        prow[i] = p;
        emit = fma(p, gd.cde[off + i], emit);
    }
    if (ch.ledger) {
        for (int o = 16; o > 0; o >>= 1) emit += __shfl_xor_sync(0xffffffffu, emit, o);
        __shared__ double wsum[32];
        if ((tid & 31) == 0) wsum[tid >> 5] = emit;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (T >> 5); ++w) t += wsum[w];
            double* lg = ch.ledger + ((size_t)cell * gd.G + g) * 2;
            lg[0] = ch.pabs[(size_t)cell * gd.G + g];
            lg[1] = t;
        }
    }
    numeric_bad = __syncthreads_or(numeric_bad);
    if (numeric_bad && tid == 0) atomicOr(ch.status, kStatNumeric);
}

// Blocks of 128 threads (a warp per task) for the task-list kernels: one per 4 tasks, or, for
// the persistent launches (ch.work set), no more than stay resident on the device at once.
template <typename K>
static unsigned task_grid(K kernel, const ChunkDev& ch) {
    const unsigned full = (unsigned)((ch.n_tasks + 3) / 4);
    if (!ch.work) return full;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 128, 0) != cudaSuccess)
        return full;
    if (ch.blocks_per_sm > 0 && ch.blocks_per_sm < occ) occ = ch.blocks_per_sm;
    const unsigned cap = (unsigned)(sms > 0 && occ > 0 ? sms * occ : 1);
    return full < cap ? full : cap;
}

cudaError_t launch_recur(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st) {
    if (ch.small) {
        const long long spectra = (long long)ch.cells * g.G;
        if (spectra == 0) return cudaSuccess;
        // a multiple of 32 threads above the widest band row (one row in progress per thread;
        // one warp needs no block barrier per column), at most 1024 (then up to four rows per
        // thread).  Measured on the single cell (rows up to 127 wide): one warp with four rows
        // per lane, 97 us; four warps with one, 57 us (the FP64 unit of one sub-partition would
        // carry every row's FMA)
        const int wm = g.wmax_all;
        const int T1 = (wm + 1 + 31) / 32 * 32;
        const bool warp = T1 == 32;
        const int T = std::min(1024, T1);
        const int K = T1 > 1024 ? 4 : 1;
        const size_t base = sizeof(double) * (size_t)g.max_bins;
        const size_t band = (build == 0 ? sizeof(double) : sizeof(float)) * (size_t)g.band_max;
        const int staged = base + band <= kSmallRecurStage ? 1 : 0;
        const size_t smem = base + (staged ? band : 0);
        using KernT = void (*)(GrainDev, ChunkDev, int);
        KernT kern = nullptr;
#define HEAT_SMALL_PICK(B, P) \
    kern = warp ? k_recur_small<B, P, 1, true> : (K == 1 ? k_recur_small<B, P, 1, false> : k_recur_small<B, P, 4, false>)
        if (build == 0) {
            if (ch.prune) HEAT_SMALL_PICK(0, true); else HEAT_SMALL_PICK(0, false);
        } else {
            if (ch.prune) HEAT_SMALL_PICK(1, true); else HEAT_SMALL_PICK(1, false);
        }
#undef HEAT_SMALL_PICK
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<(unsigned)spectra, T, smem, st>>>(g, ch, staged);
        return cudaGetLastError();
    }
    if (ch.n_tasks == 0) return cudaSuccess;
    auto kern = build == 0 ? (ch.prune ? k_recur<0, true> : k_recur<0, false>)
                           : (ch.prune ? k_recur<1, true> : k_recur<1, false>);
    kern<<<task_grid(kern, ch), 128, 0, st>>>(g, ch);
    return cudaGetLastError();
}

}  // namespace heat
