// heat_solve_noalloc: the steady-state distributions P computed without any device
// allocation.
//
// Who needs it: host codes that run the heating calculation under a fixed device-memory
// budget owned by their own allocator (a radiative-transfer code that has carved the GPU
// into pools up front), and time-critical loops that cannot afford cudaMalloc/cudaFree,
// which block until the whole device is idle and so stall every other stream.  Those
// callers set up a heat_ctx once, outside the loop, and afterwards call this entry point,
// which uses only the fixed scratch array below plus the buffers the caller passes.
//
// The scratch array lives for the life of the process on every GPU that loads the
// library.  All calls on a device share it: it keeps whatever the last call left there,
// and two calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and produce garbage.  Serialise them.
#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/heat.h"
#include "common.cuh"
#include "internal.h"

namespace heat {

static __device__ __align__(256) unsigned char g_noalloc_scratch[HEAT_NOALLOC_SCRATCH_BYTES];

// Task list for the no-allocation solve: grain-major (grain, 32-cell group) pairs, one warp
// per task (no task counters).  heat_solve instead runs its recursion persistently over a
// cost-ordered list (longest tasks first); the results are the same, but here large grains
// may start late, so this solve can take longer than heat_solve on the same cells.
__global__ void k_noalloc_tasks(int2* tasks, int G, int NG) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G * NG) tasks[t] = make_int2(t / NG, t % NG);
}

}  // namespace heat

// Defined in heat_api.cu: the grain tables a solve reads and the device status word,
// and the message heat_last_error reports.
heat_status heat_internal_grain_view(heat_ctx* ctx, heat::GrainDev* gd, int* device, int** status);
void heat_internal_fail(heat_ctx* ctx, const char* msg);

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Bytes one 32-cell group needs in the scratch array.
size_t group_bytes(int build, int G, int N, int nbt, long long band) {
    size_t tab = (size_t)band * 32 * (build == HEAT_BUILD_F64 ? sizeof(double) : sizeof(float));
    size_t xs = (size_t)nbt * 32 * (sizeof(double) + sizeof(unsigned short));
    size_t uf = (size_t)N * 32 * 2 * (build == HEAT_BUILD_F64 ? sizeof(double) : sizeof(float));
    size_t tasks = (size_t)G * sizeof(int2);
    return tab + xs + uf + tasks + 9 * 256;  // plus alignment slack of the carve-up
}

}  // namespace

extern "C" heat_status heat_solve_noalloc(heat_ctx* ctx, int build, const double* u_dev, int n_cells, double* P_out,
                                          void* stream) {
    using namespace heat;
    if (!ctx) return HEAT_EINVAL;
    auto fail = [&](heat_status s, const char* msg) {
        heat_internal_fail(ctx, msg);
        return s;
    };
    auto cuda_fail = [&](cudaError_t e, const char* where) {
        std::string m = std::string("heat_solve_noalloc: ") + where + ": " + cudaGetErrorString(e);
        heat_internal_fail(ctx, m.c_str());
        return HEAT_ECUDA;
    };
    if (build != HEAT_BUILD_F64 && build != HEAT_BUILD_F32)
        return fail(HEAT_EINVAL, "heat_solve_noalloc: build must be HEAT_BUILD_F64 or HEAT_BUILD_F32");
    if (n_cells < 0 || (n_cells > 0 && (!u_dev || !P_out)))
        return fail(HEAT_EINVAL, "heat_solve_noalloc: negative cell count or null field/output pointer");
    GrainDev gd;
    int device = 0;
    int* status = nullptr;
    heat_status s = heat_internal_grain_view(ctx, &gd, &device, &status);
    if (s != HEAT_OK) return s;
    if (n_cells == 0) return HEAT_OK;
    if (device < 0 || device >= kMaxDevices)
        return fail(HEAT_EINVAL, "heat_solve_noalloc: device ordinal beyond the supported 64");
    cudaError_t ce = cudaSetDevice(device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");

    // One-time set-up per device: the host-side symbol is only a stand-in, so look up
    // the array's device address with this device current.
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mutex);
        if (!g_addr[device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
            if (!p) return fail(HEAT_ECUDA, "heat_solve_noalloc: null device address of the scratch array");
            g_addr[device] = p;
        }
        base = g_addr[device];
    }

    const int N = gd.N, G = gd.G, nbt = gd.nbt;
    const size_t per_group = group_bytes(build, G, N, nbt, gd.band_total);
    if (per_group > HEAT_NOALLOC_SCRATCH_BYTES) {
        heat_internal_fail(ctx, "heat_solve_noalloc: one 32-cell group of these grains needs more scratch than "
                                "HEAT_NOALLOC_SCRATCH_BYTES (32 MiB); use heat_solve, or fewer grains/bins/wavelengths");
        return HEAT_EINVAL;
    }
    int max_groups = (int)(HEAT_NOALLOC_SCRATCH_BYTES / per_group);
    cudaStream_t st = (cudaStream_t)stream;
    const int ngroups_total = (n_cells + 31) / 32;

    for (int g0 = 0; g0 < ngroups_total; g0 += max_groups) {
        int NG = std::min(max_groups, ngroups_total - g0);
        int Cc = NG * 32;
        int cells = std::min(Cc, n_cells - g0 * 32);
        // carve the scratch array
        unsigned char* p = (unsigned char*)base;
        auto take = [&](size_t bytes) {
            unsigned char* q = p;
            p += align256(bytes);
            return (void*)q;
        };
        ChunkDev ch{};
        ch.small = n_cells <= kSmallCells ? 1 : 0;  // as heat_solve decides
        ch.cells = cells;
        ch.Cc = Cc;
        ch.NG = NG;
        ch.n_tasks = G * NG;
        int2* tasks = (int2*)take(sizeof(int2) * (size_t)G * NG);
        ch.tasks = tasks;
        if (build == HEAT_BUILD_F64) {
            ch.ua64 = (double*)take(sizeof(double) * (size_t)N * Cc);
            ch.su64 = (double*)take(sizeof(double) * (size_t)N * Cc);
            ch.Bb64 = (double*)take(sizeof(double) * (size_t)NG * gd.band_total * 32);
        } else {
            ch.ua32 = (float*)take(sizeof(float2) * (size_t)N * Cc);  // (u, slope) pairs
            ch.Bb32 = (float*)take(sizeof(float) * (size_t)NG * gd.band_total * 32);
        }
        ch.xs = (double*)take(sizeof(double) * (size_t)NG * nbt * 32);
        ch.ep = (unsigned short*)take(sizeof(unsigned short) * (size_t)NG * nbt * 32);
        ch.pabs = nullptr;
        ch.P = P_out + (size_t)g0 * 32 * nbt;
        ch.ldP = nbt;
        ch.status = status;
        if ((size_t)(p - (unsigned char*)base) > HEAT_NOALLOC_SCRATCH_BYTES)
            return fail(HEAT_EINVAL, "heat_solve_noalloc: internal error: scratch carve-up exceeds the array");
        // Every scratch word is written before it is read (tasks, field tables, the B band,
        // intra-bin terms, then X row by row), so nothing needs clearing.
        k_noalloc_tasks<<<(ch.n_tasks + 127) / 128, 128, 0, st>>>(tasks, G, NG);
        if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_fail(ce, "task-list launch");
        if ((ce = launch_field(gd, u_dev, HEAT_F64, (long long)g0 * 32, ch, build, st)) != cudaSuccess)
            return cuda_fail(ce, "field launch");
        if ((ce = launch_build(gd, ch, build, st)) != cudaSuccess) return cuda_fail(ce, "build launch");
        if ((ce = launch_recur(gd, ch, build, st)) != cudaSuccess) return cuda_fail(ce, "recursion launch");
    }
    return HEAT_OK;
}
