// The mixed path's matrix build fused into the Guhathakurta-Draine recursion (Eq. xf): a
// persistent lane-per-cell kernel (warp = grain x 32 cells) that never writes the B band.
//
// Per task, first a prologue walks the wavelength segments once in each direction, as the
// separate build does:
//   forward:  the photon prefix Phi_n = (1/h) sum_{m<n} int_m Omega lambda (compensated FP32)
//             at the start of every segment, stored per lane in the warp's table phs[n]
//             (FP32; its sign bit carries the segment's short-series flag), Phi at the
//             grid's end in phs[N-1] and 0 in phs[N];
//   backward: the intra-bin terms W_j / (E_{j+1} - E_j) (Eq. bmatrix's diagonal), parked in
//             the X-history slot of row j+1, which the recursion reads before it writes X_{j+1}
//             there; and the absorbed power for the energy check.
// Then the recursion runs row by row over the band as k_recur does, except that each B value
// is made where it is used, B_fj = phs[n] + u_n cat E1(fmaf(su_n, t, zt)), from the
// row-ordered element table (n, t, cat, zt) and the cell's prefix and field values at
// segment n.  Those per-lane values are gathered ahead of use by asynchronous copies
// (cp.async) into a per-warp staging ring in shared memory, in groups of 8 elements, one
// group ahead of the group being consumed; the element entries arrive the same way, 32 at a
// time, and are read by all lanes from shared memory.  No register waits on a gather, and
// the recursion's own loop is unchanged.  The element expressions, the order of every sum
// and the recursion's FMA order are those of k_build<F32> + k_recur, so the result is bit
// for bit the same; only the 4 bytes per element and cell of the B band (written once, read
// once) are gone.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace heat {

namespace {

constexpr int kGroup = 8;     // elements per staged group
constexpr int kStage = 32;    // staged elements per warp (4 groups: one being consumed, one
                              // straddled by a batch, one in flight, one free)
constexpr int kWarps = 4;     // warps per block
constexpr int kBlocksPerSm = 4;

// Per-warp shared memory: staged prefix values [kStage][32], staged field values
// [kStage][32] and two blocks of 32 element entries.
struct WarpStage {
    float phi[kStage * 32];
    float2 us[kStage * 32];
    int4 ent[2 * 32];
};
constexpr size_t kSmemBytes = sizeof(WarpStage) * kWarps;

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// x * 2^(-800 d) for x >= 0 on the integer pipe (the exponent field lowered), zero below
// the normal range; the same operation as k_recur's rescale.
__device__ __forceinline__ double scale_down(double x, int d) {
    const long long bits = __double_as_longlong(x);
    const long long e = (bits >> 52) - 800LL * d;
    return (d == 0) ? x : (e > 0 ? __longlong_as_double(bits - ((800LL * d) << 52)) : 0.0);
}

// FP32 bits parked in an FP64 slot of the X history (the slot is overwritten with X later)
__device__ __forceinline__ double park(float v) { return __longlong_as_double((long long)__float_as_uint(v)); }
__device__ __forceinline__ float unpark(double x) { return __uint_as_float((unsigned)__double_as_longlong(x)); }

// The cell's B value of one element: the expression of k_build<F32> (short series where the
// segment's flag, the sign bit of its prefix entry, says so).
// en = (n, t, cat, zt) of a RowEnt32 as one 16-byte load.  The short series serves nearly every
// segment of smooth fields; when it serves every lane the warp skips the general form (each
// lane's value is the same either way).
__device__ __noinline__ float e1f_mixed(bool sh, float z) { return sh ? e1f_small(z) : e1f(z); }

__device__ __forceinline__ float element_b(int4 en, float ph, float2 us) {
    const float z = fmaf(us.y, __int_as_float(en.y), __int_as_float(en.w));
    const bool sh = signbit(ph);
    const float E = __all_sync(0xffffffffu, sh) ? e1f_small(z) : e1f_mixed(sh, z);
    return fmaf(us.x * __int_as_float(en.z), E, fabsf(ph));
}

// Issue the asynchronous copies of staged group k (its elements' prefix and field values,
// and with every fourth group the next block of element entries).
__device__ __noinline__ void issue_group(int k, int lane, int e_begin, int N, int Cc, const RowEnt32* ents,
                                         const float* phs, const float2* uasu, WarpStage& sm);

__device__ __noinline__ void issue_group(int k, int lane, int e_begin, int N, int Cc, const RowEnt32* ents,
                                         const float* phs, const float2* uasu, WarpStage& sm) {
    if ((k & 3) == 2) {
        const int b = (k >> 2) + 1;
        cp_async16(&sm.ent[(b & 1) * 32 + lane], ents + e_begin + b * 32 + lane);
    }
    const int4* eb = sm.ent + ((k >> 2) & 1) * 32 + ((k & 3) << 3);
#pragma unroll
    for (int t = 0; t < kGroup; ++t) {
        const int n = eb[t].x;
        const int slot = ((k << 3) + t) & (kStage - 1);
        cp_async4(&sm.phi[slot * 32 + lane], phs + (size_t)n * 32);
        cp_async8(&sm.us[slot * 32 + lane], uasu + (size_t)min(n, N - 1) * Cc);
    }
    cp_async_commit();
}

// Prologue of one task: the prefix table, the parked intra-bin terms, the absorbed power.
__device__ __noinline__ double prologue(const GrainDev& gd, const ChunkDev& ch, int g, int cc, float* phs,
                                           double* xl) {
    const int N = gd.N, Cc = ch.Cc;
    const float* ca = gd.ca32 + (size_t)g * N;
    const float* ce = gd.ce32 + (size_t)g * N;
    const float* sC = gd.sC32 + (size_t)g * N;
    const float2* uasu = (const float2*)ch.ua32;
    const int off = gd.bin_off[g];
    // forward walk, field values loaded eight segments at a time, a batch ahead
    Sum32 Phi32;
    constexpr int PB = 8;
    float2 ua_[PB], ub_[PB];
#pragma unroll
    for (int k = 0; k < PB; ++k) ua_[k] = k < N - 1 ? uasu[(size_t)k * Cc + cc] : make_float2(0.0f, 0.0f);
    for (int n0 = 0; n0 < N - 1; n0 += PB) {
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int n = n0 + PB + k;
            ub_[k] = n < N - 1 ? uasu[(size_t)n * Cc + cc] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int n = n0 + k;
            if (n < N - 1) {
                const float ua = ua_[k].x, su = ua_[k].y;
                const float phi = Phi32.val();
                const float dl = gd.dln32[n];
                phs[(size_t)n * 32] = short_series(su, sC[n], dl) ? -phi : phi;
                const float a = ua * ca[n];
                if (a > 0.0f) Phi32.add(a * dl * e1f((su + sC[n] + 2.0f) * dl));
            }
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) ua_[k] = ub_[k];
    }
    phs[(size_t)(N - 1) * 32] = Phi32.val();
    phs[(size_t)N * 32] = 0.0f;

    // backward walk: intra-bin terms (soft-photon list of the grain, by segment descending)
    const SoftF64* soft = gd.soft;
    int p = gd.soft_off[g];
    const int p1 = gd.soft_off[g + 1];
    while (p < p1 && soft[p].n == N - 1) {
        xl[(size_t)(soft[p].j + 1) * 32] = park(0.0f);
        ++p;
    }
    Sum32 Psi32;  // c int Omega from lambda_{n+1} to lambda_{N-1}
    // segments N-2 down to 0, field values loaded eight at a time, a batch ahead
#pragma unroll
    for (int k = 0; k < PB; ++k) {
        const int n = N - 2 - k;
        ua_[k] = n >= 0 ? uasu[(size_t)n * Cc + cc] : make_float2(0.0f, 0.0f);
    }
    for (int nt = N - 2; nt >= 0; nt -= PB) {
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int n = nt - PB - k;
            ub_[k] = n >= 0 ? uasu[(size_t)n * Cc + cc] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int n = nt - k;
            if (n >= 0) {
                const float ua = ua_[k].x, su = ua_[k].y;
                const float b = ua * ce[n];
                const float q0 = su + sC[n] + 1.0f;
                const float dl = gd.dln32[n];
                while (p < p1 && soft[p].n == n) {
                    const SoftF64 sf = soft[p];
                    float part = 0.0f;
                    if (b > 0.0f) {
                        const float ts = (float)sf.t;
                        const float L = dl - ts;
                        part = b * __expf(q0 * ts) * L * e1f(q0 * L);
                    }
                    xl[(size_t)(sf.j + 1) * 32] = park((part + Psi32.val()) * gd.invdE32[off + sf.j]);
                    ++p;
                }
                if (b > 0.0f) Psi32.add(b * dl * e1f(q0 * dl));
            }
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) ua_[k] = ub_[k];
    }
    const float psi_end = Psi32.val();
    for (; p < p1; ++p) xl[(size_t)(soft[p].j + 1) * 32] = park(psi_end * gd.invdE32[off + soft[p].j]);
    return Psi32.wide();
}

// One task of the fused kernel: prologue, then the recursion of grain g for the 32 cells of
// group grp (lane = cell) with the B values made on the fly.  The recursion's structure is
// k_recur's: register window of the last W values of X, one accumulator per row in element
// order, lazy power-of-two rescaling with per-value epochs, tail pruning.
template <int W, bool PRUNE>
__device__ __forceinline__ void fused_task(const GrainDev& gd, const ChunkDev& ch, int g, int grp, int lane,
                                           float* phs, WarpStage& sm) {
    const int nbt = gd.nbt, N = gd.N, Cc = ch.Cc;
    const int off = gd.bin_off[g];
    const int M = gd.bin_off[g + 1] - off - 1;
    const int cc = grp * 32 + lane;
    const size_t xb = ((size_t)grp * nbt + off) * 32 + lane;
    const int* rp = gd.rowptr + off + g;
    const double* ic_row = gd.invC + off;
    double* xl = ch.xs + xb;
    unsigned short* epl = ch.ep + xb;
    const float2* uasu = (const float2*)ch.ua32 + cc;
    const RowEnt32* __restrict__ ents = gd.rent;

    const double pabs = prologue(gd, ch, g, cc, phs, xl);

    // Staging: element e (counted from e_begin, x = e - e_begin) has its gathered prefix and
    // field values at slot x % kStage and its entry in block (x / 32) % 2; group k holds
    // x in [8k, 8k + 8).  Groups below `ready` have landed; groups below `issued` are in
    // flight or landed.  ensure(e) issues at most one group past e's, so when group k is
    // issued the elements still to be read lie in groups k-2 and k-1: group k may reuse the
    // slots of group k-4, and entry block b + 1 may replace block b - 1 from group 4b + 2 on,
    // which is two groups before its first use (issuing group 4b + 4).  The table is padded
    // past its end (more than two blocks), so whole groups and blocks may pass e_end.
    const int e_begin = rp[1];
    __threadfence_block();  // the prologue's table writes precede the copies that read them
    cp_async16(&sm.ent[lane], ents + e_begin + lane);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    int issued = 0, ready = 0;
    auto issue = [&](int k) { issue_group(k, lane, e_begin, N, Cc, ents, phs, uasu, sm); };
    // make every element up to e (inclusive) readable
    auto ensure = [&](int e_last) {
        const int gx = (e_last - e_begin) >> 3;
        while (ready <= gx) {
            while (issued <= ready + 1) issue(issued++);
            cp_async_wait<1>();  // all but the newest group have landed
            __syncwarp();        // entry blocks are written by all lanes
            ++ready;
        }
    };
    auto stage_b = [&](int e) {
        const int x = e - e_begin;
        const int slot = x & (kStage - 1);
        const int4 en = sm.ent[((x >> 5) & 1) * 32 + (x & 31)];
        return element_b(en, sm.phi[slot * 32 + lane], sm.us[slot * 32 + lane]);
    };
    auto ring_b = [&](int e) { return widen_pos(stage_b(e)); };

    bool numeric_bad = false;
    int epoch = 0;
    // row 1's intra-bin term was parked in slot 1; X_0 = 1 overwrites nothing of use
    float soft = unpark(xl[32]);
    xl[0] = 1.0;
    epl[0] = 0;
    double total = 1.0;
    double w[W];
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = 0.0;
    w[0] = 1.0;
    int e = rp[1];
    int e1 = rp[2];
    int e2 = M >= 2 ? rp[3] : e1;
    double ic = ic_row[1];
    const int* kx = gd.kexp + off;
    int xmax = 1023, cmax = 0, last_big = 0, f_last = M;
    bool stopped = false;
    if constexpr (PRUNE) cmax = 1023 + kx[0];
    for (int f = 1; f <= M; ++f) {
        int kf = 0;
        if constexpr (PRUNE) kf = kx[f];
        const bool more = f < M;
        const int e3 = f + 2 <= M ? rp[f + 3] : e2;
        const double ic_n = more ? ic_row[f + 1] : 0.0;
        const float soft_n = more ? unpark(xl[(size_t)(f + 1) * 32]) : 0.0f;  // row f+1's intra-bin term
        const int width = e1 - e;
        const int nreg = min(width, W);
        const int e_mem = e1 - nreg;
        double S = 0.0;
        if (e < e_mem) {
            int j = f - width;
            const int nb = (e_mem - e) >> 3;
            if (nb > 0) {
                double xA[8], xB[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) xA[k] = xl[(j + k) * 32];
                int i = 0;
                for (; i + 2 <= nb; i += 2) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) xB[k] = xl[(j + 8 + k) * 32];
                    ensure(e + 7);
#pragma unroll
                    for (int k = 0; k < 8; ++k) S = fma(ring_b(e + k), xA[k], S);
                    if (i + 2 < nb) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) xA[k] = xl[(j + 16 + k) * 32];
                    }
                    ensure(e + 15);
#pragma unroll
                    for (int k = 0; k < 8; ++k) S = fma(ring_b(e + 8 + k), xB[k], S);
                    e += 16;
                    j += 16;
                }
                if (i < nb) {
                    ensure(e + 7);
#pragma unroll
                    for (int k = 0; k < 8; ++k) S = fma(ring_b(e + k), xA[k], S);
                    e += 8;
                    j += 8;
                }
            }
            if (e < e_mem) ensure(e_mem - 1);
            for (; e < e_mem; ++e, ++j) S = fma(ring_b(e), xl[j * 32], S);
        }
        // window part: element e1-1-k multiplies X_{f-1-k} = w[k]; k = 0 is the diagonal,
        // which carries the intra-bin term (added in FP32, as the separate build does)
        {
            ensure(e1 - 1);
            double bw[W];
#pragma unroll
            for (int k = 0; k < W; ++k) bw[k] = 0.0;
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < nreg) {
                    const float r = stage_b(e1 - 1 - k);
                    bw[k] = widen_pos(k == 0 ? r + soft : r);
                }
            switch (nreg) {
                case 8: if constexpr (W > 7) S = fma(bw[7 % W], w[7 % W], S);  // fallthrough
                case 7: if constexpr (W > 6) S = fma(bw[6 % W], w[6 % W], S);  // fallthrough
                case 6: if constexpr (W > 5) S = fma(bw[5 % W], w[5 % W], S);  // fallthrough
                case 5: if constexpr (W > 4) S = fma(bw[4 % W], w[4 % W], S);  // fallthrough
                case 4: if constexpr (W > 3) S = fma(bw[3 % W], w[3 % W], S);  // fallthrough
                case 3: if constexpr (W > 2) S = fma(bw[2 % W], w[2 % W], S);  // fallthrough
                case 2: if constexpr (W > 1) S = fma(bw[1 % W], w[1 % W], S);  // fallthrough
                case 1: S = fma(bw[0], w[0], S);                               // fallthrough
                default: break;
            }
        }
        double X = S * ic;
        if (__double2hiint(ic) == 0 && __double2loint(ic) == 0) {
            X = 0.0;
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
#pragma unroll
        for (int k = W - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = X;
        if (above_rescale(X)) {
            ++epoch;
            const int lo = more ? (f + 1) - (e2 - e1) : f + 1;
            for (int i = lo; i <= f; ++i) {
                xl[i * 32] = scale_down(xl[i * 32], 1);
                epl[i * 32] = (unsigned short)epoch;
            }
            total = scale_down(total, 1);
#pragma unroll
            for (int k = 0; k < W; ++k) w[k] = scale_down(w[k], 1);
        }
        if constexpr (PRUNE) {
            if (__all_sync(0xffffffffu, stopped)) {
                f_last = f;
                break;
            }
        }
        e = e1;
        e1 = e2;
        e2 = e3;
        ic = ic_n;
        soft = soft_n;
    }
    if (cc < ch.cells) {
        const double inv = 1.0 / total;
        double* prow = ch.P + (size_t)cc * ch.ldP + off;
        double emit = 0.0;
        const double* cde = gd.cde + off;
        const int i_end = PRUNE ? f_last : M;
        if (ch.ledger) {
            for (int i = 0; i <= i_end; ++i) {
                const double pv = scale_down(xl[i * 32], epoch - (int)epl[i * 32]) * inv;
                prow[i] = pv;
                emit = fma(pv, cde[i], emit);
            }
        } else {
            for (int i = 0; i <= i_end; ++i) prow[i] = scale_down(xl[i * 32], epoch - (int)epl[i * 32]) * inv;
        }
        if constexpr (PRUNE)
            for (int i = f_last + 1; i <= M; ++i) prow[i] = 0.0;
        if (ch.pabs) ch.pabs[(size_t)cc * gd.G + g] = pabs;
        if (ch.ledger) {
            double* lg = ch.ledger + ((size_t)cc * gd.G + g) * 2;
            lg[0] = pabs;
            lg[1] = emit;
        }
    }
    if (numeric_bad) atomicOr(ch.status, kStatNumeric);
}

template <bool PRUNE>
__global__ void __launch_bounds__(kWarps * 32, kBlocksPerSm) k_fused(GrainDev gd, ChunkDev ch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStage& sm = ((WarpStage*)smem_raw)[warp];
    float* phs = ch.phs + ((size_t)blockIdx.x * kWarps + warp) * (size_t)(gd.N + 1) * 32 + lane;
    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(ch.work + 1, 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= ch.n_tasks) return;
        const int g = ch.tasks[task].x, grp = ch.tasks[task].y;
        const int wm = gd.wmax[g];  // warp-uniform
        if (wm <= 1)
            fused_task<1, PRUNE>(gd, ch, g, grp, lane, phs, sm);
        else if (wm <= 2)
            fused_task<2, PRUNE>(gd, ch, g, grp, lane, phs, sm);
        else if (wm <= 4)
            fused_task<4, PRUNE>(gd, ch, g, grp, lane, phs, sm);
        else
            fused_task<8, PRUNE>(gd, ch, g, grp, lane, phs, sm);
    }
}

int resident_blocks() {
    static int cache[64] = {};
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[dev]) return cache[dev];
    if (cudaFuncSetAttribute(k_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<false>, kWarps * 32, kSmemBytes) != cudaSuccess)
        return 0;
    int occ2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_fused<true>, kWarps * 32, kSmemBytes) != cudaSuccess)
        return 0;
    cache[dev] = sms * std::max(1, std::min(occ, occ2));
    return cache[dev];
}

}  // namespace

int fused_warps(int n_tasks) {
    const int full = (n_tasks + kWarps - 1) / kWarps;
    const int cap = resident_blocks();
    if (cap <= 0) return 0;
    return std::min(full, cap) * kWarps;
}

cudaError_t launch_fused(const GrainDev& g, const ChunkDev& ch, cudaStream_t st) {
    if (ch.n_tasks == 0) return cudaSuccess;
    if (!ch.work || !ch.phs) return cudaErrorInvalidValue;
    const int warps = fused_warps(ch.n_tasks);
    if (warps <= 0) return cudaErrorInvalidConfiguration;
    const unsigned blocks = (unsigned)(warps / kWarps);
    if (ch.prune)
        k_fused<true><<<blocks, kWarps * 32, kSmemBytes, st>>>(g, ch);
    else
        k_fused<false><<<blocks, kWarps * 32, kSmemBytes, st>>>(g, ch);
    return cudaGetLastError();
}

}  // namespace heat
