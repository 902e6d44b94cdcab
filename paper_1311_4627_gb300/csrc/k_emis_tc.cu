// Emissivity contraction on the tensor cores (Eq. emission, Eq. emission-lambda):
//   j[c][g][n] = 2^{eP[c,g]} 2^{eK[g,n]} sum_k A'_g[c][k] B'_g[n][k]
// with A' = the cell's P of grain g divided by its power-of-two row scale and B' = the
// grain's Planck kernel C_abs B_lambda(T_i) [E_i >= hc/lambda] divided by its power-of-two
// column scale, both rounded to BF16 or TF32.  In the split modes the operands hold the
// bins twice, [P_hi | P_lo] and [K_hi | K_lo]; each stage loads the four tiles of one k block
// once and issues P_hi K_hi + P_hi K_lo + P_lo K_hi into the FP32 accumulator.
//
// tcgen05 GEMM, one persistent CTA per SM, warp-specialised:
//   warp 0 lane 0 : TMA producer (2D tiled loads, 128B swizzle) into a 192 KB smem ring
//                   (4 stages of one A and one B tile, or 2 stages of two each when split)
//   warp 1 lane 0 : MMA issuer (tcgen05.mma cta_group::1, M=128 N=256, FP32 in TMEM)
//   warps 2..5    : epilogue (tcgen05.ld -> scale -> 16-byte stores, one row per lane)
// Two TMEM accumulators (2 x 256 columns) let the epilogue of one tile overlap the MMAs
// of the next.  Every mbarrier wait is bounded; on timeout the kernel flags
// kStatTimeout, drains its own copies and MMAs with bounded waits, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "emis_tc.h"
#include "pack.cuh"
#include "tc_ptx.cuh"

namespace heat {

namespace {

// Tile M = 128 rows (cells) by NT = 256 or 128 columns (wavelengths); the operand ring is
// 192 KB either way: 4 stages of one A and one B tile at NT = 256 (2 when split), 6 at
// NT = 128 (3 when split).
constexpr int kM = 128;
constexpr int kAStage = kM * 128;            // bytes of one A tile: 128 rows x 128 B
constexpr int kRingBytes = 4 * (kAStage + 256 * 128);
constexpr int kMaxStages = 6;
constexpr int kEpiWarps = 4;

}  // namespace

using namespace tc;

namespace {

__device__ __forceinline__ void tile_of(const EmisTcParams& p, int t, int& gi, int& mt, int& nt) {
    int per = p.mtiles * p.ntiles;
    gi = t / per;
    int r = t - gi * per;
    mt = r / p.ntiles;
    nt = r - mt * p.ntiles;
}

}  // namespace

template <bool TF32, bool SPLIT, int kN>
__global__ void __launch_bounds__(192, 1) k_emis_tc(const __grid_constant__ EmisTcParams p) {
    constexpr int NP = SPLIT ? 2 : 1;                        // operand parts (hi, lo)
    constexpr int kBStage = kN * 128;                        // bytes of one B tile: kN rows x 128 B
    constexpr int kStageBytes = NP * (kAStage + kBStage);
    constexpr int kStages = kRingBytes / kStageBytes;
    constexpr uint32_t kTmemCols = 2 * kN;                   // two accumulators
    static_assert(kStages >= 2 && kStages <= kMaxStages, "operand ring");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage s: A parts at s * kStageBytes + q * kAStage, B parts after the NP A tiles
    uint64_t* bars = (uint64_t*)(smem + kRingBytes);
    // bars: full[kStages], empty[kStages], tfull[2], tempty[2], done
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kStages + 5);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + kStages);
    const uint32_t b_tfull = smem_u32(bars + 2 * kStages), b_tempty = smem_u32(bars + 2 * kStages + 2);
    const uint32_t b_done = smem_u32(bars + 2 * kStages + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(b_tfull + 8 * a, 1);
            mbar_init(b_tempty + 8 * a, kEpiWarps);
        }
        mbar_init(b_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int total = p.ng * p.mtiles * p.ntiles;
    const int KE = TF32 ? 32 : 64;  // elements per 128-byte k slice

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[kStages];
            for (int s = 0; s < kStages; ++s) last_phase[s] = -1;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                int gi, mt, nt;
                tile_of(p, t, gi, mt, nt);
                const int khalf = p.ksteps[gi] * KE;  // elements of one operand part
                for (int ks = 0; ks < p.ksteps[gi]; ++ks) {
                    if (!mbar_wait(b_empty + 8 * stage, phase ^ 1, abort_flag, p.wait_polls)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(b_full + 8 * stage, kStageBytes);
                    unsigned char* sb = smem + stage * kStageBytes;
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        tma_load_2d(smem_u32(sb + q * kAStage), &p.ta[gi], q * khalf + ks * KE, mt * kM,
                                    b_full + 8 * stage);
                        tma_load_2d(smem_u32(sb + NP * kAStage + q * kBStage), &p.tb[gi], q * khalf + ks * KE,
                                    nt * kN, b_full + 8 * stage);
                    }
                    last_phase[stage] = (int)phase;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (!ok) {
                atomicOr(p.status, kStatTimeout);
                *abort_flag = 1;
            }
            // every copy this thread issued has landed before the CTA may exit
            for (int s = 0; s < kStages; ++s)
                if (last_phase[s] >= 0) {
                    for (long long i = 0; i < kTcSpinLimit; ++i)
                        if (mbar_try(b_full + 8 * s, (uint32_t)last_phase[s])) break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            const uint32_t id = idesc(TF32 ? 2 : 1, kM, kN);
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                int gi, mt, nt;
                tile_of(p, t, gi, mt, nt);
                if (!mbar_wait(b_tempty + 8 * acc, acc_phase ^ 1, abort_flag, p.wait_polls)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)acc * kN;
                for (int ks = 0; ks < p.ksteps[gi]; ++ks) {
                    if (!mbar_wait(b_full + 8 * stage, phase, abort_flag, p.wait_polls)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    unsigned char* sb = smem + stage * kStageBytes;
                    const uint64_t a_hi = sdesc(smem_u32(sb));
                    const uint64_t b_hi = sdesc(smem_u32(sb + NP * kAStage));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma<TF32>(d, a_hi + 2 * kk, b_hi + 2 * kk, id, (ks | kk) != 0 ? 1u : 0u);
                    if constexpr (SPLIT) {
                        const uint64_t a_lo = sdesc(smem_u32(sb + kAStage));
                        const uint64_t b_lo = sdesc(smem_u32(sb + NP * kAStage + kBStage));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) umma<TF32>(d, a_hi + 2 * kk, b_lo + 2 * kk, id, 1u);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) umma<TF32>(d, a_lo + 2 * kk, b_hi + 2 * kk, id, 1u);
                    }
                    umma_commit(b_empty + 8 * stage);
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(b_tfull + 8 * acc);
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            }
            if (!ok) {
                atomicOr(p.status, kStatTimeout);
                *abort_flag = 1;
            }
            // all MMAs this thread issued have completed before TMEM is freed
            umma_commit(b_done);
            for (long long i = 0; i < kTcSpinLimit; ++i)
                if (mbar_try(b_done, 0)) break;
        }
    } else {
        // ---------------- epilogue: warps 2..5 own TMEM lane quarters (warp % 4); lane = row
        // of the tile.  Each lane scales its 32 columns of a chunk and writes them as eight
        // 16-byte stores (one 128-byte run per row); the column scales are broadcast loads.
        const int q = warp & 3;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            int gi, mt, nt;
            tile_of(p, t, gi, mt, nt);
            bool ok = __all_sync(0xffffffffu, mbar_wait(b_tfull + 8 * acc, acc_phase, abort_flag, p.wait_polls));
            if (!ok) {  // warp-uniform: the tcgen05.ld below is a warp-wide instruction
                if (lane == 0) {
                    atomicOr(p.status, kStatTimeout);
                    *abort_flag = 1;
                }
                break;
            }
            tc_fence_after();
            const int g = p.grain[gi];
            const int row = mt * kM + q * 32 + lane;
            const bool rok = row < p.cells;
            const float rs = rok ? p.rowscale[(size_t)row * p.G + g] : 0.0f;
            const size_t jrow = (size_t)(rok ? row : 0) * p.ldj + (size_t)g * p.N;
            const float* csg = p.colscale + (size_t)g * p.N;
            for (int c = 0; c < kN / 32; ++c) {
                uint32_t v[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kN + c * 32), v);
                const int col0 = nt * kN + c * 32;
                if (col0 >= p.N) continue;
                float* dst = (float*)p.j + jrow + col0;
                const bool fast = !p.j_f64 && col0 + 32 <= p.N &&
                                  __all_sync(0xffffffffu, ((uintptr_t)dst & 15u) == 0 && ((uintptr_t)(csg + col0) & 15u) == 0);
                if (fast) {
                    const float4* cs4 = (const float4*)(csg + col0);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float4 cs = cs4[k];
                        float4 o;
                        o.x = __uint_as_float(v[4 * k]) * rs * cs.x;
                        o.y = __uint_as_float(v[4 * k + 1]) * rs * cs.y;
                        o.z = __uint_as_float(v[4 * k + 2]) * rs * cs.z;
                        o.w = __uint_as_float(v[4 * k + 3]) * rs * cs.w;
                        if (rok) __stcs((float4*)dst + k, o);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int col = col0 + i;
                        if (rok && col < p.N) {
                            const float val = __uint_as_float(v[i]);
                            const float cs = csg[col];
                            const size_t o = jrow + col;
                            if (p.j_f64)
                                ((double*)p.j)[o] = (double)val * (double)rs * (double)cs;
                            else
                                ((float*)p.j)[o] = val * rs * cs;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_tempty + 8 * acc);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1;
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kTmemCols)
                     : "memory");
    }
}

size_t emis_tc_smem_bytes() { return 1024 + (size_t)kRingBytes + (2 * kMaxStages + 5) * 8 + 16; }

template <bool TF32, bool SPLIT, int NT>
static cudaError_t launch_emis_tc_t(const EmisTcParams& p, int grid, size_t smem, cudaStream_t st) {
    // the shared-memory opt-in is set once per device (not a stream operation, but kept out
    // of the launch path so that a solve can be captured into a CUDA graph)
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_emis_tc<TF32, SPLIT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    k_emis_tc<TF32, SPLIT, NT><<<grid, 192, smem, st>>>(p);
    return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_emis_tc_nt(const EmisTcParams& p, bool tf32, bool split, int grid, size_t smem,
                                     cudaStream_t st) {
    if (tf32)
        return split ? launch_emis_tc_t<true, true, NT>(p, grid, smem, st)
                     : launch_emis_tc_t<true, false, NT>(p, grid, smem, st);
    return split ? launch_emis_tc_t<false, true, NT>(p, grid, smem, st)
                 : launch_emis_tc_t<false, false, NT>(p, grid, smem, st);
}

cudaError_t launch_emis_tc(const EmisTcParams& p, bool tf32, bool split, int ntile, int sms, cudaStream_t st) {
    int total = p.ng * p.mtiles * p.ntiles;
    if (total <= 0) return cudaSuccess;
    size_t smem = emis_tc_smem_bytes();
    int grid = total < sms ? total : sms;
    if (ntile == 128) return launch_emis_tc_nt<128>(p, tf32, split, grid, smem, st);
    if (ntile == 256) return launch_emis_tc_nt<256>(p, tf32, split, grid, smem, st);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Operand packing.

// Split a value already scaled into [0, 1] into hi + lo for the operand format.
__device__ __forceinline__ void split_bf16(double v, uint16_t& hi, uint16_t& lo) {
    hi = bf16_rn((float)v);
    lo = bf16_rn((float)(v - (double)bf16_f(hi)));
}
__device__ __forceinline__ void split_tf32(double v, float& hi, float& lo) {
    hi = tf32_rn((float)v);
    lo = tf32_rn((float)(v - (double)hi));
}

__device__ __forceinline__ int scale_exp(double m) {
    // smallest e with m / 2^e < 1 (m > 0); 0 for m == 0
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);
    return e;
}

// A' for one chunk: one warp per (cell, grain).  P [cells][nbt] FP64 in, per grain
// A'_g [cells][Kp_g] (BF16 or TF32-in-FP32; [P_hi | P_lo] when split) out, and rowscale [cells][G] = 2^e with e
// the smallest exponent for which the row's largest P divided by 2^e is below 1.
__global__ void k_pack_p(int cells, int G, const int* __restrict__ bin_off, const double* __restrict__ P,
                         long long ldP, const long long* __restrict__ aoff, const int* __restrict__ kp, int split,
                         int tf32, void* __restrict__ A, float* __restrict__ rowscale) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= (long long)cells * G) return;
    int c = (int)(w / G), g = (int)(w % G);
    int off = bin_off[g], nb = bin_off[g + 1] - off;
    const double* pr = P + (size_t)c * ldP + off;
    // the largest high word has the largest exponent (P >= 0: bit patterns order as values)
    unsigned mh = 0;
    for (int i = lane; i < nb; i += 32) mh = max(mh, (unsigned)__double2hiint(pr[i]));
    mh = __reduce_max_sync(0xffffffffu, mh);
    const int e = row_scale_exp(mh);
    if (lane == 0) rowscale[(size_t)c * G + g] = ldexpf(1.0f, e);
    const int K = kp[g], half = split ? K / 2 : K;  // [hi | lo], each part half wide
    if (tf32) {
        float* row = (float*)A + aoff[g] + (size_t)c * K;
        for (int i = lane; i < half; i += 32) {
            const float v = i < nb ? scaled_to_f32(pr[i], e) : 0.0f;
            const float hi = tf32_rn(v);
            row[i] = hi;
            if (split) row[half + i] = tf32_rn(v - hi);
        }
    } else {
        uint16_t* row = (uint16_t*)A + aoff[g] + (size_t)c * K;
        for (int i = lane; i < half; i += 32) {
            const float v = i < nb ? scaled_to_f32(pr[i], e) : 0.0f;
            const uint16_t hi = bf16_rn(v);
            row[i] = hi;
            if (split) row[half + i] = bf16_rn(v - bf16_f(hi));
        }
    }
}

// B' of every grain: one thread per (grain, wavelength).  K [nbt][N] FP64 in, per grain
// B'_g [N][Kp_g] with parts [K_hi | K_lo] (split) or [K_hi], and colscale [G][N].
__global__ void k_pack_k(int N, int G, const int* __restrict__ bin_off, const double* __restrict__ K,
                         const long long* __restrict__ boff, const int* __restrict__ kp, int split, int tf32,
                         void* __restrict__ B, float* __restrict__ colscale) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)G * N) return;
    int g = (int)(idx / N), n = (int)(idx % N);
    int off = bin_off[g], nb = bin_off[g + 1] - off;
    double m = 0.0;
    for (int i = 0; i < nb; ++i) m = fmax(m, K[(size_t)(off + i) * N + n]);
    int e = scale_exp(m);
    double inv = ldexp(1.0, -e);
    colscale[(size_t)g * N + n] = ldexpf(1.0f, e);
    const int Kp = kp[g], half = split ? Kp / 2 : Kp;  // [K_hi | K_lo], each part half wide
    if (tf32) {
        float* row = (float*)B + boff[g] + (size_t)n * Kp;
        for (int i = 0; i < half; ++i) {
            float hi = 0.0f, lo = 0.0f;
            if (i < nb) split_tf32(K[(size_t)(off + i) * N + n] * inv, hi, lo);
            row[i] = hi;
            if (split) row[half + i] = lo;
        }
    } else {
        uint16_t* row = (uint16_t*)B + boff[g] + (size_t)n * Kp;
        for (int i = 0; i < half; ++i) {
            uint16_t hi = 0, lo = 0;
            if (i < nb) split_bf16(K[(size_t)(off + i) * N + n] * inv, hi, lo);
            row[i] = hi;
            if (split) row[half + i] = lo;
        }
    }
}

cudaError_t launch_pack_p(int cells, int G, const int* bin_off, const double* P, long long ldP, const long long* aoff,
                          const int* kp, int split, int tf32, void* A, float* rowscale, cudaStream_t st) {
    long long warps = (long long)cells * G;
    if (warps <= 0) return cudaSuccess;
    int threads = 256;
    long long blocks = (warps * 32 + threads - 1) / threads;
    k_pack_p<<<(unsigned)blocks, threads, 0, st>>>(cells, G, bin_off, P, ldP, aoff, kp, split, tf32, A, rowscale);
    return cudaGetLastError();
}

cudaError_t launch_pack_k(int N, int G, const int* bin_off, const double* K, const long long* boff, const int* kp,
                          int split, int tf32, void* B, float* colscale, cudaStream_t st) {
    long long total = (long long)G * N;
    int threads = 128;
    k_pack_k<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(N, G, bin_off, K, boff, kp, split, tf32,
                                                                            B, colscale);
    return cudaGetLastError();
}

}  // namespace heat
