// Kernels of the learned surrogate (an MLP ensemble over the binned field):
//   k_gemm_bf16   tcgen05 GEMM  C[z] = A[z] . B[z]^T (+ bias), BF16 operands K-major,
//                 FP32 accumulation in TMEM, FP32 and/or BF16 (optionally GELU) outputs;
//                 z = ensemble member
//   elementwise   GELU forward/backward, transposes, column sums, masked MSE, Adam
// The GEMM reuses the warp-specialised layout of the emissivity kernel: warp 0 issues
// TMA loads into a 6-stage ring, warp 1 issues tcgen05.mma (M = 128, N = 128), warps 2..9
// drain the double-buffered TMEM accumulators (two warps per lane quadrant, each half of the
// columns: the epilogue's GELU and stores, not the MMAs, bound the hidden layers).  Every
// mbarrier wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "mlp.h"
#include "tc_ptx.cuh"

namespace heat {

using namespace tc;

namespace {

constexpr int gM = 128, gN = 128, gStages = 6;
constexpr int gAStage = gM * 128, gBStage = gN * 128;
constexpr int gEpiWarps = 8;  // two per TMEM lane quadrant, each half of a tile's columns

__device__ __forceinline__ void gtile(const GemmTcParams& p, int t, int& z, int& mt, int& nt) {
    int per = p.mtiles * p.ntiles;
    z = t / per;
    int r = t - z * per;
    mt = r / p.ntiles;
    nt = r - mt * p.ntiles;
}

}  // namespace

// GELU in its tanh form, x/2 (1 + tanh(y)), y = sqrt(2/pi) (x + 0.044715 x^3), with
// tanh(y) = 1 - 2 / (e^{2y} + 1) on the hardware exponential (|y| clamped at 15, where tanh
// is 1 to FP32 precision): a few instructions per value instead of erf's polynomial, which
// made the hidden layers' epilogue, not the tensor cores, their bound.
__device__ __forceinline__ float gelu_tanh_y(float y) {
    y = fminf(fmaxf(y, -15.0f), 15.0f);
    return 1.0f - __fdividef(2.0f, __expf(2.0f * y) + 1.0f);
}
__device__ __forceinline__ float gelu(float x) {
    const float t = gelu_tanh_y(0.79788456080286536f * fmaf(0.044715f * x * x, x, x));
    return 0.5f * x * (1.0f + t);
}

__global__ void __launch_bounds__(64 + 32 * gEpiWarps, 1) k_gemm_bf16(const __grid_constant__ GemmTcParams p) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + gStages * gAStage;
    uint64_t* bars = (uint64_t*)(sB + gStages * gBStage);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * gStages + 5);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + gStages);
    const uint32_t b_tfull = smem_u32(bars + 2 * gStages), b_tempty = smem_u32(bars + 2 * gStages + 2);
    const uint32_t b_done = smem_u32(bars + 2 * gStages + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < gStages; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(b_tfull + 8 * a, 1);
            mbar_init(b_tempty + 8 * a, gEpiWarps);
        }
        mbar_init(b_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int total = p.nz * p.mtiles * p.ntiles;
    const int ksteps = p.K / 64;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[gStages];
            for (int s = 0; s < gStages; ++s) last_phase[s] = -1;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                int z, mt, nt;
                gtile(p, t, z, mt, nt);
                for (int ks = 0; ks < ksteps; ++ks) {
                    if (!mbar_wait(b_empty + 8 * stage, phase ^ 1, abort_flag, p.wait_polls)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(b_full + 8 * stage, gAStage + gBStage);
                    tma_load_2d(smem_u32(sA + stage * gAStage), &p.ta[z], ks * 64, mt * gM, b_full + 8 * stage);
                    tma_load_2d(smem_u32(sB + stage * gBStage), &p.tb[z], ks * 64, nt * gN, b_full + 8 * stage);
                    last_phase[stage] = (int)phase;
                    if (++stage == gStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (!ok) {
                atomicOr(p.status, kStatTimeout);
                *abort_flag = 1;
            }
            for (int s = 0; s < gStages; ++s)
                if (last_phase[s] >= 0)
                    for (long long i = 0; i < kTcSpinLimit; ++i)
                        if (mbar_try(b_full + 8 * s, (uint32_t)last_phase[s])) break;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = idesc(1, gM, gN);
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                if (!mbar_wait(b_tempty + 8 * acc, acc_phase ^ 1, abort_flag, p.wait_polls)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)acc * gN;
                for (int ks = 0; ks < ksteps; ++ks) {
                    if (!mbar_wait(b_full + 8 * stage, phase, abort_flag, p.wait_polls)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t a0 = sdesc(smem_u32(sA + stage * gAStage));
                    const uint64_t b0 = sdesc(smem_u32(sB + stage * gBStage));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) umma<false>(d, a0 + 2 * kk, b0 + 2 * kk, id, (ks | kk) != 0 ? 1u : 0u);
                    umma_commit(b_empty + 8 * stage);
                    if (++stage == gStages) {
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
            umma_commit(b_done);
            for (long long i = 0; i < kTcSpinLimit; ++i)
                if (mbar_try(b_done, 0)) break;
        }
    } else {
        // epilogue: lane = row of the tile; each chunk of 32 columns gets its bias (broadcast
        // loads), optional GELU for the BF16 output, and 16-byte stores of the row's run
        const int q = warp & 3;                          // the TMEM lane quadrant this warp may read
        const int c0 = ((warp - 2) >> 2) * (gN / 64);    // its half of the tile's 32-column chunks
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            int z, mt, nt;
            gtile(p, t, z, mt, nt);
            bool ok = __all_sync(0xffffffffu, mbar_wait(b_tfull + 8 * acc, acc_phase, abort_flag, p.wait_polls));
            if (!ok) {
                if (lane == 0) {
                    atomicOr(p.status, kStatTimeout);
                    *abort_flag = 1;
                }
                break;
            }
            tc_fence_after();
            const int row = mt * gM + q * 32 + lane;
            const bool rok = row < p.M;
            float* C = p.c[z];
            __nv_bfloat16* Cb = p.cb[z];
            const float* bias = p.bias[z];
            for (int c = c0; c < c0 + gN / 64; ++c) {
                uint32_t v[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * gN + c * 32), v);
                const int col0 = nt * gN + c * 32;
                if (col0 >= p.N) continue;
                float* crow = C ? C + (size_t)(rok ? row : 0) * p.ldc + col0 : nullptr;
                __nv_bfloat16* brow = Cb ? Cb + (size_t)(rok ? row : 0) * p.ldcb + col0 : nullptr;
                const bool fast =
                    col0 + 32 <= p.N &&
                    __all_sync(0xffffffffu, ((uintptr_t)crow & 15u) == 0 && ((uintptr_t)brow & 15u) == 0 &&
                                                (!bias || ((uintptr_t)(bias + col0) & 15u) == 0));
                if (fast) {
                    float val[32];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float4 b4 = bias ? ((const float4*)(bias + col0))[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                        val[4 * k] = __uint_as_float(v[4 * k]) + b4.x;
                        val[4 * k + 1] = __uint_as_float(v[4 * k + 1]) + b4.y;
                        val[4 * k + 2] = __uint_as_float(v[4 * k + 2]) + b4.z;
                        val[4 * k + 3] = __uint_as_float(v[4 * k + 3]) + b4.w;
                    }
                    if (rok && crow) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            float4 o = make_float4(val[4 * k], val[4 * k + 1], val[4 * k + 2], val[4 * k + 3]);
                            if (p.accumulate) {
                                const float4 old = ((const float4*)crow)[k];
                                o.x += old.x;
                                o.y += old.y;
                                o.z += old.z;
                                o.w += old.w;
                            }
                            ((float4*)crow)[k] = o;
                        }
                    }
                    if (rok && brow) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            uint32_t w[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                float x0 = val[8 * k + 2 * h], x1 = val[8 * k + 2 * h + 1];
                                if (p.act) {
                                    x0 = gelu(x0);
                                    x1 = gelu(x1);
                                }
                                const __nv_bfloat162 pr = __floats2bfloat162_rn(x0, x1);
                                w[h] = *(const uint32_t*)&pr;
                            }
                            ((uint4*)brow)[k] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int col = col0 + i;
                        if (rok && col < p.N) {
                            const float val = __uint_as_float(v[i]) + (bias ? bias[col] : 0.0f);
                            if (C) {
                                float* o = C + (size_t)row * p.ldc + col;
                                *o = p.accumulate ? *o + val : val;
                            }
                            if (Cb) Cb[(size_t)row * p.ldcb + col] = __float2bfloat16_rn(p.act ? gelu(val) : val);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem_base) : "memory");
    }
}

size_t gemm_bf16_smem_bytes() {
    return 1024 + (size_t)gStages * (gAStage + gBStage) + (2 * gStages + 5) * 8 + 16;
}

cudaError_t launch_gemm_bf16(const GemmTcParams& p, int sms, cudaStream_t st) {
    int total = p.nz * p.mtiles * p.ntiles;
    if (total <= 0) return cudaSuccess;
    size_t smem = gemm_bf16_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gemm_bf16<<<total < sms ? total : sms, 64 + 32 * gEpiWarps, smem, st>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// elementwise kernels

__device__ __forceinline__ float gelu_grad(float x) {  // d/dx of gelu above
    const float t = gelu_tanh_y(0.79788456080286536f * fmaf(0.044715f * x * x, x, x));
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * 0.79788456080286536f * fmaf(0.134145f, x * x, 1.0f);
}

// X = GELU(Z) as BF16 (Z stays FP32 for the backward pass).
__global__ void k_gelu_fwd(long long n, const float* __restrict__ Z, __nv_bfloat16* __restrict__ X) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) X[i] = __float2bfloat16_rn(gelu(Z[i]));
}

// dZ = dX * GELU'(Z) as BF16.
__global__ void k_gelu_bwd(long long n, const float* __restrict__ dX, const float* __restrict__ Z,
                           __nv_bfloat16* __restrict__ dZ) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dZ[i] = __float2bfloat16_rn(dX[i] * gelu_grad(Z[i]));
}

// out[c][r] = in[r][c] for a rows x cols BF16 matrix (32 x 32 tiles through shared memory).
__global__ void k_transpose_bf16(int rows, int cols, const __nv_bfloat16* __restrict__ in,
                                 __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 t[32][33];
    int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][k];
    }
}

// colsum[c] = sum_r A[r][c] (BF16 in, FP32 out) for the bias gradients.
__global__ void k_colsum_bf16(int rows, int cols, const __nv_bfloat16* __restrict__ A, float* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(A[(size_t)r * cols + c]);
    out[c] = s;
}

// Masked squared error: targets NaN are excluded.  dY = 2 (Y - T) / count (BF16);
// loss partial sums per block into loss[blockIdx.x].
// Weight of the one-sided penalty relative to the fitted entries (it only has to keep the
// masked tail below the mask, not fit it).
constexpr float kTailWeight = 0.3f;

__global__ void k_mse(long long n, int N, const float* __restrict__ Y, const float* __restrict__ T,
                      const float* __restrict__ tb, const float* __restrict__ ym, const float* __restrict__ ys,
                      const unsigned long long* __restrict__ count, __nv_bfloat16* __restrict__ dY,
                      double* __restrict__ loss_acc) {
    __shared__ float red[256];
    const unsigned long long c = *count;
    const float inv = c > 0 ? 1.0f / (float)c : 0.0f;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float e2 = 0.0f;
    if (i < n) {
        float t = T[i], y = Y[i], d = 0.0f;
        if (t == t) {
            d = y - t;
        } else if (tb) {
            // masked entry: penalise only a prediction above the row's mask level
            int k = (int)(i % N);
            float bound = tb[i / N];
            float over = y * ys[k] + ym[k] - bound;
            if (bound == bound && over > 0.0f) d = kTailWeight * over / ys[k];
        }
        dY[i] = __float2bfloat16_rn(2.0f * d * inv);
        e2 = d * d;
    }
    red[threadIdx.x] = e2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_acc && red[0] != 0.0f) atomicAdd(loss_acc, (double)red[0] * (double)inv);
}

// Adam step on FP32 master weights; refreshes the BF16 copy W [rows][cols] and, when
// given, its transpose WT [cols][rows].
__global__ void k_adam(long long n, int rows, int cols, float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, __nv_bfloat16* __restrict__ Wb, __nv_bfloat16* __restrict__ WTb) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    if (Wb) {
        __nv_bfloat16 h = __float2bfloat16_rn(wi);
        Wb[i] = h;
        if (WTb) {
            int r = (int)(i / cols), c = (int)(i % cols);
            WTb[(size_t)c * rows + r] = h;
        }
    }
}

// BF16 copy W [rows][cols] of FP32 weights and, when given, its transpose WT [cols][rows].
__global__ void k_to_bf16(long long n, int rows, int cols, const float* __restrict__ w, __nv_bfloat16* __restrict__ Wb,
                          __nv_bfloat16* __restrict__ WTb) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
    Wb[i] = h;
    if (WTb) {
        int r = (int)(i / cols), c = (int)(i % cols);
        WTb[(size_t)c * rows + r] = h;
    }
}

// Count of non-NaN entries (targets that take part in the loss).
__global__ void k_count_valid(long long n, const float* __restrict__ T, unsigned long long* __restrict__ count) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v = (i < n && T[i] == T[i]) ? 1u : 0u;
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(count, (unsigned long long)v);
}

cudaError_t launch_to_bf16(long long n, int rows, int cols, const float* w, __nv_bfloat16* Wb, __nv_bfloat16* WTb,
                           cudaStream_t st) {
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, rows, cols, w, Wb, WTb);
    return cudaGetLastError();
}
cudaError_t launch_count_valid(long long n, const float* T, unsigned long long* count, cudaStream_t st) {
    k_count_valid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, T, count);
    return cudaGetLastError();
}

cudaError_t launch_gelu_fwd(long long n, const float* Z, __nv_bfloat16* X, cudaStream_t st) {
    k_gelu_fwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, Z, X);
    return cudaGetLastError();
}
cudaError_t launch_gelu_bwd(long long n, const float* dX, const float* Z, __nv_bfloat16* dZ, cudaStream_t st) {
    k_gelu_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, dX, Z, dZ);
    return cudaGetLastError();
}
cudaError_t launch_transpose_bf16(int rows, int cols, const __nv_bfloat16* in, __nv_bfloat16* out, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    k_transpose_bf16<<<grid, block, 0, st>>>(rows, cols, in, out);
    return cudaGetLastError();
}
cudaError_t launch_colsum_bf16(int rows, int cols, const __nv_bfloat16* A, float* out, cudaStream_t st) {
    k_colsum_bf16<<<(cols + 127) / 128, 128, 0, st>>>(rows, cols, A, out);
    return cudaGetLastError();
}
cudaError_t launch_mse(long long n, int N, const float* Y, const float* T, const float* tb, const float* ym,
                       const float* ys, const unsigned long long* count, __nv_bfloat16* dY, double* loss_acc,
                       cudaStream_t st) {
    k_mse<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, N, Y, T, tb, ym, ys, count, dY, loss_acc);
    return cudaGetLastError();
}
cudaError_t launch_adam(long long n, int rows, int cols, float* w, const float* g, float* m, float* v, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, __nv_bfloat16* Wb, __nv_bfloat16* WTb,
                        cudaStream_t st) {
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, rows, cols, w, g, m, v, lr, b1, b2, eps, bc1, bc2, Wb,
                                                        WTb);
    return cudaGetLastError();
}

}  // namespace heat
