// Learned surrogate of the emissivity: an ensemble of MLPs (128 padded inputs -> 4 x 512
// GELU -> N outputs) trained on spectra the exact path computes, with the exact path as
// fallback where the ensemble disagrees.  The method itself (Sec. 2 of the paper) has no
// surrogate; this is the serving-side extension built on top of it.
//
// Inputs per (cell, grain) sample: ln of the power the grain absorbs in 64 wavelength bands,
// ln a, a composition flag, ln of the total absorbed power, zero padding; standardised with
// statistics of the training set.
// Output: y_lambda = ln j_lambda - ln P_abs (P_abs = c int u C dlambda on the grid, exact
// and cheap), standardised per wavelength; targets are masked (NaN) where j < 1e-6 of the
// spectrum's peak.  Training: masked MSE plus a one-sided penalty that keeps masked entries
// predicted below the mask, Adam with cosine decay, FP32 master weights, BF16 operands on
// tcgen05 with FP32 accumulation.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../../include/heat.h"
#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "mlp.h"

namespace heat {

constexpr int kFeat = 128;  // padded input width
constexpr int kBands = 64;
constexpr int kHidden = 512;
constexpr int kLayers = 5;
constexpr float kMaskRel = 1e-6f;  // accuracy mask: j above this fraction of the peak

struct Surrogate {
    int members = 0, N = 0, G = 0;
    int Kin[kLayers], Nout[kLayers];
    long long woff[kLayers], boff[kLayers], nparams = 0;
    long long wflat[kLayers], wtot = 0;  // offsets of the weight tensors in the BF16 copies
    DevBuf params, grads, adam_m, adam_v;  // [members][nparams] FP32
    DevBuf wb, wtb;                        // [members][wtot] BF16 W and W^T
    DevBuf xmean, xstd, ymean, ystd;       // standardisation
    bool norm_ready = false;
    std::vector<float> gfeat;              // [G][2] ln a, composition flag
    DevBuf d_gfeat;
    long long step = 0;
    unsigned long long seed = 0;
    // work buffers for one member and a batch of B rows
    int B = 0;
    DevBuf Xn, Tn, Z[kLayers], Act[kLayers], dYb, dXf, dZb, T1, T2, loss, ens_mean, ens_m2, tb, cnt;
    // inference of all members at once: hidden activations (ping-pong) and outputs per member
    int IB = 0;
    DevBuf H[8][2], Zo[8];
};

void surrogate_free(Surrogate* s) {
    if (!s) return;
    DevBuf* bufs[] = {&s->params, &s->grads, &s->adam_m, &s->adam_v, &s->wb, &s->wtb, &s->xmean, &s->xstd,
                      &s->ymean, &s->ystd, &s->d_gfeat, &s->Xn, &s->Tn, &s->dYb, &s->dXf, &s->dZb, &s->T1,
                      &s->T2, &s->loss, &s->ens_mean, &s->ens_m2, &s->tb, &s->cnt};
    for (DevBuf* b : bufs) b->release();
    for (int l = 0; l < kLayers; ++l) {
        s->Z[l].release();
        s->Act[l].release();
    }
    for (int m = 0; m < 8; ++m) {
        s->H[m][0].release();
        s->H[m][1].release();
        s->Zo[m].release();
    }
    delete s;
}

// ---------------------------------------------------------------------------
// feature, target and statistics kernels

// Inputs of each (cell, grain) sample, one warp per sample: the power the grain absorbs in
// each of 64 wavelength bands, c int u C dlambda on the log-log interpolant (FP32 segment
// integrals, FP64 sums), as ln, floored at 1e-12 of the total; ln a, the composition flag,
// ln of the total; zero padding.  lnp receives ln of the total (the output normalisation).
__global__ void __launch_bounds__(256) k_sample_features(int N, int G, int cells, const float* __restrict__ uasu,
                                                         int Cc, const float* __restrict__ ce,
                                                         const float* __restrict__ sC, const float* __restrict__ dln,
                                                         const float* __restrict__ gfeat, float* __restrict__ X,
                                                         float* __restrict__ lnp) {
    __shared__ double band[8][kBands];
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (w >= (long long)cells * G) return;
    int c = (int)(w / G), g = (int)(w % G);
    const float2* us = (const float2*)uasu;
    double total = 0.0;
    for (int b = 0; b < kBands; ++b) {
        int n0 = (int)((long long)b * (N - 1) / kBands), n1 = (int)((long long)(b + 1) * (N - 1) / kBands);
        double acc = 0.0;
        for (int n = n0 + lane; n < n1; n += 32) {
            float2 v = us[(size_t)n * Cc + c];
            float bb = v.x * ce[(size_t)g * N + n];
            if (bb > 0.0f) {
                float q0 = v.y + sC[(size_t)g * N + n] + 1.0f, dl = dln[n];
                acc += (double)(bb * dl * e1f(q0 * dl));
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        total += acc;
        if (lane == 0) band[wid][b] = acc;
    }
    __syncwarp();
    float* row = X + (size_t)w * kFeat;
    const double floor_v = fmax(total * 1e-12, 1e-300);
    for (int f = lane; f < kFeat; f += 32) {
        float v = 0.0f;
        if (f < kBands) v = (float)log(fmax(band[wid][f], floor_v));
        else if (f == kBands) v = gfeat[2 * g];
        else if (f == kBands + 1) v = gfeat[2 * g + 1];
        else if (f == kBands + 2) v = (float)log(fmax(total, 1e-300));
        row[f] = v;
    }
    if (lane == 0) lnp[w] = (float)log(fmax(total, 1e-300));
}

// Targets y = ln j - ln P_abs where j > 1e-6 of the spectrum's peak, NaN (masked) elsewhere.
// One block per sample.
__global__ void k_targets(int N, const float* __restrict__ j, const float* __restrict__ lnp, float* __restrict__ Y) {
    __shared__ float red[256];
    long long s = blockIdx.x;
    const float* js = j + (size_t)s * N;
    float m = 0.0f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) m = fmaxf(m, js[n]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    float thr = red[0] * kMaskRel;
    float lp = lnp[s];
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float v = js[n];
        Y[(size_t)s * N + n] = (v > thr && v > 0.0f) ? logf(v) - lp : __int_as_float(0x7fc00000);
    }
}

// Column mean and standard deviation of a rows x cols FP32 matrix, NaN entries skipped
// (std 1 for columns without data or without spread).  Block: 32 columns x 8 row lanes.
__global__ void k_colstats(long long rows, int cols, const float* __restrict__ A, float* __restrict__ mean,
                           float* __restrict__ stdv) {
    __shared__ double s1[8][32], s2[8][32], sn[8][32];
    int c = blockIdx.x * 32 + threadIdx.x;
    double a = 0, b = 0, n = 0;
    if (c < cols)
        for (long long r = threadIdx.y; r < rows; r += 8) {
            float v = A[(size_t)r * cols + c];
            if (v == v) {
                a += v;
                b += (double)v * v;
                n += 1;
            }
        }
    s1[threadIdx.y][threadIdx.x] = a;
    s2[threadIdx.y][threadIdx.x] = b;
    sn[threadIdx.y][threadIdx.x] = n;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        for (int k = 1; k < 8; ++k) {
            a += s1[k][threadIdx.x];
            b += s2[k][threadIdx.x];
            n += sn[k][threadIdx.x];
        }
        double mu = n > 0 ? a / n : 0.0;
        double var = n > 1 ? b / n - mu * mu : 0.0;
        double sd = var > 1e-12 ? sqrt(var) : 1.0;
        mean[c] = (float)mu;
        stdv[c] = (float)sd;
    }
}

// Normalised batch: Xn[b] = bf16((X[idx[b]] - mean) / std), Tn[b] = (T[idx[b]] - ymean) / ystd
// (idx null: row b itself); tb[b] (when given) = the row's mask level in raw units, the
// largest finite target + ln 1e-6 (NaN if it has none).  blockDim.x = 128.
__global__ void k_gather_norm(int count, int B, int N, const int* __restrict__ idx, const float* __restrict__ X,
                              const float* __restrict__ T, const float* __restrict__ xm, const float* __restrict__ xs,
                              const float* __restrict__ ym, const float* __restrict__ ys,
                              __nv_bfloat16* __restrict__ Xn, float* __restrict__ Tn, float* __restrict__ tb) {
    __shared__ float red[128];
    int b = blockIdx.x;
    if (b >= B) return;
    long long r = b < count ? (idx ? idx[b] : b) : -1;
    for (int f = threadIdx.x; f < kFeat; f += blockDim.x) {
        float v = r >= 0 ? (X[(size_t)r * kFeat + f] - xm[f]) / xs[f] : 0.0f;
        Xn[(size_t)b * kFeat + f] = __float2bfloat16_rn(v);
    }
    if (!Tn) return;
    float mx = -INFINITY;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float v = r >= 0 ? T[(size_t)r * N + n] : __int_as_float(0x7fc00000);
        if (v == v) mx = fmaxf(mx, v);
        Tn[(size_t)b * N + n] = (v == v) ? (v - ym[n]) / ys[n] : v;
    }
    if (!tb) return;
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) tb[b] = red[0] > -INFINITY ? red[0] + logf(kMaskRel) : __int_as_float(0x7fc00000);
}

// Ensemble accumulation (Welford over members) of de-normalised outputs.
__global__ void k_ens_acc(long long n, int N, int m, const float* __restrict__ Y, const float* __restrict__ ym,
                          const float* __restrict__ ys, float* __restrict__ mean, float* __restrict__ m2) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = (int)(i % N);
    float y = Y[i] * ys[k] + ym[k];
    if (m == 0) {
        mean[i] = y;
        m2[i] = 0.0f;
    } else {
        float d = y - mean[i];
        float mu = mean[i] + d / (float)(m + 1);
        m2[i] += d * (y - mu);
        mean[i] = mu;
    }
}

// Per sample: ln j = mean + ln P_abs; spread = max over the predicted emission (within
// 1e-6 of the predicted peak) of the ensemble standard deviation of ln j.
__global__ void k_ens_final(int rows, int N, int members, const float* __restrict__ mean,
                            const float* __restrict__ m2, const float* __restrict__ lnp, float* __restrict__ lnj,
                            float* __restrict__ spread) {
    __shared__ float red[256];
    int s = blockIdx.x;
    if (s >= rows) return;
    const float* mu = mean + (size_t)s * N;
    float mx = -INFINITY;
    for (int n = threadIdx.x; n < N; n += blockDim.x) mx = fmaxf(mx, mu[n]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    const float thr = red[0] + logf(kMaskRel);
    __syncthreads();
    float sp = 0.0f;
    const float lp = lnp[s];
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float v = mu[n];
        lnj[(size_t)s * N + n] = v + lp;
        if (v > thr) sp = fmaxf(sp, sqrtf(fmaxf(m2[(size_t)s * N + n], 0.0f) / (float)(members > 1 ? members - 1 : 1)));
    }
    red[threadIdx.x] = sp;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) spread[s] = red[0];
}

// Ensemble statistics of one sample per block from the members' standardised outputs
// Zo[m][s][n]: ln j = mean over members + ln P_abs; spread = the largest standard deviation
// (members - 1 in the denominator) of ln j over the predicted emission (mean within 1e-6 of
// its peak).
struct ZoPtrs {
    const float* z[8];
};
// A thread holds the members' values of up to kEnsPer wavelengths in registers (one read of
// the outputs, one write of ln j); the maxima are warp shuffles and one shared-memory pass.
constexpr int kEnsPer = 4;
__device__ __forceinline__ float block_max_f(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = lane < nw ? red[lane] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}
template <int MAXM>
__global__ void __launch_bounds__(1024) k_ens_stats(int rows, int N, int members, ZoPtrs zo,
                                                    const float* __restrict__ ym, const float* __restrict__ ys,
                                                    const float* __restrict__ lnp, float* __restrict__ lnj,
                                                    float* __restrict__ spread) {
    __shared__ float red[32];
    const int s = blockIdx.x;
    if (s >= rows) return;
    const int T = blockDim.x;
    float* out = lnj + (size_t)s * N;
    float v[kEnsPer][MAXM], mu[kEnsPer];
    float mx = -INFINITY;
#pragma unroll
    for (int q = 0; q < kEnsPer; ++q) {
        const int n = threadIdx.x + q * T;
        mu[q] = 0.0f;
        if (n < N) {
            const float a = ys[n], b = ym[n];
            float sum = 0.0f;
#pragma unroll
            for (int m = 0; m < MAXM; ++m)
                if (m < members) {
                    v[q][m] = zo.z[m][(size_t)s * N + n] * a + b;
                    sum += v[q][m];
                }
            mu[q] = sum / (float)members;
            mx = fmaxf(mx, mu[q]);
        }
    }
    const float thr = block_max_f(mx, red) + logf(kMaskRel);
    const float lp = lnp[s];
    float sp = 0.0f;
#pragma unroll
    for (int q = 0; q < kEnsPer; ++q) {
        const int n = threadIdx.x + q * T;
        if (n < N) {
            if (mu[q] > thr && members > 1) {
                float ss = 0.0f;
#pragma unroll
                for (int m = 0; m < MAXM; ++m)
                    if (m < members) {
                        const float d = v[q][m] - mu[q];
                        ss += d * d;
                    }
                sp = fmaxf(sp, sqrtf(ss / (float)(members - 1)));
            }
            out[n] = mu[q] + lp;
        }
    }
    sp = block_max_f(sp, red);
    if (threadIdx.x == 0) spread[s] = sp;
}

// j = exp(ln j) for the surrogate output; flags the cells with any grain above tol.
__global__ void k_sur_output(long long n, int N, int G, const float* __restrict__ lnj, const float* __restrict__ spread,
                             float tol, float* __restrict__ j, int* __restrict__ cell_flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    j[i] = __expf(lnj[i]);
    long long s = i / N;
    if (i % N == 0 && spread[s] > tol) cell_flag[s / G] = 1;
}

// Energy check of surrogate spectra, one warp per (cell, grain) sample: [absorbed power
// P_abs = exp(lnp), emitted power 4 pi int j dlambda by the trapezoid rule on the grid].
__global__ void k_sur_energy(long long samples, int N, const double* __restrict__ lam, const float* __restrict__ j,
                             const float* __restrict__ lnp, double* __restrict__ ledger) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= samples) return;
    const float* js = j + (size_t)w * N;
    double acc = 0.0;
    for (int n = lane; n < N - 1; n += 32) acc += 0.5 * ((double)js[n] + (double)js[n + 1]) * (lam[n + 1] - lam[n]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        ledger[2 * w] = exp((double)lnp[w]);
        ledger[2 * w + 1] = 4.0 * 3.14159265358979323846 * acc;
    }
}

// Ledger rows of the cells solved exactly, back to their places.
__global__ void k_fallback_ledger(int n, int row, const int* __restrict__ list, const double* __restrict__ src,
                                  double* __restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * row) return;
    int r = (int)(i / row), k = (int)(i % row);
    dst[(size_t)list[r] * row + k] = src[i];
}

// Compact flagged cells into a list (order-independent: positions by atomic counter,
// then sorted on the host).
__global__ void k_compact(int cells, const int* __restrict__ flag, int* __restrict__ list, int* __restrict__ count) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cells && flag[c]) list[atomicAdd(count, 1)] = c;
}

// Gather the fields of the listed cells into a contiguous buffer.
__global__ void k_fallback_gather(int n, int N, const int* __restrict__ list, const double* __restrict__ u,
                                  long long cell0, double* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * N) return;
    int r = (int)(i / N), k = (int)(i % N);
    out[i] = u[(size_t)(cell0 + list[r]) * N + k];
}

// Scatter exact emissivities of the listed cells over the surrogate output.
__global__ void k_fallback_scatter(int n, long long row, const int* __restrict__ list, const float* __restrict__ src,
                                   float* __restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * row) return;
    int r = (int)(i / row);
    long long k = i % row;
    dst[(size_t)list[r] * row + k] = src[i];
}

}  // namespace heat

using namespace heat;

namespace {

// K-major BF16 operand map: rows x k elements (k a multiple of 64), box (64, 128).
bool encode_bf16(CUtensorMap* m, const void* base, long long rows, long long k) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return false;
        enc = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(k * 2)};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

#define SCK(call)                                         \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
    } while (0)

// C[M x N] = A[M x K] . B[N x K]^T (+ bias): both operands BF16 row-major (K contiguous).
heat_status gemm(heat_ctx* ctx, int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C,
                 __nv_bfloat16* Cb, const float* bias, int accumulate, cudaStream_t st, int act = 0) {
    GemmTcParams p;
    std::memset(&p, 0, sizeof(p));
    if (!encode_bf16(&p.ta[0], A, M, K) || !encode_bf16(&p.tb[0], B, N, K))
        return ctx->fail(HEAT_ECUDA, "surrogate: cuTensorMapEncodeTiled failed");
    p.c[0] = C;
    p.cb[0] = Cb;
    p.bias[0] = bias;
    p.ldc = N;
    p.ldcb = N;
    p.M = M;
    p.N = N;
    p.K = K;
    p.nz = 1;
    p.mtiles = (M + 127) / 128;
    p.ntiles = (N + 127) / 128;
    p.accumulate = accumulate;
    p.act = act;
    p.status = ctx->d_status.as<int>();
    p.wait_polls = ctx->wait_polls;
    SCK(launch_gemm_bf16(p, ctx->sms, st));
    return HEAT_OK;
}

// One layer of every member in one launch (problem z = member): C[z] = A[z] W[z]^T + b[z].
heat_status gemm_members(heat_ctx* ctx, Surrogate* s, int l, int M, const __nv_bfloat16* const* A, float* const* C,
                         __nv_bfloat16* const* Cb, int act, cudaStream_t st);

heat_status ensure_batch(heat_ctx* ctx, Surrogate* s, int B) {
    if (s->B >= B) return HEAT_OK;
    const size_t bf = 2, f4 = 4;
    const int wmax = std::max(s->N, kHidden);
    bool ok = !s->Xn.ensure(bf * (size_t)B * kFeat) && !s->Tn.ensure(f4 * (size_t)B * s->N) &&
              !s->dYb.ensure(bf * (size_t)B * wmax) && !s->dXf.ensure(f4 * (size_t)B * kHidden) &&
              !s->dZb.ensure(bf * (size_t)B * kHidden) && !s->T1.ensure(bf * (size_t)B * wmax) &&
              !s->T2.ensure(bf * (size_t)B * std::max(kFeat, kHidden)) && !s->loss.ensure(16) &&
              !s->ens_mean.ensure(f4 * (size_t)B * s->N) && !s->ens_m2.ensure(f4 * (size_t)B * s->N) &&
              !s->tb.ensure(sizeof(float) * (size_t)B) && !s->cnt.ensure(16);
    for (int l = 0; l < kLayers; ++l) {
        ok = ok && !s->Z[l].ensure(f4 * (size_t)B * s->Nout[l]);
        ok = ok && !s->Act[l].ensure(bf * (size_t)B * s->Kin[l]);
    }
    if (!ok) return ctx->fail(HEAT_ENOMEM, "surrogate: batch buffers");
    s->B = B;
    return HEAT_OK;
}

__nv_bfloat16* Wb(Surrogate* s, int m, int l) { return s->wb.as<__nv_bfloat16>() + (size_t)m * s->wtot + s->wflat[l]; }
__nv_bfloat16* WTb(Surrogate* s, int m, int l) { return s->wtb.as<__nv_bfloat16>() + (size_t)m * s->wtot + s->wflat[l]; }
float* Pm(Surrogate* s, int m) { return s->params.as<float>() + (size_t)m * s->nparams; }
float* Gm(Surrogate* s, int m) { return s->grads.as<float>() + (size_t)m * s->nparams; }

heat_status gemm_members(heat_ctx* ctx, Surrogate* s, int l, int M, const __nv_bfloat16* const* A, float* const* C,
                         __nv_bfloat16* const* Cb, int act, cudaStream_t st) {
    const int N = s->Nout[l], K = s->Kin[l];
    GemmTcParams p;
    std::memset(&p, 0, sizeof(p));
    for (int m = 0; m < s->members; ++m) {
        if (!encode_bf16(&p.ta[m], A[m], M, K) || !encode_bf16(&p.tb[m], Wb(s, m, l), N, K))
            return ctx->fail(HEAT_ECUDA, "surrogate: cuTensorMapEncodeTiled failed");
        p.c[m] = C[m];
        p.cb[m] = Cb[m];
        p.bias[m] = Pm(s, m) + s->boff[l];
    }
    p.ldc = N;
    p.ldcb = N;
    p.M = M;
    p.N = N;
    p.K = K;
    p.nz = s->members;
    p.mtiles = (M + 127) / 128;
    p.ntiles = (N + 127) / 128;
    p.act = act;
    p.status = ctx->d_status.as<int>();
    p.wait_polls = ctx->wait_polls;
    SCK(launch_gemm_bf16(p, ctx->sms, st));
    return HEAT_OK;
}

// Forward of member m on the normalised batch in s->Act[0] (rows B): Z[l] FP32, Act[l+1] BF16;
// the output Z[kLayers-1] is the standardised prediction.
heat_status forward(heat_ctx* ctx, Surrogate* s, int m, int B, cudaStream_t st) {
    // hidden layers keep Z (FP32, for the backward pass) and write GELU(Z) as the next BF16
    // input from the GEMM epilogue
    for (int l = 0; l < kLayers; ++l) {
        const bool hidden = l + 1 < kLayers;
        heat_status h = gemm(ctx, B, s->Nout[l], s->Kin[l], s->Act[l].as<__nv_bfloat16>(), Wb(s, m, l),
                             s->Z[l].as<float>(), hidden ? s->Act[l + 1].as<__nv_bfloat16>() : nullptr,
                             Pm(s, m) + s->boff[l], 0, st, hidden ? 1 : 0);
        if (h != HEAT_OK) return h;
    }
    return HEAT_OK;
}

// Backward of member m (after forward and the loss gradient in s->dYb): gradients of every
// weight and bias into Gm(m).
heat_status backward(heat_ctx* ctx, Surrogate* s, int m, int B, cudaStream_t st) {
    __nv_bfloat16* Gb = s->dYb.as<__nv_bfloat16>();  // gradient w.r.t. the layer output, [B][Nout]
    for (int l = kLayers - 1; l >= 0; --l) {
        const int K = s->Kin[l], Nn = s->Nout[l];
        // dW = G^T Act[l]: operands transposed so both are K-major over the batch
        SCK(launch_transpose_bf16(B, Nn, Gb, s->T1.as<__nv_bfloat16>(), st));
        SCK(launch_transpose_bf16(B, K, s->Act[l].as<__nv_bfloat16>(), s->T2.as<__nv_bfloat16>(), st));
        heat_status h = gemm(ctx, Nn, K, B, s->T1.as<__nv_bfloat16>(), s->T2.as<__nv_bfloat16>(),
                             Gm(s, m) + s->woff[l], nullptr, nullptr, 0, st);
        if (h != HEAT_OK) return h;
        SCK(launch_colsum_bf16(B, Nn, Gb, Gm(s, m) + s->boff[l], st));
        if (l == 0) break;
        // dAct = G W  (B-operand W^T, K-major over Nout); then through the GELU of layer l-1
        h = gemm(ctx, B, K, Nn, Gb, WTb(s, m, l), s->dXf.as<float>(), nullptr, nullptr, 0, st);
        if (h != HEAT_OK) return h;
        SCK(launch_gelu_bwd((long long)B * K, s->dXf.as<float>(), s->Z[l - 1].as<float>(), s->dZb.as<__nv_bfloat16>(),
                            st));
        Gb = s->dZb.as<__nv_bfloat16>();
    }
    return HEAT_OK;
}

// Masked MSE of member m's prediction against s->Tn; dY into s->dYb; returns the loss
// (mean over valid targets) through *loss when non-null (synchronises).
// Loss gradient of the batch in Tn against the last layer's output: squared error on the
// finite targets and, with `bounded`, a one-sided square penalty on masked entries predicted
// above their row's mask level (tb), so that predictions stay below the mask where the
// spectrum is; both divided by the number of finite targets (counted on the device).
// loss_acc (or null) accumulates the batch loss.
heat_status loss_grad(heat_ctx* ctx, Surrogate* s, int B, bool count, bool bounded, double* loss_acc,
                      cudaStream_t st) {
    long long n = (long long)B * s->N;
    if (count) {
        SCK(cudaMemsetAsync(s->cnt.p, 0, 8, st));
        SCK(launch_count_valid(n, s->Tn.as<float>(), s->cnt.as<unsigned long long>(), st));
    }
    SCK(launch_mse(n, s->N, s->Z[kLayers - 1].as<float>(), s->Tn.as<float>(), bounded ? s->tb.as<float>() : nullptr,
                   s->ymean.as<float>(), s->ystd.as<float>(), s->cnt.as<unsigned long long>(),
                   s->dYb.as<__nv_bfloat16>(), loss_acc, st));
    return HEAT_OK;
}

heat_status refresh_bf16(heat_ctx* ctx, Surrogate* s, int m, cudaStream_t st);

}  // namespace

extern "C" {

heat_status heat_surrogate_init(heat_ctx* ctx, int members, const float* grain_flag, unsigned long long seed) {
    if (!ctx) return HEAT_EINVAL;
    if (ctx->G == 0) return ctx->fail(HEAT_ESTATE, "heat_surrogate_init: grains not set");
    if (members < 1 || members > 8) return ctx->fail(HEAT_EINVAL, "heat_surrogate_init: 1..8 members");
    if (ctx->N % 64) return ctx->fail(HEAT_EINVAL, "heat_surrogate_init: n_lambda must be a multiple of 64");
    if (ctx->N > kEnsPer * 1024) return ctx->fail(HEAT_EINVAL, "heat_surrogate_init: at most 4096 wavelengths");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return HEAT_ECUDA;
    surrogate_free(ctx->sur);
    Surrogate* s = new (std::nothrow) Surrogate();
    if (!s) return HEAT_ENOMEM;
    ctx->sur = s;
    s->members = members;
    s->N = ctx->N;
    s->G = ctx->G;
    s->seed = seed;
    const int dims[kLayers + 1] = {kFeat, kHidden, kHidden, kHidden, kHidden, ctx->N};
    long long off = 0, woff = 0;
    for (int l = 0; l < kLayers; ++l) {
        s->Kin[l] = dims[l];
        s->Nout[l] = dims[l + 1];
        s->woff[l] = off;
        off += (long long)s->Nout[l] * s->Kin[l];
        s->boff[l] = off;
        off += s->Nout[l];
        s->wflat[l] = woff;
        woff += (long long)s->Nout[l] * s->Kin[l];
    }
    s->nparams = off;
    s->wtot = woff;
    size_t pb = sizeof(float) * (size_t)members * s->nparams;
    if (s->params.ensure(pb) || s->grads.ensure(pb) || s->adam_m.ensure(pb) || s->adam_v.ensure(pb) ||
        s->wb.ensure(2 * (size_t)members * s->wtot) || s->wtb.ensure(2 * (size_t)members * s->wtot) ||
        s->xmean.ensure(4 * kFeat) || s->xstd.ensure(4 * kFeat) || s->ymean.ensure(4 * (size_t)s->N) ||
        s->ystd.ensure(4 * (size_t)s->N) || s->d_gfeat.ensure(8 * (size_t)s->G))
        return ctx->fail(HEAT_ENOMEM, "heat_surrogate_init: allocation");
    // He-style initialisation, seeded per member; biases zero
    std::vector<float> h((size_t)s->nparams);
    for (int m = 0; m < members; ++m) {
        std::mt19937_64 rng(seed * 1000003ULL + (unsigned long long)m * 7919ULL + 17ULL);
        std::normal_distribution<float> nd(0.0f, 1.0f);
        std::fill(h.begin(), h.end(), 0.0f);
        for (int l = 0; l < kLayers; ++l) {
            float sc = std::sqrt((l + 1 < kLayers ? 2.0f : 1.0f) / (float)s->Kin[l]);
            for (long long i = 0; i < (long long)s->Nout[l] * s->Kin[l]; ++i) h[s->woff[l] + i] = nd(rng) * sc;
        }
        if (cudaMemcpy(Pm(s, m), h.data(), sizeof(float) * s->nparams, cudaMemcpyHostToDevice) != cudaSuccess)
            return HEAT_ECUDA;
    }
    if (cudaMemset(s->adam_m.p, 0, pb) != cudaSuccess || cudaMemset(s->adam_v.p, 0, pb) != cudaSuccess) return HEAT_ECUDA;
    s->gfeat.assign(2 * (size_t)s->G, 0.0f);
    for (int g = 0; g < s->G; ++g) {
        s->gfeat[2 * g] = (float)std::log(ctx->radius[g]);
        s->gfeat[2 * g + 1] = grain_flag ? grain_flag[g] : 0.0f;
    }
    if (cudaMemcpy(s->d_gfeat.p, s->gfeat.data(), 8 * (size_t)s->G, cudaMemcpyHostToDevice) != cudaSuccess)
        return HEAT_ECUDA;
    for (int m = 0; m < members; ++m) {
        heat_status hs = refresh_bf16(ctx, s, m, 0);
        if (hs != HEAT_OK) return hs;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return HEAT_ECUDA;
    return HEAT_OK;
}

heat_status heat_surrogate_samples(heat_ctx* ctx, int cell_begin, int cell_count, const float* j, float* X, float* Y,
                                   float* lnp_out, void* stream) {
    if (!ctx || !X) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s) return ctx->fail(HEAT_ESTATE, "surrogate not initialised");
    if (!ctx->u_dev || ctx->u_dtype != HEAT_F64) return ctx->fail(HEAT_ESTATE, "surrogate: FP64 fields must be set");
    if (cell_begin < 0 || cell_count <= 0 || cell_begin + cell_count > ctx->n_cells)
        return ctx->fail(HEAT_EINVAL, "heat_surrogate_samples: cell range");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = ctx->N, G = ctx->G;
    // field tables of the range (FP32 u and slopes), reusing the solve's field kernel
    int Cc = (cell_count + 31) / 32 * 32;
    DevBuf tab, lnp;
    if (tab.ensure(8 * (size_t)N * Cc) ||
        lnp.ensure(4 * (size_t)cell_count * G))
        return ctx->fail(HEAT_ENOMEM, "heat_surrogate_samples: allocation");
    GrainDev gd{};
    gd.N = N;
    gd.dln = ctx->d_dln.as<double>();
    ChunkDev ch{};
    ch.cells = cell_count;
    ch.Cc = Cc;
    ch.ua32 = tab.as<float>();
    ch.status = ctx->d_status.as<int>();
    SCK(launch_field(gd, ctx->u_dev, HEAT_F64, cell_begin, ch, HEAT_BUILD_F32, st));
    long long warps = (long long)cell_count * G;
    k_sample_features<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
        N, G, cell_count, tab.as<float>(), Cc, ctx->d_ce32.as<float>(), ctx->d_sC32.as<float>(),
        ctx->d_dln32.as<float>(), s->d_gfeat.as<float>(), X, lnp.as<float>());
    if (j && Y) k_targets<<<(unsigned)warps, 256, 0, st>>>(N, j, lnp.as<float>(), Y);
    if (lnp_out) SCK(cudaMemcpyAsync(lnp_out, lnp.p, 4 * (size_t)warps, cudaMemcpyDeviceToDevice, st));
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(st));  // the temporaries are released on return
    return HEAT_OK;
}

heat_status heat_surrogate_fit_norm(heat_ctx* ctx, const float* X, const float* Y, long long n, void* stream) {
    if (!ctx || !X || !Y || n <= 0) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s) return ctx->fail(HEAT_ESTATE, "surrogate not initialised");
    cudaStream_t st = (cudaStream_t)stream;
    k_colstats<<<(kFeat + 31) / 32, dim3(32, 8), 0, st>>>(n, kFeat, X, s->xmean.as<float>(), s->xstd.as<float>());
    k_colstats<<<(s->N + 31) / 32, dim3(32, 8), 0, st>>>(n, s->N, Y, s->ymean.as<float>(), s->ystd.as<float>());
    SCK(cudaGetLastError());
    s->norm_ready = true;
    return HEAT_OK;
}

heat_status heat_surrogate_train(heat_ctx* ctx, const float* X, const float* Y, long long n, int batch, int epochs,
                                 float lr, unsigned long long seed, double* loss_history, void* stream) {
    if (!ctx || !X || !Y || n <= 0 || batch <= 0 || batch % 64 || epochs <= 0) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s) return ctx->fail(HEAT_ESTATE, "surrogate not initialised");
    if (!s->norm_ready) return ctx->fail(HEAT_ESTATE, "surrogate: heat_surrogate_fit_norm first");
    cudaStream_t st = (cudaStream_t)stream;
    heat_status h = ensure_batch(ctx, s, batch);
    if (h != HEAT_OK) return h;
    std::mt19937_64 rng(seed);
    std::vector<int> perm((size_t)n);
    DevBuf dperm;
    if (dperm.ensure(sizeof(int) * (size_t)n)) return ctx->fail(HEAT_ENOMEM, "heat_surrogate_train: allocation");
    const long long steps = (long long)epochs * ((n + batch - 1) / batch);
    long long t = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (long long i = 0; i < n; ++i) perm[i] = (int)i;
        std::shuffle(perm.begin(), perm.end(), rng);
        SCK(cudaMemcpyAsync(dperm.p, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
        SCK(cudaMemsetAsync(s->loss.p, 0, sizeof(double), st));
        long long ep_batches = 0;
        for (long long b0 = 0; b0 < n; b0 += batch, ++t) {
            int cnt = (int)std::min<long long>(batch, n - b0);
            k_gather_norm<<<batch, 128, 0, st>>>(cnt, batch, s->N, dperm.as<int>() + b0, X, Y, s->xmean.as<float>(),
                                                 s->xstd.as<float>(), s->ymean.as<float>(), s->ystd.as<float>(),
                                                 s->Act[0].as<__nv_bfloat16>(), s->Tn.as<float>(), s->tb.as<float>());
            SCK(cudaGetLastError());
            ++s->step;
            const float b1 = 0.9f, b2 = 0.999f;
            const float bc1 = 1.0f - std::pow(b1, (float)s->step), bc2 = 1.0f - std::pow(b2, (float)s->step);
            // cosine decay from lr to lr/100 over the steps of this call
            const float lr_t =
                lr * (0.01f + 0.99f * 0.5f * (1.0f + std::cos(3.14159265358979f * (float)t / (float)steps)));
            for (int m = 0; m < s->members; ++m) {
                if ((h = forward(ctx, s, m, batch, st)) != HEAT_OK) return h;
                if ((h = loss_grad(ctx, s, batch, m == 0, true, m == 0 ? s->loss.as<double>() : nullptr, st)) != HEAT_OK)
                    return h;
                if ((h = backward(ctx, s, m, batch, st)) != HEAT_OK) return h;
                SCK(launch_adam(s->nparams, 1, (int)s->nparams, Pm(s, m), Gm(s, m),
                                s->adam_m.as<float>() + (size_t)m * s->nparams,
                                s->adam_v.as<float>() + (size_t)m * s->nparams, lr_t, b1, b2, 1e-8f, bc1, bc2, nullptr,
                                nullptr, st));
                if ((h = refresh_bf16(ctx, s, m, st)) != HEAT_OK) return h;
            }
            ++ep_batches;
        }
        double acc = 0.0;
        SCK(cudaMemcpyAsync(&acc, s->loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));  // also keeps perm's upload ahead of the next shuffle
        if (loss_history) loss_history[ep] = acc / (double)std::max(1LL, ep_batches);
    }
    SCK(cudaStreamSynchronize(st));
    return HEAT_OK;
}

heat_status heat_surrogate_predict(heat_ctx* ctx, const float* X, const float* lnp, long long n, float* lnj,
                                   float* spread, void* stream) {
    if (!ctx || !X || !lnp || !lnj || !spread || n <= 0) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s || !s->norm_ready) return ctx->fail(HEAT_ESTATE, "surrogate not trained");
    cudaStream_t st = (cudaStream_t)stream;
    // samples per pass: every pass launches 7 kernels and encodes 8 tensor maps per layer on
    // the host, so passes are made large (the activations of 4 members: ~1.5 GB at 65536)
    const int B = (int)std::min<long long>(65536, std::max<long long>(16384, n));
    heat_status h = ensure_batch(ctx, s, B);
    if (h != HEAT_OK) return h;
    // all members at once: per-member hidden activations (ping-pong) and standardised outputs
    if (s->IB < B) {
        bool ok = true;
        for (int m = 0; m < s->members; ++m) {
            ok = ok && !s->H[m][0].ensure(2 * (size_t)B * kHidden) && !s->H[m][1].ensure(2 * (size_t)B * kHidden);
            ok = ok && !s->Zo[m].ensure(4 * (size_t)B * s->N);
        }
        if (!ok) return ctx->fail(HEAT_ENOMEM, "surrogate: inference buffers");
        s->IB = B;
    }
    for (long long b0 = 0; b0 < n; b0 += B) {
        int cnt = (int)std::min<long long>(B, n - b0);
        k_gather_norm<<<cnt, 128, 0, st>>>(cnt, cnt, s->N, nullptr, X + (size_t)b0 * kFeat, nullptr,
                                           s->xmean.as<float>(), s->xstd.as<float>(), s->ymean.as<float>(),
                                           s->ystd.as<float>(), s->Act[0].as<__nv_bfloat16>(), nullptr, nullptr);
        int rows = (cnt + 63) / 64 * 64;  // GEMM rows in whole tiles of 64 (extra rows are ignored)
        const __nv_bfloat16* A[8];
        __nv_bfloat16* Hb[8];
        float* Zo[8];
        for (int l = 0; l < kLayers; ++l) {
            const bool hidden = l + 1 < kLayers;
            for (int m = 0; m < s->members; ++m) {
                A[m] = l == 0 ? s->Act[0].as<__nv_bfloat16>() : s->H[m][(l - 1) & 1].as<__nv_bfloat16>();
                Hb[m] = hidden ? s->H[m][l & 1].as<__nv_bfloat16>() : nullptr;
                Zo[m] = hidden ? nullptr : s->Zo[m].as<float>();
            }
            if ((h = gemm_members(ctx, s, l, rows, A, Zo, Hb, hidden ? 1 : 0, st)) != HEAT_OK) return h;
        }
        ZoPtrs zp{};
        for (int m = 0; m < s->members; ++m) zp.z[m] = s->Zo[m].as<float>();
        const int ens_threads = std::min(1024, ((s->N + kEnsPer - 1) / kEnsPer + 31) / 32 * 32);
        auto ens = s->members <= 4 ? k_ens_stats<4> : k_ens_stats<8>;
        ens<<<cnt, ens_threads, 0, st>>>(cnt, s->N, s->members, zp, s->ymean.as<float>(), s->ystd.as<float>(),
                                         lnp + b0, lnj + (size_t)b0 * s->N, spread + b0);
        SCK(cudaGetLastError());
    }
    return HEAT_OK;
}

heat_status heat_surrogate_grads(heat_ctx* ctx, int member, const float* Xn, const float* Tn, int n, float* grad_out,
                                 double* loss_out, void* stream) {
    if (!ctx || !Xn || !Tn || !grad_out || n <= 0 || n % 64) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s || member < 0 || member >= s->members) return ctx->fail(HEAT_ESTATE, "surrogate member");
    cudaStream_t st = (cudaStream_t)stream;
    heat_status h = ensure_batch(ctx, s, n);
    if (h != HEAT_OK) return h;
    // inputs given already standardised: round to BF16 into the activation buffer
    std::vector<float> xh((size_t)n * kFeat);
    std::vector<__nv_bfloat16> xb(xh.size());
    SCK(cudaMemcpy(xh.data(), Xn, 4 * xh.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < xh.size(); ++i) xb[i] = __float2bfloat16_rn(xh[i]);
    SCK(cudaMemcpy(s->Act[0].p, xb.data(), 2 * xb.size(), cudaMemcpyHostToDevice));
    SCK(cudaMemcpy(s->Tn.p, Tn, 4 * (size_t)n * s->N, cudaMemcpyDeviceToDevice));
    if ((h = forward(ctx, s, member, n, st)) != HEAT_OK) return h;
    SCK(cudaMemsetAsync(s->loss.p, 0, sizeof(double), st));
    if ((h = loss_grad(ctx, s, n, true, false, s->loss.as<double>(), st)) != HEAT_OK) return h;
    if ((h = backward(ctx, s, member, n, st)) != HEAT_OK) return h;
    SCK(cudaMemcpyAsync(grad_out, Gm(s, member), 4 * (size_t)s->nparams, cudaMemcpyDeviceToDevice, st));
    double l = 0.0;
    SCK(cudaMemcpyAsync(&l, s->loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (loss_out) *loss_out = l;
    return HEAT_OK;
}

heat_status heat_surrogate_params(heat_ctx* ctx, int member, float* host, int set, long long* nparams) {
    if (!ctx) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s || member < 0 || member >= s->members) return ctx->fail(HEAT_ESTATE, "surrogate member");
    if (nparams) *nparams = s->nparams;
    if (!host) return HEAT_OK;
    if (set) {
        SCK(cudaMemcpy(Pm(s, member), host, 4 * (size_t)s->nparams, cudaMemcpyHostToDevice));
        return refresh_bf16(ctx, s, member, 0);
    }
    SCK(cudaMemcpy(host, Pm(s, member), 4 * (size_t)s->nparams, cudaMemcpyDeviceToHost));
    return HEAT_OK;
}

heat_status heat_surrogate_save(heat_ctx* ctx, const char* path) {
    if (!ctx || !path) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s) return ctx->fail(HEAT_ESTATE, "surrogate not initialised");
    SCK(cudaDeviceSynchronize());
    FILE* f = std::fopen(path, "wb");
    if (!f) return ctx->fail(HEAT_EINVAL, "heat_surrogate_save: cannot open file");
    long long hdr[6] = {0x68656174737572LL, s->members, s->N, s->G, s->nparams, s->step};
    std::fwrite(hdr, sizeof(hdr), 1, f);
    std::fwrite(&s->seed, sizeof(s->seed), 1, f);
    int nr = s->norm_ready ? 1 : 0;
    std::fwrite(&nr, sizeof(nr), 1, f);
    auto dump = [&](DevBuf& b, size_t bytes) {
        std::vector<char> h(bytes);
        cudaMemcpy(h.data(), b.p, bytes, cudaMemcpyDeviceToHost);
        std::fwrite(h.data(), 1, bytes, f);
    };
    size_t pb = 4 * (size_t)s->members * s->nparams;
    dump(s->params, pb);
    dump(s->adam_m, pb);
    dump(s->adam_v, pb);
    dump(s->xmean, 4 * kFeat);
    dump(s->xstd, 4 * kFeat);
    dump(s->ymean, 4 * (size_t)s->N);
    dump(s->ystd, 4 * (size_t)s->N);
    std::fwrite(s->gfeat.data(), 4, s->gfeat.size(), f);
    bool ok = std::ferror(f) == 0;
    std::fclose(f);
    return ok ? HEAT_OK : ctx->fail(HEAT_EINVAL, "heat_surrogate_save: write failed");
}

heat_status heat_surrogate_load(heat_ctx* ctx, const char* path) {
    if (!ctx || !path) return HEAT_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return ctx->fail(HEAT_EINVAL, "heat_surrogate_load: cannot open file");
    long long hdr[6];
    unsigned long long seed = 0;
    int nr = 0;
    bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&seed, sizeof(seed), 1, f) == 1 &&
              std::fread(&nr, sizeof(nr), 1, f) == 1 && hdr[0] == 0x68656174737572LL && hdr[2] == ctx->N &&
              hdr[3] == ctx->G;
    if (!ok) {
        std::fclose(f);
        return ctx->fail(HEAT_EINVAL, "heat_surrogate_load: not a checkpoint of this grid and grain set");
    }
    heat_status h = heat_surrogate_init(ctx, (int)hdr[1], nullptr, seed);
    if (h != HEAT_OK) {
        std::fclose(f);
        return h;
    }
    Surrogate* s = ctx->sur;
    s->step = hdr[5];
    s->norm_ready = nr != 0;
    auto load = [&](DevBuf& b, size_t bytes) {
        std::vector<char> hb(bytes);
        bool r = std::fread(hb.data(), 1, bytes, f) == bytes;
        cudaMemcpy(b.p, hb.data(), bytes, cudaMemcpyHostToDevice);
        return r;
    };
    size_t pb = 4 * (size_t)s->members * s->nparams;
    ok = load(s->params, pb) && load(s->adam_m, pb) && load(s->adam_v, pb) && load(s->xmean, 4 * kFeat) &&
         load(s->xstd, 4 * kFeat) && load(s->ymean, 4 * (size_t)s->N) && load(s->ystd, 4 * (size_t)s->N);
    ok = ok && std::fread(s->gfeat.data(), 4, s->gfeat.size(), f) == s->gfeat.size();
    std::fclose(f);
    if (!ok) return ctx->fail(HEAT_EINVAL, "heat_surrogate_load: truncated checkpoint");
    SCK(cudaMemcpy(s->d_gfeat.p, s->gfeat.data(), 8 * (size_t)s->G, cudaMemcpyHostToDevice));
    for (int m = 0; m < s->members; ++m)
        if ((h = refresh_bf16(ctx, s, m, 0)) != HEAT_OK) return h;
    SCK(cudaDeviceSynchronize());
    return HEAT_OK;
}

heat_status heat_solve_surrogate(heat_ctx* ctx, const heat_opts* fallback_opts, float tol, float* j_out,
                                 int* n_fallback, void* stream) {
    if (!ctx || !fallback_opts || !j_out || !(tol > 0.0f)) return HEAT_EINVAL;
    Surrogate* s = ctx->sur;
    if (!s || !s->norm_ready) return ctx->fail(HEAT_ESTATE, "surrogate not trained");
    if (fallback_opts->size_integrate || fallback_opts->host_io || fallback_opts->j_dtype != HEAT_F32 ||
        fallback_opts->emis == HEAT_EMIS_NONE)
        return ctx->fail(HEAT_EINVAL, "heat_solve_surrogate: fallback needs per-grain FP32 device j");
    if (fallback_opts->heating != HEAT_HEATING_INTEGRAL)  // the network learns the integral form
        return ctx->fail(HEAT_EINVAL, "heat_solve_surrogate: the surrogate is trained on the integral heating form");
    cudaStream_t st = (cudaStream_t)stream;
    const heat_opts& o = *fallback_opts;
    const int N = ctx->N, G = ctx->G;
    int c_begin = o.cell_begin, count = o.cell_count > 0 ? o.cell_count : ctx->n_cells - o.cell_begin;
    if (c_begin < 0 || count <= 0 || c_begin + count > ctx->n_cells)
        return ctx->fail(HEAT_EINVAL, "heat_solve_surrogate: cell range");
    const long long samples = (long long)count * G;
    DevBuf X, lnp, lnj, spread, flag, list, cnt, ufb, jfb;
    if (X.ensure(4 * (size_t)samples * kFeat) || lnp.ensure(4 * (size_t)samples) ||
        lnj.ensure(4 * (size_t)samples * N) || spread.ensure(4 * (size_t)samples) || flag.ensure(4 * (size_t)count) ||
        list.ensure(4 * (size_t)count) || cnt.ensure(4))
        return ctx->fail(HEAT_ENOMEM, "heat_solve_surrogate: allocation");
    heat_status h = heat_surrogate_samples(ctx, c_begin, count, nullptr, X.as<float>(), nullptr, lnp.as<float>(), st);
    if (h != HEAT_OK) return h;
    if ((h = heat_surrogate_predict(ctx, X.as<float>(), lnp.as<float>(), samples, lnj.as<float>(), spread.as<float>(),
                                    st)) != HEAT_OK)
        return h;
    SCK(cudaMemsetAsync(flag.p, 0, 4 * (size_t)count, st));
    SCK(cudaMemsetAsync(cnt.p, 0, 4, st));
    long long ne = samples * N;
    k_sur_output<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(ne, N, G, lnj.as<float>(), spread.as<float>(), tol, j_out,
                                                              flag.as<int>());
    k_compact<<<(count + 255) / 256, 256, 0, st>>>(count, flag.as<int>(), list.as<int>(), cnt.as<int>());
    if (o.ledger_out)
        k_sur_energy<<<(unsigned)((samples * 32 + 255) / 256), 256, 0, st>>>(
            samples, N, ctx->d_lam.as<double>(), j_out, lnp.as<float>(), o.ledger_out);
    SCK(cudaGetLastError());
    int nfb = 0;
    SCK(cudaMemcpyAsync(&nfb, cnt.p, 4, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (n_fallback) *n_fallback = nfb;
    if (nfb == 0) return HEAT_OK;
    // exact path on the flagged cells: gather their fields (sorted), solve, scatter
    std::vector<int> hl(nfb);
    SCK(cudaMemcpy(hl.data(), list.p, 4 * (size_t)nfb, cudaMemcpyDeviceToHost));
    std::sort(hl.begin(), hl.end());
    SCK(cudaMemcpy(list.p, hl.data(), 4 * (size_t)nfb, cudaMemcpyHostToDevice));
    DevBuf lfb;
    if (ufb.ensure(8 * (size_t)nfb * N) || jfb.ensure(4 * (size_t)nfb * G * N) ||
        (o.ledger_out && lfb.ensure(sizeof(double) * 2 * (size_t)nfb * G)))
        return ctx->fail(HEAT_ENOMEM, "heat_solve_surrogate: allocation");
    long long nu = (long long)nfb * N;
    k_fallback_gather<<<(unsigned)((nu + 255) / 256), 256, 0, st>>>(nfb, N, list.as<int>(), (const double*)ctx->u_dev,
                                                                    c_begin, ufb.as<double>());
    SCK(cudaGetLastError());
    const void* u_save = ctx->u_dev;
    int n_save = ctx->n_cells, d_save = ctx->u_dtype;
    ctx->u_dev = ufb.p;
    ctx->n_cells = nfb;
    ctx->u_dtype = HEAT_F64;
    heat_opts fo = o;
    fo.cell_begin = 0;
    fo.cell_count = nfb;
    fo.ledger_out = o.ledger_out ? lfb.as<double>() : nullptr;
    h = heat_solve(ctx, &fo, nullptr, jfb.p, stream);
    ctx->u_dev = u_save;
    ctx->n_cells = n_save;
    ctx->u_dtype = d_save;
    if (h != HEAT_OK) return h;
    long long row = (long long)G * N;
    k_fallback_scatter<<<(unsigned)((nfb * row + 255) / 256), 256, 0, st>>>(nfb, row, list.as<int>(), jfb.as<float>(),
                                                                           j_out);
    if (o.ledger_out)
        k_fallback_ledger<<<(unsigned)((nfb * 2 * G + 255) / 256), 256, 0, st>>>(nfb, 2 * G, list.as<int>(),
                                                                                lfb.as<double>(), o.ledger_out);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(st));  // temporaries are released on return
    return HEAT_OK;
}

}  // extern "C"

namespace {

heat_status refresh_bf16(heat_ctx* ctx, Surrogate* s, int m, cudaStream_t st) {
    // BF16 copies of the FP32 master weights, and their transposes for the backward GEMMs
    for (int l = 0; l < kLayers; ++l) {
        long long n = (long long)s->Nout[l] * s->Kin[l];
        SCK(launch_to_bf16(n, s->Nout[l], s->Kin[l], Pm(s, m) + s->woff[l], Wb(s, m, l), WTb(s, m, l), st));
    }
    return HEAT_OK;
}

}  // namespace
