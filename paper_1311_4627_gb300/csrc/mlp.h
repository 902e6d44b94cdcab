// Surrogate MLP kernels: parameters and launchers (k_mlp.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace heat {

constexpr int kMaxGemmZ = 8;  // batched problems per launch (ensemble members)

struct GemmTcParams {
    CUtensorMap ta[kMaxGemmZ];  // A[z]: M x K BF16, K-major, 128B swizzle, box (64, 128)
    CUtensorMap tb[kMaxGemmZ];  // B[z]: N x K BF16, K-major, box (64, 128)
    float* c[kMaxGemmZ];        // FP32 output (or null), row stride ldc
    __nv_bfloat16* cb[kMaxGemmZ];  // BF16 output (or null), row stride ldcb
    const float* bias[kMaxGemmZ];  // per-column bias (or null)
    long long ldc, ldcb;
    int M, N, K, nz;               // K a multiple of 64
    int mtiles, ntiles;
    int accumulate;                // 1: c += result
    int act;                       // 1: the BF16 output is GELU of the result (the FP32 output is not)
    long long wait_polls;          // polls before a wait on another role gives up (kStatTimeout)
    int* status;
};

cudaError_t launch_gemm_bf16(const GemmTcParams& p, int sms, cudaStream_t st);
cudaError_t launch_to_bf16(long long n, int rows, int cols, const float* w, __nv_bfloat16* Wb, __nv_bfloat16* WTb,
                           cudaStream_t st);
cudaError_t launch_count_valid(long long n, const float* T, unsigned long long* count, cudaStream_t st);
cudaError_t launch_gelu_fwd(long long n, const float* Z, __nv_bfloat16* X, cudaStream_t st);
cudaError_t launch_gelu_bwd(long long n, const float* dX, const float* Z, __nv_bfloat16* dZ, cudaStream_t st);
cudaError_t launch_transpose_bf16(int rows, int cols, const __nv_bfloat16* in, __nv_bfloat16* out, cudaStream_t st);
cudaError_t launch_colsum_bf16(int rows, int cols, const __nv_bfloat16* A, float* out, cudaStream_t st);
// Rows of N standardised outputs Y against targets T: d = Y - T where T is finite; where T is
// NaN and tb (per-row mask level in raw units, or null) is given, d = 0.3 max(0, raw Y - tb)
// in standardised units (ym, ys de-standardise).  dY = 2 d / count, loss_acc (or null) += sum
// d^2 / count, count = finite targets (device).
cudaError_t launch_mse(long long n, int N, const float* Y, const float* T, const float* tb, const float* ym,
                       const float* ys, const unsigned long long* count, __nv_bfloat16* dY, double* loss_acc,
                       cudaStream_t st);
cudaError_t launch_adam(long long n, int rows, int cols, float* w, const float* g, float* m, float* v, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, __nv_bfloat16* Wb, __nv_bfloat16* WTb,
                        cudaStream_t st);

}  // namespace heat
