// Emissivity contraction (Eq. emission, Eq. emission-lambda) in FP64:
//   j[c][g][n] = sum_i P[c][off_g + i] K[off_g + i][n],   K = C_abs B_lambda(T_i) [E_i >= hc/lambda_n],
// and the size-integrated form over the concatenated bins with K scaled by w_g (Eq. convolution).
// Register-tiled SIMT GEMM on the FP64 FMA pipe: 64 x 64 output tile per block,
// 16-deep k slices staged in shared memory, 4 x 4 outputs per thread; a thread-per-output
// form for few rows.
#include "common.cuh"
#include "internal.h"

namespace heat {

template <typename TC>
__global__ void __launch_bounds__(256, 2) k_gemm_f64(int M, int N, const int* __restrict__ koff,
                                                  const double* __restrict__ A, long long lda,
                                                  const double* __restrict__ B, long long ldb, TC* __restrict__ C,
                                                  long long ldc, long long zs) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][64];
    const int z = blockIdx.z;
    const int k0 = koff[z], k1 = koff[z + 1];
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = 0.0;
    for (int kb = k0; kb < k1; kb += 16) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + 256 * r;
            int mm = idx >> 4, kk = idx & 15;
            double v = 0.0;
            if (m0 + mm < M && kb + kk < k1) v = A[(size_t)(m0 + mm) * lda + kb + kk];
            As[kk][mm] = v;
            int kr = idx >> 6, nn = idx & 63;
            double w = 0.0;
            if (kb + kr < k1 && n0 + nn < N) w = B[(size_t)(kb + kr) * ldb + n0 + nn];
            Bs[kr][nn] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int s = 0; s < 4; ++s) b[s] = Bs[kk][tx + 16 * s];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
        }
        __syncthreads();
    }
    TC* Cz = C + (size_t)z * zs;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int m = m0 + ty + 16 * r;
        if (m >= M) continue;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int n = n0 + tx + 16 * s;
            if (n < N) Cz[(size_t)m * ldc + n] = (TC)acc[r][s];
        }
    }
}

// Few rows (solves of few cells): a thread per output, threads along n (coalesced rows of K),
// one accumulator in ascending k as in k_gemm_f64, so both give the same bits; the 64-row
// tile above would spend 64 FMAs per useful one on a single cell.
template <typename TC>
__global__ void __launch_bounds__(128) k_gemv_f64(int N, const int* __restrict__ koff, const double* __restrict__ A,
                                                  long long lda, const double* __restrict__ B, long long ldb,
                                                  TC* __restrict__ C, long long ldc, long long zs) {
    const int z = blockIdx.z, m = blockIdx.y, n = blockIdx.x * 128 + threadIdx.x;
    if (n >= N) return;
    const int k0 = koff[z], k1 = koff[z + 1];
    const double* a = A + (size_t)m * lda;
    double acc = 0.0;
    for (int k = k0; k < k1; ++k) acc = fma(a[k], B[(size_t)k * ldb + n], acc);
    C[(size_t)z * zs + (size_t)m * ldc + n] = (TC)acc;
}

cudaError_t launch_gemm_f64(int M, int N, int nz, const int* koff, const double* A, long long lda, const double* B,
                            long long ldb, void* C, long long ldc, long long zstride_c, int c_is_f32, cudaStream_t st) {
    if (M <= 0 || N <= 0 || nz <= 0) return cudaSuccess;
    if (M <= kSmallCells) {
        dim3 g1((N + 127) / 128, M, nz);
        if (c_is_f32)
            k_gemv_f64<float><<<g1, 128, 0, st>>>(N, koff, A, lda, B, ldb, (float*)C, ldc, zstride_c);
        else
            k_gemv_f64<double><<<g1, 128, 0, st>>>(N, koff, A, lda, B, ldb, (double*)C, ldc, zstride_c);
        return cudaGetLastError();
    }
    dim3 grid((N + 63) / 64, (M + 63) / 64, nz);
    if (c_is_f32)
        k_gemm_f64<float><<<grid, 256, 0, st>>>(M, N, koff, A, lda, B, ldb, (float*)C, ldc, zstride_c);
    else
        k_gemm_f64<double><<<grid, 256, 0, st>>>(M, N, koff, A, lda, B, ldb, (double*)C, ldc, zstride_c);
    return cudaGetLastError();
}

}  // namespace heat
