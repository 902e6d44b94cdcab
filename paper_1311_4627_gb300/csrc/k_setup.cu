// Grain set-up kernels: cooling rates (Eq. cooling) and Planck kernels (Eq. emission).
// Run once per heat_set_grains; FP64 throughout.
#include "common.cuh"
#include "internal.h"

namespace heat {

__constant__ double c_gl_x[kGLPoints];  // Gauss-Legendre nodes on [-1, 1]
__constant__ double c_gl_w[kGLPoints];  // and weights

// Integrand of the emitted power in y = ln(lambda): C(lambda) B_lambda(T) lambda.
__device__ __forceinline__ double cool_integrand(double lam, double c_lam, double T) {
    double x = kHC / (lam * kK * T);
    if (x > 745.0) return 0.0;
    double l2 = lam * lam;
    double bl = 2.0 * kH * kC * kC / (l2 * l2 * lam) / expm1(x);
    return c_lam * bl * lam;
}

// Gauss-Legendre panel over [ya, yb] in y = ln(lambda) of a power-law cross-section
// C = c0 (lambda/lam0)^s.
__device__ double cool_panel(double ya, double yb, double c0, double lam0, double s, double T) {
    double m = 0.5 * (ya + yb), r = 0.5 * (yb - ya), acc = 0.0;
#pragma unroll 4
    for (int k = 0; k < kGLPoints; ++k) {
        double lam = exp(m + r * c_gl_x[k]);
        double c = c0 * pow(lam / lam0, s);
        acc += c_gl_w[k] * cool_integrand(lam, c, T);
    }
    return acc * r;
}

// One warp per (grain, bin f >= 1):
//   Cf = 4 pi int_{hc/E_f}^inf C(lambda) B_lambda(T_f) dlambda / (E_f - E_{f-1})
// with C the log-log interpolant of the nodes inside the grid and its end-segment
// power law beyond.  Panels: every grid segment above the cut-off, 100 panels of
// 0.25 in ln(lambda) past the last node, and 0.25-wide panels below the first node
// down to the cut-off (or to hc/(800 k T), where the integrand is below 1e-340).
__global__ void k_cooling(int N, const double* __restrict__ lam, const double* __restrict__ cabs,
                          const int* __restrict__ bin_off, int G, const double* __restrict__ T,
                          const double* __restrict__ E, double* __restrict__ Cf, const int2* __restrict__ work,
                          int n_work) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n_work) return;
    int g = work[warp].x, f = work[warp].y;
    int off = bin_off[g];
    const double* C = cabs + (size_t)g * N;
    double Tf = T[off + f], Ef = E[off + f];
    double lcut = kHC / Ef;
    double lmin = kHC / (800.0 * kK * Tf);
    double lo = lcut > lmin ? lcut : lmin;
    double acc = 0.0;
    // grid segments
    for (int n = lane; n < N - 1; n += 32) {
        double a = lam[n], b = lam[n + 1];
        if (b <= lo || !(C[n] > 0.0 && C[n + 1] > 0.0)) continue;
        double s = log(C[n + 1] / C[n]) / log(b / a);
        double ya = log(a > lo ? a : lo), yb = log(b);
        acc += cool_panel(ya, yb, C[n], a, s, Tf);
    }
    // past the last node
    if (C[N - 2] > 0.0 && C[N - 1] > 0.0) {
        double s = log(C[N - 1] / C[N - 2]) / log(lam[N - 1] / lam[N - 2]);
        double y0 = log(lam[N - 1] > lo ? lam[N - 1] : lo);
        for (int k = lane; k < 100; k += 32) acc += cool_panel(y0 + 0.25 * k, y0 + 0.25 * (k + 1), C[N - 1], lam[N - 1], s, Tf);
    }
    // below the first node
    if (lo < lam[0] && C[0] > 0.0 && C[1] > 0.0) {
        double s = log(C[1] / C[0]) / log(lam[1] / lam[0]);
        double ytop = log(lam[0]), ybot = log(lo);
        int np = (int)ceil((ytop - ybot) / 0.25);
        for (int k = lane; k < np; k += 32) {
            double yb = ytop - 0.25 * k, ya = yb - 0.25;
            if (ya < ybot) ya = ybot;
            acc += cool_panel(ya, yb, C[0], lam[0], s, Tf);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const double pi = 3.141592653589793;
        double p_emit = 4.0 * pi * acc;
        Cf[off + f] = p_emit / (Ef - E[off + f - 1]);
    }
}

// K[bin][n] = C_n B_lambda_n(T_i) [E_i >= hc/lambda_n] (FP64), and the size-weighted
// copy Kw = w_g K when weights are given.
__global__ void k_planck(int N, int nbt, const double* __restrict__ lam, const double* __restrict__ cabs,
                         const int* __restrict__ bin_grain, const double* __restrict__ T,
                         const double* __restrict__ E, const double* __restrict__ w, double* __restrict__ K,
                         double* __restrict__ Kw) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nbt * N) return;
    int i = (int)(idx / N), n = (int)(idx % N);
    int g = bin_grain[i];
    double l = lam[n];
    double v = 0.0;
    if (E[i] >= kHC / l) {
        double x = kHC / (l * kK * T[i]);
        if (x <= 745.0) {
            double l2 = l * l;
            v = cabs[(size_t)g * N + n] * (2.0 * kH * kC * kC / (l2 * l2 * l) / expm1(x));
        }
    }
    K[idx] = v;
    if (Kw) Kw[idx] = w[g] * v;
}

cudaError_t launch_cooling(int N, const double* lam, const double* cabs, const int* bin_off, int G, const double* T,
                           const double* E, double* Cf, const int2* work, int n_work, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    int threads = 128;
    int blocks = (n_work * 32 + threads - 1) / threads;
    k_cooling<<<blocks, threads, 0, st>>>(N, lam, cabs, bin_off, G, T, E, Cf, work, n_work);
    return cudaGetLastError();
}

cudaError_t launch_planck(int N, int nbt, const double* lam, const double* cabs, const int* bin_grain, const double* T,
                          const double* E, const double* w, double* K, double* Kw, cudaStream_t st) {
    long long total = (long long)nbt * N;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    k_planck<<<(unsigned)blocks, threads, 0, st>>>(N, nbt, lam, cabs, bin_grain, T, E, w, K, Kw);
    return cudaGetLastError();
}

// Binary exponent (biased, as stored in the double) of Kmax_i = max_lambda K[i][lambda], the
// largest emission kernel of bin i; warp per bin.  -100000 where the bin emits nothing on the grid.
__global__ void k_kexp(int N, int nbt, const double* __restrict__ K, int* __restrict__ kexp) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nbt) return;
    double m = 0.0;
    for (int n = lane; n < N; n += 32) m = fmax(m, K[(size_t)w * N + n]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) kexp[w] = m > 0.0 ? ((__double2hiint(m) >> 20) & 0x7ff) : -100000;
}

cudaError_t launch_kexp(int N, int nbt, const double* K, int* kexp, cudaStream_t st) {
    const long long threads = (long long)nbt * 32;
    k_kexp<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, nbt, K, kexp);
    return cudaGetLastError();
}

cudaError_t set_gauss_legendre(const double* x, const double* w) {
    cudaError_t e = cudaMemcpyToSymbol(c_gl_x, x, sizeof(double) * kGLPoints);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_gl_w, w, sizeof(double) * kGLPoints);
}

}  // namespace heat
