// Arithmetic peaks of the device, measured: the roofline of the FP64-bound kernels (the
// recursion, the exact build and emissivity, the thermal-discrete state reduction) is the
// FP64 FMA rate, known otherwise only as a nominal figure.  Every thread runs
// kChains independent FMA chains of kIters steps (no loads, no dependences between chains),
// enough blocks for full occupancy on every SM; the flop count is 2 per FMA.
#include <cuda_runtime.h>

#include "heat.h"

namespace heat {

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T a, T b, T* sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) sink[0] = s;  // keeps the chains live; never true for these inputs
}

template <typename T>
cudaError_t time_peak(int device, double* tflops) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, 256, 0)) != cudaSuccess) return e;
    const unsigned blocks = (unsigned)(sms * per_sm * 4);
    T* sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(T))) != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a multiplier just below 1 and a small addend keep every value finite and normal
    const T a = (T)0.999999, b = (T)1e-3;
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {  // the first launch warms the clocks; the fastest counts
        cudaEventRecord(e0, 0);
        k_fma_peak<T><<<blocks, 256>>>(a, b, sink);
        cudaEventRecord(e1, 0);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    const double flop = 2.0 * kChains * kIters * 256.0 * (double)blocks;
    *tflops = flop / ((double)best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace

}  // namespace heat

extern "C" heat_status heat_measure_fma_peak(int device, int fp64, double* tflops) {
    if (!tflops || device < 0) return HEAT_EINVAL;
    const cudaError_t e = fp64 ? heat::time_peak<double>(device, tflops) : heat::time_peak<float>(device, tflops);
    return e == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}
