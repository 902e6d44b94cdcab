// Shared device-side definitions for the libheat CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace heat {

// CODATA 2018 exact values (CGS).
constexpr double kH = 6.62607015e-27;   // erg s
constexpr double kC = 2.99792458e10;    // cm s^-1
constexpr double kK = 1.380649e-16;     // erg K^-1
constexpr double kHC = kH * kC;         // erg cm (rounded product of the two)

// Device status bits (OR-ed into the context's status word).
constexpr int kStatNumeric = 1;   // zero cooling rate with non-zero inflow
constexpr int kStatBadInput = 2;  // non-finite or negative field value
constexpr int kStatTimeout = 4;   // bounded wait gave up


// Pattern entry of a band element, grouped by wavelength segment (the matrix build walks
// the segments in order and fills every element whose transition wavelength
// hc/(Elo_f - E_j) lies in the current one).  e is the element's index in the band
// storage (row-major over f, then j); t = ln(lambda_fj / lambda_n), 0 past the last node.
struct __align__(16) PatF64 {
    int e;
    int pad;
    double t;
};

// FP32 build: with a_n = u_n ca_n and z = (su_n + sC_n + 2) t,
//   B = Phi_n + u_n cat E1(fma(su_n, t, zt)),   cat = ca_n t,  zt = (sC_n + 2) t,
// where ca_n = C_n lambda_n^2 / h (0 on an inactive C segment).
struct __align__(16) PatF32 {  // one 128-bit load
    int e;
    float t;
    float cat;
    float zt;
};

// Band element in row order (the fused build + recursion of the mixed path): with the
// cell's photon prefix phi_n at the start of segment n and its field values (u_n, su_n),
//   B = phi_n + u_n cat E1(fmaf(su_n, t, zt))          (the same expression as PatF32)
// n = the segment of the transition wavelength; N-1 where it is at or beyond the last node
// (cat = t = zt = 0: B = the whole grid's prefix); N for a diagonal element whose transition
// wavelength is below the grid (no photon part: B = 0 before the intra-bin term).
struct __align__(16) RowEnt32 {
    int n;
    float t;
    float cat;
    float zt;
};

// Point-rule element (Eq. heating at the bin centres) of band element e = (u, j):
// T_uj = Omega(lambda_uj) fac with lambda_uj = hc / (E_u - E_j) in segment n at offset
// t = ln(lambda_uj / lambda_n), fac = lambda_uj^3 dE_u / (h^2 c); n = -1 where lambda_uj is
// off the grid (T = 0).  Entries run down each column j (u descending), so a column's
// suffix sums B_uj = B_{u+1,j} + T_uj come out in order.
struct __align__(8) PointEnt {
    int e;
    int n;
    double t;
    double fac;
};

// Soft-photon abscissa for the intra-bin term of row j+1:
// lambda_s = hc / (Elo_{j+1} - E_j) in segment n with offset t; n = -1 below the
// grid (all absorbed power counts), n = N-1 at or above the last node (none).
// The term is added to the diagonal band element (j+1, j), at band index e_diag;
// diag_in_band = 0 when that element's transition wavelength is below the grid (its
// photon part is zero and only the intra-bin term remains).
struct SoftF64 {
    int j;
    int n;
    double t;
    int e_diag;
    int diag_in_band;
};

// X > 2^800 for a positive finite double, tested on the exponent bits (integer pipe).
__device__ __forceinline__ bool above_rescale(double x) {
    return __double2hiint(x) > (int)((1023 + 800) << 20) - 1;
}

// E1(z) = (e^z - 1)/z in FP32: Taylor series for |z| < 0.5 (truncation below
// 1.2e-8 relative); for |z| >= 0.5, where e^z - 1 has no cancellation, the fast
// exponential (relative error a few 1e-7).
__device__ __forceinline__ float e1f(float z) {
    if (fabsf(z) < 0.5f) {
        float p = 1.0f / 40320.0f;
        p = fmaf(p, z, 1.0f / 5040.0f);
        p = fmaf(p, z, 1.0f / 720.0f);
        p = fmaf(p, z, 1.0f / 120.0f);
        p = fmaf(p, z, 1.0f / 24.0f);
        p = fmaf(p, z, 1.0f / 6.0f);
        p = fmaf(p, z, 0.5f);
        p = fmaf(p, z, 1.0f);
        return p;
    }
    // |z| >= 0.5: e^z - 1 loses no digits here; hardware exp2 and a fast divide
    return __fdividef(__expf(z) - 1.0f, z);
}

// E1(z) in FP64 (library expm1; exact at z = 0).
// E1 for |z| <= 0.25: Taylor to z^5 (truncation < 5e-8 relative, below FP32 rounding).
__device__ __forceinline__ float e1f_small(float z) {
    float p = 1.0f / 720.0f;
    p = fmaf(p, z, 1.0f / 120.0f);
    p = fmaf(p, z, 1.0f / 24.0f);
    p = fmaf(p, z, 1.0f / 6.0f);
    p = fmaf(p, z, 0.5f);
    return fmaf(p, z, 1.0f);
}

// Whether a segment's elements may use e1f_small: every argument there is z = q t with
// t in [0, dl] and q = su + sC + 2, so |z| <= |q| dl.
__device__ __forceinline__ bool short_series(float su, float sC, float dl) {
    return fabsf(su + sC + 2.0f) * dl <= 0.25f;
}

__device__ __forceinline__ double e1d(double z) {
    return z == 0.0 ? 1.0 : expm1(z) / z;
}

// E1(z) in FP64 for |z| <= 1/4 from its Taylor series sum_{k>=0} z^k / (k+1)!, to k = 12
// (the first dropped term is below 2e-19 relative): 12 FMAs instead of expm1 and a divide.
__device__ __forceinline__ double e1d_series(double z) {
    double p = 1.0 / 6227020800.0;  // 1/13!
    p = fma(p, z, 1.0 / 479001600.0);
    p = fma(p, z, 1.0 / 39916800.0);
    p = fma(p, z, 1.0 / 3628800.0);
    p = fma(p, z, 1.0 / 362880.0);
    p = fma(p, z, 1.0 / 40320.0);
    p = fma(p, z, 1.0 / 5040.0);
    p = fma(p, z, 1.0 / 720.0);
    p = fma(p, z, 1.0 / 120.0);
    p = fma(p, z, 1.0 / 24.0);
    p = fma(p, z, 1.0 / 6.0);
    p = fma(p, z, 0.5);
    return fma(p, z, 1.0);
}

// The same for |z| <= 1/16, to k = 8 (first dropped term below 5e-18 relative): 8 FMAs.
__device__ __forceinline__ double e1d_series_short(double z) {
    double p = 1.0 / 362880.0;  // 1/9!
    p = fma(p, z, 1.0 / 40320.0);
    p = fma(p, z, 1.0 / 5040.0);
    p = fma(p, z, 1.0 / 720.0);
    p = fma(p, z, 1.0 / 120.0);
    p = fma(p, z, 1.0 / 24.0);
    p = fma(p, z, 1.0 / 6.0);
    p = fma(p, z, 0.5);
    return fma(p, z, 1.0);
}

// Which FP64 form serves every argument z = q t with t in [0, dl] (per cell): 2 = the short
// series (|z| <= 1/16), 1 = the series (|z| <= 1/4), 0 = the library expm1.
__device__ __forceinline__ int series_class64(double q, double dl) {
    const double zmax = fabs(q) * dl;
    return zmax <= 0.0625 ? 2 : (zmax <= 0.25 ? 1 : 0);
}
__device__ __forceinline__ bool short_series64(double q, double dl) { return series_class64(q, dl) != 0; }
__device__ __forceinline__ double e1d_by_class(int cls, double z) {
    return cls == 2 ? e1d_series_short(z) : e1d_series(z);
}

// Compensated FP32 running sum (Knuth's TwoSum error term collected in c): s + c carries the
// sum of non-negative FP32 terms to about 2^-46 relative, on the FP32 pipes (a GB300 SM
// sub-partition's FP64 unit takes 64 cycles per warp instruction).  val() rounds it to FP32.
// The _rn intrinsics keep the compiler from fusing a product that feeds add() into an FMA,
// so the sum is the same wherever the term comes from.
struct Sum32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        s = t;
        c = __fadd_rn(c, err);
    }
    __device__ __forceinline__ float val() const { return __fadd_rn(s, c); }
    __device__ __forceinline__ double wide() const { return (double)s + (double)c; }
};

// Widen a non-negative finite float to double with integer operations only
// (rebias the exponent, shift the mantissa); zero and subnormals map to 0.
// Keeps the conversion off the FP64 pipe, which is the bound of the recursion.
__device__ __forceinline__ double widen_pos(float x) {
    unsigned b = __float_as_uint(x);
    unsigned hi = (b >> 3) + 0x38000000u;
    unsigned lo = b << 29;
    bool tiny = b < 0x00800000u;
    hi = tiny ? 0u : hi;
    lo = tiny ? 0u : lo;
    return __hiloint2double((int)hi, (int)lo);
}

}  // namespace heat
