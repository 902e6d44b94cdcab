// Rounding of the emissivity's P operand (Eq. emission on the tensor cores): P of a (cell,
// grain) row divided by the row's power-of-two scale, rounded to FP32, then to BF16 or TF32
// with a hi + lo split.  Shared by the packing kernel and the recursion's epilogue, so that
// both give the same bits.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace heat {

__device__ __forceinline__ uint16_t bf16_rn(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_f(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// Round an FP32 value to TF32 (10 explicit mantissa bits), ties away from zero.
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// P * 2^-e rounded to FP32 (to nearest even) with integer operations only: P >= 0 is an
// FP64 value and e its row's scale exponent; results below the FP32 normal range flush
// to 0.  The FP64 pipe (one warp-wide instruction per 64 cycles on this part) stays out
// of the packing, which is then bound by its memory traffic.
__device__ __forceinline__ float scaled_to_f32(double p, int e) {
    const unsigned hi = (unsigned)__double2hiint(p), lo = (unsigned)__double2loint(p);
    const int fe = (int)(hi >> 20) - e - 896;  // FP32 biased exponent of p * 2^-e
    if (fe <= 0) return 0.0f;
    const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    unsigned fb = ((unsigned)fe << 23) | m23;
    fb += (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
    return __uint_as_float(fb);
}

// The frexp exponent of a row's largest P from the high word of that FP64 value (P >= 0, so
// the largest value has the largest high word): m = f 2^e with f in [0.5, 1); 0 for a row
// of zeros (or of subnormals).
__device__ __forceinline__ int row_scale_exp(unsigned max_hi) {
    return max_hi >= 0x00100000u ? (int)(max_hi >> 20) - 1022 : 0;
}

}  // namespace heat
