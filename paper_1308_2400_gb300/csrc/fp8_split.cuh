// Device helpers of the FP8 (E4M3) tensor-core form: round-to-nearest E4M3
// conversion, the per-row power-of-two scaling and the four-slice split of
// a real value.  Shared by the conversions (tc_fp8.cu), which scale and
// split, and the product's epilogue (tc_gemm.cu), which undoes the scale.
//
// E4M3 holds 4 significant bits (3 stored), normal exponents -6 .. 8,
// subnormals down to 2^-9, largest finite value 448.  A row of the real
// factor scaled by 2^sh so that its largest |value| lies in [128, 256)
// splits as v = q1 + q2 + q3 + 2^-12 q4 + rest: q1..q3 are the E4M3
// roundings of v and of its residuals, q4 that of the third residual times
// 2^12 (the residual itself is below 2^-7, in E4M3's subnormal range).
// Each rounding is to nearest with ties to even and keeps 4 significant
// bits (fewer for subnormals), so every residual is exact in FP32 and the
// rest is at most 2^-16 |v| or 2^-21 times the row's largest |value|,
// whichever is larger.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace afmm {

// E4M3 of two floats, round to nearest even, saturating at +-448; lo in the
// low byte.
__device__ __forceinline__ uint16_t e4m3x2_rn(float lo, float hi) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}

// The two E4M3 values of q (low byte first) as floats, exactly (every
// E4M3 value is an FP16 value).
__device__ __forceinline__ float2 e4m3x2_value(uint16_t q) {
    uint32_t h;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h) : "h"(q));
    __half2 v;
    *reinterpret_cast<uint32_t*>(&v) = h;
    return __half22float2(v);
}

// Shift sh with |v| 2^sh < 256 for every |v| up to the maximum whose FP32
// bits are given (the largest |value| of a row): sh = 7 - floor(log2 max).
// 0 for a zero or non-finite maximum.
__device__ __forceinline__ int f8_row_shift(uint32_t max_bits) {
    if (max_bits == 0u || max_bits >= 0x7F800000u) return 0;
    const int be = (int)(max_bits >> 23);
    const int e = be > 0 ? be - 127 : (31 - __clz((int)max_bits)) - 149;
    return 7 - e;
}

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float f8_pow2(int e) { return __int_as_float((127 + e) << 23); }

// v 2^sh for a row shift (-120 <= sh <= 156), as two exact scalings.
__device__ __forceinline__ float f8_scale(float v, int sh) {
    const int e1 = sh < 127 ? sh : 127;
    return v * f8_pow2(e1) * f8_pow2(sh - e1);
}

// Four E4M3 slices of two scaled values (|v| < 256): q[s] holds slice s
// of v0 in its low byte and of v1 in its high byte.
__device__ __forceinline__ void f8_split4(float v0, float v1, uint16_t (&q)[4]) {
    float r0 = v0, r1 = v1;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        q[s] = e4m3x2_rn(r0, r1);
        const float2 b = e4m3x2_value(q[s]);
        r0 -= b.x;
        r1 -= b.y;
    }
    q[3] = e4m3x2_rn(r0 * 0x1p12f, r1 * 0x1p12f);
}

}  // namespace afmm
