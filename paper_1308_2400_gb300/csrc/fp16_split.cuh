// FP16 two-slice form of the real factor (split half precision for FP32
// products; Ootomo and Yokota, IJHPCA 2022, here with one exact integer
// factor): each row is scaled by a power of two so that its largest
// |value| lies in [2^14, 2^15), then every scaled value v is written as
// hi + lo 2^-8, hi = v rounded to 8 significant bits (an FP16 value) and lo
// = (v - hi) 2^8 rounded to FP16 (11 bits).  v - hi is exact in FP32, so
// hi + lo 2^-8 equals v to within 2^-20 |v| (and to 2^-46 of the row's
// largest value where FP16's subnormal range cuts the slices short).
// Rep-factors up to 2048 are exact in FP16, so the products hi Y and lo Y
// on the FP16 tensor path, in two FP32 accumulators, take two MMAs per k
// step where three BF16 slices take three.  hi keeps 8 bits, like the
// BF16 hi slice, because the tensor pipe's FP32 sums drop low bits of
// products much smaller than the running sum: an 11-bit hi (16-bit
// products with the Rep-factors) measured 1.5e-6 relative error at
// n = 8192, past the FP32 target, where 8 bits keep products of 13.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "fp8_split.cuh"

namespace afmm {

// The shift sh of a row whose largest |value| has FP32 bits m: m 2^sh lies
// in [2^14, 2^15).  0 for an all-zero or a non-finite row.
__device__ __forceinline__ int h16_row_shift(uint32_t m) {
    if (m == 0u || m >= 0x7F800000u) return 0;
    const int be = (int)(m >> 23);
    const int e = be > 0 ? be - 127 : (31 - __clz((int)m)) - 149;
    return 14 - e;
}

// The two FP16 slices of a scaled value v (|v| < 2^15), as raw bits: hi
// rounds v to 8 significant bits (to nearest even, the BF16 rounding; FP16
// holds the result unless it falls in its subnormal range, where it rounds
// again), lo the exact remainder times 2^8.
__device__ __forceinline__ void h16_split2(float v, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(__bfloat162float(__float2bfloat16_rn(v)));
    const __half l = __float2half_rn((v - __half2float(h)) * 256.f);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
}

}  // namespace afmm
