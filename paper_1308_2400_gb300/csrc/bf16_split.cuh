// Device helpers that turn operand values into BF16 tensor-core operands:
// exact widening of Rep-factors and the hi/mid/lo split of real values.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "elem.cuh"

namespace afmm {

// Whether a dtype's values are exact in FP32 (then the split runs in FP32;
// FP64 arithmetic is slow on this part and kept off the hot path).
template <int DT>
constexpr bool kExactInF32 = DT != AFMM_F64 && DT != AFMM_I32;

// Round-to-nearest BF16 slices of v: out[0] = bf16(v), out[s] = bf16 of the
// residual left by out[0..s-1].  Each residual is exact in the arithmetic
// used (FP32 for FP32-exact inputs, FP64 otherwise).
template <int S, typename T>
__device__ __forceinline__ void split_bf16(T v, __nv_bfloat16 (&out)[S]) {
    T r = v;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if constexpr (sizeof(T) == 8) out[s] = __double2bfloat16(r);
        else out[s] = __float2bfloat16_rn(r);
        r -= (T)__bfloat162float(out[s]);
    }
}

template <int DT>
__device__ __forceinline__ auto load_val(const void* p, int64_t i) {
    if constexpr (kExactInF32<DT>) return (float)Elem<DT>::get(p, i);
    else return Elem<DT>::get(p, i);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) |
           ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Runtime-dtype read as double (for kernels that serve several dtypes per
// launch, e.g. the grouped conversions of a batch).
__device__ __forceinline__ double load_any(const void* p, int64_t i, int dt) {
    switch (dt) {
        case AFMM_F64: return Elem<AFMM_F64>::get(p, i);
        case AFMM_F32: return Elem<AFMM_F32>::get(p, i);
        case AFMM_BF16: return Elem<AFMM_BF16>::get(p, i);
        case AFMM_E4M3: return Elem<AFMM_E4M3>::get(p, i);
        case AFMM_I32: return Elem<AFMM_I32>::get(p, i);
        case AFMM_I8: return Elem<AFMM_I8>::get(p, i);
        default: return Elem<AFMM_U8>::get(p, i);
    }
}

// Runtime-dtype read as float (FP64 values are rounded to FP32; integers
// above 2^24 lose their low bits, which the exactness checks then flag).
__device__ __forceinline__ float load_any_f(const void* p, int64_t i, int dt) {
    switch (dt) {
        case AFMM_F64: return (float)static_cast<const double*>(p)[i];
        case AFMM_F32: return static_cast<const float*>(p)[i];
        case AFMM_BF16:
            return __bfloat162float(__ushort_as_bfloat16(static_cast<const uint16_t*>(p)[i]));
        case AFMM_E4M3: {
            __nv_fp8_e4m3 v;
            v.__x = static_cast<const uint8_t*>(p)[i];
            return static_cast<float>(v);
        }
        case AFMM_I32: return (float)static_cast<const int32_t*>(p)[i];
        case AFMM_I8: return (float)static_cast<const int8_t*>(p)[i];
        default: return (float)static_cast<const uint8_t*>(p)[i];
    }
}

}  // namespace afmm
