// Element access by afmm_dtype for the conversion and scan kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cstdint>

#include "afmm.h"

namespace afmm {

template <int DT> struct Elem;

template <> struct Elem<AFMM_F64> {
    using T = double;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        return static_cast<const double*>(p)[i];
    }
};
template <> struct Elem<AFMM_F32> {
    using T = float;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        return static_cast<const float*>(p)[i];
    }
};
template <> struct Elem<AFMM_BF16> {
    using T = uint16_t;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        return __bfloat162float(
            __ushort_as_bfloat16(static_cast<const uint16_t*>(p)[i]));
    }
};
template <> struct Elem<AFMM_E4M3> {
    using T = uint8_t;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        __nv_fp8_e4m3 v;
        v.__x = static_cast<const uint8_t*>(p)[i];
        return static_cast<float>(v);
    }
};
template <> struct Elem<AFMM_I32> {
    using T = int32_t;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        return static_cast<const int32_t*>(p)[i];
    }
};
template <> struct Elem<AFMM_I8> {
    using T = int8_t;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        return static_cast<const int8_t*>(p)[i];
    }
};
template <> struct Elem<AFMM_U8> {
    using T = uint8_t;
    static __device__ __forceinline__ double get(const void* p, int64_t i) {
        return static_cast<const uint8_t*>(p)[i];
    }
};

// Calls f.template operator()<DT>() for the runtime dtype `dt`.
template <typename F>
inline afmm_status dispatch_dtype(int dt, F&& f) {
    switch (dt) {
        case AFMM_F64: return f.template operator()<AFMM_F64>();
        case AFMM_F32: return f.template operator()<AFMM_F32>();
        case AFMM_BF16: return f.template operator()<AFMM_BF16>();
        case AFMM_E4M3: return f.template operator()<AFMM_E4M3>();
        case AFMM_I32: return f.template operator()<AFMM_I32>();
        case AFMM_I8: return f.template operator()<AFMM_I8>();
        case AFMM_U8: return f.template operator()<AFMM_U8>();
        default: return AFMM_ERR_INVALID_ARG;
    }
}

}  // namespace afmm
