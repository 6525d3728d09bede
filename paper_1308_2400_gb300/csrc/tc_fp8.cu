// Operand conversions of the FP8 (E4M3) tensor-core form: the real factor
// as four row-scaled E4M3 slices (fp8_split.cuh), the Rep-factors as E4M3
// (exact for the integers 0..16 and for every integral E4M3 value up to
// 448), rows kept (K-major A operand) or transposed (K-major B operand).
// One byte per element and slice; HBM-bound single passes, plus a column
// maximum pass when the split rows are the source's columns (Case B).
#include <cuda_runtime.h>

#include "afmm_common.cuh"
#include "elem.cuh"
#include "fp8_split.cuh"
#include "tc_gemm.cuh"
#include "tile_convert.cuh"

namespace afmm {
namespace {

constexpr int F8_THREADS = 256;

// Eight elements from column c of a row as floats (zero past n): one
// vector load when `vec` (rows aligned for it) and c + 8 <= n.
template <int DT>
__device__ __forceinline__ void load8_f(const void* row, int64_t c, int64_t n, bool vec,
                                        float (&v)[8]) {
    if (vec && c + 8 <= n) {
        alignas(16) typename Elem<DT>::T e[8];
        load8<DT>(row, c, e);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (float)Elem<DT>::get(e, t);
    } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = c + t < n ? (float)Elem<DT>::get(row, c + t) : 0.f;
    }
}

// Maximum of a uint over the block's 256 threads (every thread gets it).
__device__ __forceinline__ uint32_t block_max(uint32_t v, uint32_t* red) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();                   // red is reused row after row
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = red[threadIdx.x & 7];
#pragma unroll
    for (int o = 4; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sixteen values (already scaled for the split) as E4M3 bytes: REP, one
// slice that must equal the value (bad otherwise); else the four slices.
template <bool REP>
__device__ __forceinline__ void f8_encode16(const float (&v)[16], uint32_t (&w)[4][4],
                                            bool& bad) {
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        const int word = j >> 2, half = (j >> 1) & 1;
        if constexpr (REP) {
            const uint16_t q = e4m3x2_rn(v[j], v[j + 1]);
            const float2 b = e4m3x2_value(q);
            bad |= b.x != v[j] || b.y != v[j + 1];
            w[0][word] = half ? (w[0][word] | ((uint32_t)q << 16)) : (uint32_t)q;
        } else {
            uint16_t q[4];
            f8_split4(v[j], v[j + 1], q);
#pragma unroll
            for (int s = 0; s < 4; ++s)
                w[s][word] = half ? (w[s][word] | ((uint32_t)q[s] << 16)) : (uint32_t)q[s];
        }
    }
}

// Rows [r0, r1) of the row-major n x n source kept as K-major E4M3 rows,
// dst[(s * n + r) * ldk + c] (zero for n <= c < ldk; ldk a multiple of 16).
// REP: one exact slice (Rep-factors, which must also be non-negative
// integers: AFMM_ERR_NEGATIVE_REP / _NONINTEGER_REP).  Else the row's largest |value| (its
// FP32 bits in amax[r]) sets the shift and the four slices are written; a
// non-finite value is reported as AFMM_ERR_OVERFLOW_RISK.  One block per
// row: the maximum pass reads the row, the slicing pass reads it again
// (from L2) and writes 16 bytes per thread and slice.
template <int DT, bool REP>
__global__ void __launch_bounds__(F8_THREADS)
f8_rows_kernel(const void* __restrict__ src, int64_t n, int64_t lds, uint8_t* __restrict__ dst,
               int64_t ldk, int vec, uint32_t* __restrict__ amax, int* status, int64_t r0,
               int64_t r1) {
    __shared__ uint32_t red[8];
    using T = typename Elem<DT>::T;
    bool bad = false;
    int bits = 0;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const T* row = static_cast<const T*>(src) + r * lds;
        int sh = 0;
        if constexpr (!REP) {
            uint32_t m = 0;
            for (int64_t c = 8 * (int64_t)threadIdx.x; c < n; c += 8 * F8_THREADS) {
                float v[8];
                load8_f<DT>(row, c, n, vec != 0, v);
#pragma unroll
                for (int t = 0; t < 8; ++t) m = max(m, __float_as_uint(fabsf(v[t])));
            }
            m = block_max(m, red);
            if (threadIdx.x == 0) amax[r] = m;
            bad |= m >= 0x7F800000u;
            sh = f8_row_shift(m);
        }
        for (int64_t c = 16 * (int64_t)threadIdx.x; c < ldk; c += 16 * F8_THREADS) {
            float v[16];
            load8_f<DT>(row, c, n, vec != 0, *reinterpret_cast<float(*)[8]>(v));
            load8_f<DT>(row, c + 8, n, vec != 0, *reinterpret_cast<float(*)[8]>(v + 8));
            if constexpr (!REP) {
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] = f8_scale(v[t], sh);
            }
            if constexpr (REP) {
#pragma unroll
                for (int t = 0; t < 16; ++t) bits |= rep_bits(v[t]);
            }
            uint32_t w[4][4];
            f8_encode16<REP>(v, w, bad);
#pragma unroll
            for (int s = 0; s < (REP ? 1 : 4); ++s)
                *reinterpret_cast<uint4*>(dst + ((int64_t)s * n + r) * ldk + c) =
                    make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
        }
    }
    if (bad) bits |= kBadRange;
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

// amax[c] = FP32 bits of the largest |src[r][c]| over rows r (the caller
// zeroes amax; bits of non-negative floats order like the values, NaN
// above infinity).  Threads on consecutive columns, 64 rows per block.
template <int DT>
__global__ void __launch_bounds__(F8_THREADS)
f8_colmax_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                 uint32_t* __restrict__ amax) {
    const int64_t c = (int64_t)blockIdx.x * F8_THREADS + threadIdx.x;
    if (c >= n) return;
    const int64_t rb = (int64_t)blockIdx.y * 64, re = rb + 64 < n ? rb + 64 : n;
    uint32_t m = 0;
    for (int64_t r = rb; r < re; ++r)
        m = max(m, __float_as_uint(fabsf((float)Elem<DT>::get(src, r * lds + c))));
    atomicMax(amax + c, m);
}

// Columns become K-major rows: dst[(s * n + c) * ldk + r] from src[r][c],
// one 64 x 64 tile per block (tile_load_f32, then four threads per output
// row write 16 bytes each per slice).  REP: one exact slice.  Else column c
// is scaled by 2^f8_row_shift(amax[c]) and split into four slices.
template <int DT, bool REP>
__global__ void __launch_bounds__(F8_THREADS)
f8_transpose_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                    uint8_t* __restrict__ dst, int64_t ldk, int vec,
                    const uint32_t* __restrict__ amax, int* status) {
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    bool bad = false;
    tile_load_f32<DT>(src, n, lds, r0, c0, 3.0e38f, vec != 0, tile, bad);
    bad = false;       // the E4M3 checks below decide
    __syncthreads();
    const int cc = threadIdx.x >> 2, qq = threadIdx.x & 3;
    const int64_t c = c0 + cc, r = r0 + 16 * qq;
    if (c < n && r < ldk) {
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = tile[16 * qq + e][cc];
        if constexpr (!REP) {
            const uint32_t m = amax[c];
            bad |= m >= 0x7F800000u;
            const int sh = f8_row_shift(m);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = f8_scale(v[e], sh);
        }
        int bits = 0;
        if constexpr (REP) {
#pragma unroll
            for (int e = 0; e < 16; ++e) bits |= rep_bits(v[e]);
        }
        uint32_t w[4][4];
        f8_encode16<REP>(v, w, bad);
#pragma unroll
        for (int s = 0; s < (REP ? 1 : 4); ++s)
            *reinterpret_cast<uint4*>(dst + ((int64_t)s * n + c) * ldk + r) =
                make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
        if (bad) bits |= kBadRange;
        if (bits) atomicCAS(status, 0, bad_status(bits));
    }
}

}  // namespace

afmm_status tc_f8_rows(bool rep, const void* src, int dt, int64_t n, int64_t lds, void* dst,
                       int64_t ldk, uint32_t* amax, int* status, cudaStream_t st, int64_t r0,
                       int64_t r1) {
    if (r1 < 0) r1 = n;
    const int64_t rows = r1 - r0;
    if (rows <= 0) return AFMM_OK;
    if (ldk % 16 != 0) return AFMM_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)(rows < (1 << 20) ? rows : (1 << 20));
    const size_t es = dtype_size(dt), va = es * 8 < 16 ? es * 8 : 16;
    const int vec = (lds * es) % va == 0 && (reinterpret_cast<uintptr_t>(src) % va) == 0;
    auto* d = static_cast<uint8_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        if (rep)
            f8_rows_kernel<DT, true><<<grid, F8_THREADS, 0, st>>>(src, n, lds, d, ldk, vec,
                                                                  amax, status, r0, r1);
        else
            f8_rows_kernel<DT, false><<<grid, F8_THREADS, 0, st>>>(src, n, lds, d, ldk, vec,
                                                                   amax, status, r0, r1);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status tc_f8_transpose(bool rep, const void* src, int dt, int64_t n, int64_t lds,
                            void* dst, int64_t ldk, uint32_t* amax, int* status,
                            cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 16 != 0) return AFMM_ERR_INVALID_ARG;
    const int64_t g = (n + 63) / 64;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    const int vec = rows_aligned16(src, lds, (int64_t)dtype_size(dt));
    auto* d = static_cast<uint8_t*>(dst);
    if (!rep) AFMM_CUDA_TRY(cudaMemsetAsync(amax, 0, (size_t)n * sizeof(uint32_t), st));
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        if (rep) {
            f8_transpose_kernel<DT, true><<<dim3((unsigned)g, (unsigned)g), F8_THREADS, 0, st>>>(
                src, n, lds, d, ldk, vec, amax, status);
        } else {
            f8_colmax_kernel<DT><<<dim3((unsigned)((n + F8_THREADS - 1) / F8_THREADS),
                                        (unsigned)g),
                                   F8_THREADS, 0, st>>>(src, n, lds, amax);
            f8_transpose_kernel<DT, false><<<dim3((unsigned)g, (unsigned)g), F8_THREADS, 0,
                                             st>>>(src, n, lds, d, ldk, vec, amax, status);
        }
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(rep ? 1 : 2);
    return AFMM_OK;
}

}  // namespace afmm
