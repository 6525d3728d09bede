// Conversions of the FP16 two-slice tensor-core form (fp16_split.cuh):
// the real factor scaled by a power of two per row of the A operand and
// written as two K-major FP16 slices -- Case A from the rows of X (one
// block per row: a maximum pass, then the slicing pass reading the row
// again from L2), Case B from the columns of Y (a column-maximum pass,
// then 64 x 64 tiles transposed through shared memory) -- and the
// Rep-factors of Case B as exact FP16 rows.  HBM-bound.
#include <cuda_runtime.h>

#include "afmm_common.cuh"
#include "elem.cuh"
#include "fp16_split.cuh"
#include "tc_gemm.cuh"
#include "tile_convert.cuh"

namespace afmm {
namespace {

constexpr int H16_THREADS = 256;

// Columns c .. c+7 of `row` as floats, zero from column n on; one vector
// load when `vec` (rows aligned for it) and the eight lie inside the row.
template <int DT>
__device__ __forceinline__ void row8(const void* row, int64_t c, int64_t n, bool vec,
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

// Largest of v over the block's 256 threads, returned to every thread
// (`red` holds one word per warp and is reused row after row).
__device__ __forceinline__ uint32_t block_max256(uint32_t v, uint32_t* red) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = red[threadIdx.x & 7];
#pragma unroll
    for (int o = 4; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Rows [r0, r1): amax[r] = FP32 bits of the row's largest |value| (the bit
// patterns of non-negative floats order like their values), then slice 0
// (hi) and slice 1 (lo) of every value scaled by 2^h16_row_shift(amax[r]).
template <int DT>
__global__ void __launch_bounds__(H16_THREADS)
h16_rows_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                uint16_t* __restrict__ dst, int64_t ldk, int vec, uint32_t* __restrict__ amax,
                int* status, int64_t r0, int64_t r1) {
    __shared__ uint32_t red[8];
    using T = typename Elem<DT>::T;
    bool bad = false;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const T* row = static_cast<const T*>(src) + r * lds;
        uint32_t m = 0;
        for (int64_t c = 8 * (int64_t)threadIdx.x; c < n; c += 8 * H16_THREADS) {
            float v[8];
            row8<DT>(row, c, n, vec != 0, v);
#pragma unroll
            for (int t = 0; t < 8; ++t) m = max(m, __float_as_uint(fabsf(v[t])));
        }
        m = block_max256(m, red);
        if (threadIdx.x == 0) amax[r] = m;
        bad |= m >= 0x7F800000u;
        const int sh = h16_row_shift(m);
        for (int64_t c = 8 * (int64_t)threadIdx.x; c < ldk; c += 8 * H16_THREADS) {
            float v[8];
            row8<DT>(row, c, n, vec != 0, v);
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                uint16_t h0, l0, h1, l1;
                h16_split2(f8_scale(v[t], sh), h0, l0);
                h16_split2(f8_scale(v[t + 1], sh), h1, l1);
                hw[t / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                lw[t / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
            *reinterpret_cast<uint4*>(dst + r * ldk + c) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(dst + (n + r) * ldk + c) =
                make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
    if (bad) atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
}

// amax[c] = FP32 bits of the largest |src[r][c]| over rows r (the caller
// zeroes amax).  Threads on consecutive columns, 64 rows per block.
template <int DT>
__global__ void __launch_bounds__(H16_THREADS)
h16_colmax_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                  uint32_t* __restrict__ amax) {
    const int64_t c = (int64_t)blockIdx.x * H16_THREADS + threadIdx.x;
    if (c >= n) return;
    const int64_t rb = (int64_t)blockIdx.y * 64, re = rb + 64 < n ? rb + 64 : n;
    uint32_t m = 0;
    for (int64_t r = rb; r < re; ++r)
        m = max(m, __float_as_uint(fabsf((float)Elem<DT>::get(src, r * lds + c))));
    atomicMax(amax + c, m);
}

// Columns of the source become K-major rows of two FP16 slices:
// dst[(s * n + c) * ldk + r] from src[r][c] scaled by 2^h16_row_shift
// (amax[c]).  One 64 x 64 tile per block through shared memory; four
// threads per output row, 16 values (32 bytes per slice) each.
template <int DT>
__global__ void __launch_bounds__(H16_THREADS)
h16_transpose_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                     uint16_t* __restrict__ dst, int64_t ldk, int vec,
                     const uint32_t* __restrict__ amax, int* status) {
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    bool unused = false;
    tile_load_f32<DT>(src, n, lds, r0, c0, 3.0e38f, vec != 0, tile, unused);
    __syncthreads();
    const int cc = threadIdx.x >> 2, qq = threadIdx.x & 3;
    const int64_t c = c0 + cc, r = r0 + 16 * qq;
    if (c >= n || r >= ldk) return;
    const uint32_t m = amax[c];
    if (m >= 0x7F800000u) atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
    const int sh = h16_row_shift(m);
    uint32_t hw[8], lw[8];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
        uint16_t h0, l0, h1, l1;
        h16_split2(f8_scale(tile[16 * qq + e][cc], sh), h0, l0);
        h16_split2(f8_scale(tile[16 * qq + e + 1][cc], sh), h1, l1);
        hw[e / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
        lw[e / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
    // ldk is a multiple of 8: the last run of a row may hold 8 values.
    const bool whole = r + 16 <= ldk;
    uint16_t* oh = dst + c * ldk + r;
    uint16_t* ol = dst + (n + c) * ldk + r;
    *reinterpret_cast<uint4*>(oh) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(ol) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    if (whole) {
        *reinterpret_cast<uint4*>(oh + 8) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
        *reinterpret_cast<uint4*>(ol + 8) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
    }
}

// Rep-factors rows kept as FP16 (the K-major B operand of Case B):
// dst[r * ldk + c], exact and |v| <= lim (AFMM_ERR_OVERFLOW_RISK
// otherwise), non-negative integers (AFMM_ERR_NEGATIVE_REP /
// _NONINTEGER_REP otherwise); eight columns per thread, zero from n on.
template <int DT>
__global__ void __launch_bounds__(H16_THREADS)
h16_rep_rows_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                    uint16_t* __restrict__ dst, int64_t ldk, int vec, float lim, int* status) {
    const int64_t c = ((int64_t)blockIdx.x * H16_THREADS + threadIdx.x) * 8;
    if (c >= ldk) return;
    int bits = 0;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        float v[8];
        row8<DT>(static_cast<const typename Elem<DT>::T*>(src) + r * lds, c, n, vec != 0, v);
        uint32_t w[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            uint32_t q[1];
            bits |= convert_pair<1, true, true>(v[t], v[t + 1], lim, true, q);
            w[t / 2] = q[0];
        }
        *reinterpret_cast<uint4*>(dst + r * ldk + c) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

}  // namespace

afmm_status tc_h16_transpose(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                             int64_t ldk, uint32_t* amax, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 8 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const int64_t g = (n + 63) / 64;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    const int vec = rows_aligned16(src, lds, (int64_t)dtype_size(dt));
    auto* d = static_cast<uint16_t*>(dst);
    AFMM_CUDA_TRY(cudaMemsetAsync(amax, 0, (size_t)n * sizeof(uint32_t), st));
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        h16_colmax_kernel<DT><<<dim3((unsigned)((n + H16_THREADS - 1) / H16_THREADS),
                                     (unsigned)g),
                                H16_THREADS, 0, st>>>(src, n, lds, amax);
        h16_transpose_kernel<DT><<<dim3((unsigned)g, (unsigned)g), H16_THREADS, 0, st>>>(
            src, n, lds, d, ldk, vec, amax, status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFMM_OK;
}

afmm_status tc_h16_rep_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                            int64_t ldk, float lim, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 8 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const dim3 grid((unsigned)((ldk / 8 + H16_THREADS - 1) / H16_THREADS),
                    (unsigned)(n < 65535 ? n : 65535));
    const size_t es = dtype_size(dt), va = es * 8 < 16 ? es * 8 : 16;
    const int vec = (lds * es) % va == 0 && (reinterpret_cast<uintptr_t>(src) % va) == 0;
    auto* d = static_cast<uint16_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        h16_rep_rows_kernel<DT><<<grid, H16_THREADS, 0, st>>>(src, n, lds, d, ldk, vec, lim,
                                                              status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status tc_h16_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                        int64_t ldk, uint32_t* amax, int* status, cudaStream_t st, int64_t r0,
                        int64_t r1) {
    if (r1 < 0) r1 = n;
    const int64_t rows = r1 - r0;
    if (rows <= 0) return AFMM_OK;
    if (ldk % 8 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)(rows < (1 << 20) ? rows : (1 << 20));
    // Eight-element vector loads need rows aligned to min(16, 8 * size) bytes.
    const size_t es = dtype_size(dt), va = es * 8 < 16 ? es * 8 : 16;
    const int vec = (lds * es) % va == 0 && (reinterpret_cast<uintptr_t>(src) % va) == 0;
    auto* d = static_cast<uint16_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        h16_rows_kernel<DT><<<grid, H16_THREADS, 0, st>>>(src, n, lds, d, ldk, vec, amax,
                                                          status, r0, r1);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
