// Conversions of the exact form on E4M3 digits: the integer Base values x
// (|x| <= 255; X's rows in Case A, Y's columns in Case B) as two digit slices, h = floor(x / 16) in
// [-16, 15] and l = x - 16 h in [0, 15], and the Rep-factors (0 .. 16) as
// the K-major E4M3 operand (Y transposed in Case A, X's rows in Case B);
// every digit and Rep-factor is an integer of
// magnitude at most 16, exact in E4M3, so the tensor pipe's products are
// exact and, with n 16 16 < 2^24, so are its FP32 sums.  Values outside
// those ranges (or not integers) record AFMM_ERR_OVERFLOW_RISK; a negative
// or non-integer Rep-factor AFMM_ERR_NEGATIVE_REP / _NONINTEGER_REP.
// One byte per element and slice; HBM-bound single passes.
#include <cuda_runtime.h>

#include "afmm_common.cuh"
#include "elem.cuh"
#include "fp8_split.cuh"
#include "tc_gemm.cuh"
#include "tile_convert.cuh"

namespace afmm {
namespace {

constexpr int X8_THREADS = 256;
constexpr float kX8BaseMax = 255.f, kX8RepMax = 16.f;

// Four byte-sized indices (each 0 .. 15) looked up in a 16-entry byte table
// held in four words (byte k of word j is entry 4 j + k) with two byte
// permutes: the indices' low three bits select within the table's halves,
// bit 3 picks the half.  The tables, as template arguments: the E4M3 codes
// of 0 .. 15 (E4M3_INT), and those of the high digit of a two's-complement
// byte, whose high nibble k stands for k (k < 8) or k - 16 (E4M3_HI_I8).
template <uint32_t T0, uint32_t T1, uint32_t T2, uint32_t T3>
__device__ __forceinline__ uint32_t lut16_bytes(uint32_t b) {
    const uint32_t packed = b | (b >> 4);                       // nibbles i0 i1 | i2 i3
    const uint32_t sel = __byte_perm(packed, 0u, 0x0020u) & 0x7777u;
    const uint32_t lo = __byte_perm(T0, T1, sel);
    const uint32_t hi = __byte_perm(T2, T3, sel);
    const uint32_t m = ((b >> 3) & 0x01010101u) * 0xFFu;       // indices 8 .. 15
    return (lo & ~m) | (hi & m);
}
#define E4M3_INT 0x44403800u, 0x4E4C4A48u, 0x53525150u, 0x57565554u
#define E4M3_HI_I8 0x44403800u, 0x4E4C4A48u, 0xCACCCED0u, 0xB8C0C4C8u

// Rows of X as the two digit slices dst[(s * n + r) * ldk + c] (zero for
// n <= c < ldk; ldk a multiple of 16), sixteen columns per thread.  int8
// and uint8 values are always integers within |x| <= 255: their digits are
// the nibbles (the high one read as signed for int8), coded by table.
template <int DT>
__global__ void __launch_bounds__(X8_THREADS)
x8_digit_rows_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                     uint8_t* __restrict__ dst, int64_t ldk, int vec, int* status) {
    using T = typename Elem<DT>::T;
    const int64_t c = ((int64_t)blockIdx.x * X8_THREADS + threadIdx.x) * 16;
    if (c >= ldk) return;
    bool bad = false;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        const T* row = static_cast<const T*>(src) + r * lds;
        if constexpr (DT == AFMM_I8 || DT == AFMM_U8) {
            if (vec && c + 16 <= n) {
                // Rows are 8-byte aligned here: two 8-byte loads.
                const uint2 a = *reinterpret_cast<const uint2*>(row + c);
                const uint2 b = *reinterpret_cast<const uint2*>(row + c + 8);
                const uint32_t w[4] = {a.x, a.y, b.x, b.y};
                uint32_t wh[4], wl[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    wl[k] = lut16_bytes<E4M3_INT>(w[k] & 0x0F0F0F0Fu);
                    const uint32_t hn = (w[k] >> 4) & 0x0F0F0F0Fu;
                    if constexpr (DT == AFMM_I8)
                        wh[k] = lut16_bytes<E4M3_HI_I8>(hn);
                    else
                        wh[k] = lut16_bytes<E4M3_INT>(hn);
                }
                *reinterpret_cast<uint4*>(dst + r * ldk + c) =
                    make_uint4(wh[0], wh[1], wh[2], wh[3]);
                *reinterpret_cast<uint4*>(dst + (n + r) * ldk + c) =
                    make_uint4(wl[0], wl[1], wl[2], wl[3]);
                continue;
            }
        }
        float v[16];
        if (vec && c + 16 <= n) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                alignas(16) T e[8];
                load8<DT>(row, c + 8 * q, e);
#pragma unroll
                for (int t = 0; t < 8; ++t) v[8 * q + t] = (float)Elem<DT>::get(e, t);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 16; ++t) v[t] = c + t < n ? (float)Elem<DT>::get(row, c + t) : 0.f;
        }
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int t = 0; t < 16; t += 2) {
            float h[2], l[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float x = v[t + u];
                bad |= !(truncf(x) == x) || fabsf(x) > kX8BaseMax;
                h[u] = floorf(x * 0.0625f);
                l[u] = x - 16.f * h[u];
            }
            const uint32_t qh = e4m3x2_rn(h[0], h[1]), ql = e4m3x2_rn(l[0], l[1]);
            const int word = t >> 2, half = (t >> 1) & 1;
            wh[word] = half ? (wh[word] | (qh << 16)) : qh;
            wl[word] = half ? (wl[word] | (ql << 16)) : ql;
        }
        *reinterpret_cast<uint4*>(dst + r * ldk + c) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4*>(dst + (n + r) * ldk + c) =
            make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
    if (bad) atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
}

// The Rep-factors of Y transposed: dst[c * ldk + r] = Y[r][c] as E4M3, one
// 64 x 64 tile per block through shared memory; four threads per output
// row, sixteen values (one 16-byte store) each.
template <int DT>
__global__ void __launch_bounds__(X8_THREADS)
x8_rep_transpose_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                        uint8_t* __restrict__ dst, int64_t ldk, int vec, int* status) {
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    bool unused = false;
    tile_load_f32<DT>(src, n, lds, r0, c0, 3.0e38f, vec != 0, tile, unused);
    __syncthreads();
    const int cc = threadIdx.x >> 2, qq = threadIdx.x & 3;
    const int64_t c = c0 + cc, r = r0 + 16 * qq;
    if (c >= n || r >= ldk) return;
    int bits = 0;
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
        const float y0 = tile[16 * qq + e][cc], y1 = tile[16 * qq + e + 1][cc];
        bits |= rep_bits(y0) | rep_bits(y1);
        if (y0 > kX8RepMax || y1 > kX8RepMax) bits |= kBadRange;
        const uint32_t q = e4m3x2_rn(y0, y1);
        const int word = e >> 2, half = (e >> 1) & 1;
        w[word] = half ? (w[word] | (q << 16)) : q;
    }
    *reinterpret_cast<uint4*>(dst + c * ldk + r) = make_uint4(w[0], w[1], w[2], w[3]);
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

// The same for one-byte Rep-factors (int8, uint8, E4M3): blocks of 256
// rows x 64 columns kept as bytes in shared memory, each of the 256 codes
// converted and checked once per block (tile_bytes_load and
// tile_bytes_store_lut); 8-byte stores of eight rows.
constexpr int X8_TILE_ROWS = 256;

template <int DT>
__global__ void __launch_bounds__(X8_THREADS)
x8_rep_transpose_u8_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                           uint8_t* __restrict__ dst, int64_t ldk, int vec, int* status) {
    using T = typename Elem<DT>::T;
    static_assert(sizeof(T) == 1, "one-byte elements");
    __shared__ alignas(16) uint8_t tile[X8_TILE_ROWS][64];
    __shared__ uint32_t lut[256];
    {
        const uint8_t code = (uint8_t)threadIdx.x;
        T x;
        __builtin_memcpy(&x, &code, 1);
        const float y = (float)Elem<DT>::get(&x, 0);
        const int b = rep_bits(y) | (y > kX8RepMax ? kBadRange : 0);
        lut[threadIdx.x] = (uint32_t)(e4m3x2_rn(y, 0.f) & 0xFFu) | ((uint32_t)b << 16);
    }
    const int64_t r0 = (int64_t)blockIdx.y * X8_TILE_ROWS, c0 = (int64_t)blockIdx.x * 64;
    tile_bytes_load<X8_TILE_ROWS>(static_cast<const uint8_t*>(src), n, lds, r0, c0, vec != 0,
                                  tile);
    __syncthreads();
    const uint32_t acc = tile_bytes_store_lut<X8_TILE_ROWS, 1>(tile, lut, n, r0, c0, dst, ldk);
    if (acc >> 16) atomicCAS(status, 0, bad_status((int)(acc >> 16)));
}

// Case B: the integer Base values of Y transposed into two digit slices,
// dst[(s * n + c) * ldk + r] from Y[r][c]; and the Rep-factors of X kept
// as E4M3 rows dst[r * ldk + c].  Same ranges and checks as above.
template <int DT>
__global__ void __launch_bounds__(X8_THREADS)
x8_digit_transpose_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                          uint8_t* __restrict__ dst, int64_t ldk, int vec, int* status) {
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    bool unused = false;
    tile_load_f32<DT>(src, n, lds, r0, c0, 3.0e38f, vec != 0, tile, unused);
    __syncthreads();
    const int cc = threadIdx.x >> 2, qq = threadIdx.x & 3;
    const int64_t c = c0 + cc, r = r0 + 16 * qq;
    if (c >= n || r >= ldk) return;
    bool bad = false;
    uint32_t wh[4], wl[4];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
        float h[2], l[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float x = tile[16 * qq + e + u][cc];
            bad |= !(truncf(x) == x) || fabsf(x) > kX8BaseMax;
            h[u] = floorf(x * 0.0625f);
            l[u] = x - 16.f * h[u];
        }
        const uint32_t qh = e4m3x2_rn(h[0], h[1]), ql = e4m3x2_rn(l[0], l[1]);
        const int word = e >> 2, half = (e >> 1) & 1;
        wh[word] = half ? (wh[word] | (qh << 16)) : qh;
        wl[word] = half ? (wl[word] | (ql << 16)) : ql;
    }
    *reinterpret_cast<uint4*>(dst + c * ldk + r) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(dst + (n + c) * ldk + r) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    if (bad) atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
}

template <int DT>
__global__ void __launch_bounds__(X8_THREADS)
x8_rep_rows_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                   uint8_t* __restrict__ dst, int64_t ldk, int* status) {
    const int64_t c = ((int64_t)blockIdx.x * X8_THREADS + threadIdx.x) * 16;
    if (c >= ldk) return;
    int bits = 0;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        uint32_t w[4];
#pragma unroll
        for (int t = 0; t < 16; t += 2) {
            const float y0 = c + t < n ? (float)Elem<DT>::get(src, r * lds + c + t) : 0.f;
            const float y1 = c + t + 1 < n ? (float)Elem<DT>::get(src, r * lds + c + t + 1) : 0.f;
            bits |= rep_bits(y0) | rep_bits(y1);
            if (y0 > kX8RepMax || y1 > kX8RepMax) bits |= kBadRange;
            const uint32_t q = e4m3x2_rn(y0, y1);
            const int word = t >> 2, half = (t >> 1) & 1;
            w[word] = half ? (w[word] | (q << 16)) : q;
        }
        *reinterpret_cast<uint4*>(dst + r * ldk + c) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

}  // namespace

afmm_status tc_x8_digit_transpose(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                                  int64_t ldk, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 16 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const int64_t g = (n + 63) / 64;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    const int vec = rows_aligned16(src, lds, (int64_t)dtype_size(dt));
    auto* d = static_cast<uint8_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        x8_digit_transpose_kernel<DT><<<dim3((unsigned)g, (unsigned)g), X8_THREADS, 0, st>>>(
            src, n, lds, d, ldk, vec, status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status tc_x8_rep_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                           int64_t ldk, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 16 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const dim3 grid((unsigned)((ldk / 16 + X8_THREADS - 1) / X8_THREADS),
                    (unsigned)(n < 65535 ? n : 65535));
    auto* d = static_cast<uint8_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        x8_rep_rows_kernel<DT><<<grid, X8_THREADS, 0, st>>>(src, n, lds, d, ldk, status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status tc_x8_digit_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                             int64_t ldk, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 16 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const dim3 grid((unsigned)((ldk / 16 + X8_THREADS - 1) / X8_THREADS),
                    (unsigned)(n < 65535 ? n : 65535));
    // Eight-element vector loads need rows aligned to min(16, 8 * size) bytes.
    const size_t es = dtype_size(dt), va = es * 8 < 16 ? es * 8 : 16;
    const int vec = (lds * es) % va == 0 && (reinterpret_cast<uintptr_t>(src) % va) == 0;
    auto* d = static_cast<uint8_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        x8_digit_rows_kernel<DT><<<grid, X8_THREADS, 0, st>>>(src, n, lds, d, ldk, vec,
                                                              status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status tc_x8_rep_transpose(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                                int64_t ldk, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (ldk % 16 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0)
        return AFMM_ERR_INVALID_ARG;
    const int64_t g = (n + 63) / 64;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    const int vec = rows_aligned16(src, lds, (int64_t)dtype_size(dt));
    auto* d = static_cast<uint8_t*>(dst);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        if constexpr (sizeof(typename Elem<DT>::T) == 1) {
            // Row blocks of 256 cover ldk (n rounded up to 16).
            const dim3 grid((unsigned)g, (unsigned)((n + X8_TILE_ROWS - 1) / X8_TILE_ROWS));
            x8_rep_transpose_u8_kernel<DT><<<grid, X8_THREADS, 0, st>>>(src, n, lds, d, ldk,
                                                                         vec, status);
        } else {
            x8_rep_transpose_kernel<DT><<<dim3((unsigned)g, (unsigned)g), X8_THREADS, 0, st>>>(
                src, n, lds, d, ldk, vec, status);
        }
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
