// Operand conversion building blocks shared by the single-product
// conversions (tc_operands.cu) and the grouped ones of a batch
// (batched_kernels.cu): vector loads of any element type and the 64 x 64
// tile that widens or splits a row-major factor into a K-major BF16
// operand.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "bf16_split.cuh"
#include "afmm.h"
#include "elem.cuh"

namespace afmm {

// Eight consecutive elements from element i, by aligned vector loads
// (8 * size bytes: one 8-byte load for one-byte types, one to four 16-byte
// loads otherwise).
template <int DT>
__device__ __forceinline__ void load8(const void* p, int64_t i,
                                      typename Elem<DT>::T (&e)[8]) {
    using T = typename Elem<DT>::T;
    if constexpr (sizeof(T) == 1) {
        const uint2 q = *reinterpret_cast<const uint2*>(static_cast<const T*>(p) + i);
        *reinterpret_cast<uint2*>(e) = q;
    } else {
        const uint4* q = reinterpret_cast<const uint4*>(static_cast<const T*>(p) + i);
#pragma unroll
        for (int k = 0; k < (int)sizeof(T) / 2; ++k) reinterpret_cast<uint4*>(e)[k] = q[k];
    }
}

// p[0 .. 7] for a float pointer p that lies `off` floats (0..3) past a
// 16-byte boundary: three aligned 16-byte loads from p - off and the eight
// wanted values.  The caller keeps p - off .. p - off + 11 inside the
// allocation.
__device__ __forceinline__ void load8_f32_shifted(const float* p, int off, float (&v)[8]) {
    const float4* q = reinterpret_cast<const float4*>(p - off);
    const float4 a = q[0], b = q[1], c = q[2];
    const float f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    switch (off) {
        case 0:
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = f[t];
            break;
        case 1:
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = f[t + 1];
            break;
        case 2:
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = f[t + 2];
            break;
        default:
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = f[t + 3];
            break;
    }
}

// Element value as float; `bad` records an int32 beyond lim (checked in
// integer arithmetic, so values past 2^24 cannot slip through a rounding)
// or an FP64 value that FP32 does not hold.
template <int DT>
__device__ __forceinline__ float value_checked(typename Elem<DT>::T v, float lim, bool& bad) {
    if constexpr (DT == AFMM_I32) {
        bad |= (float)(v < 0 ? -(int64_t)v : (int64_t)v) > lim;
        return (float)v;
    } else if constexpr (DT == AFMM_F64) {
        bad |= (double)(float)v != v;
        return (float)v;
    } else {
        return (float)Elem<DT>::get(&v, 0);
    }
}

// Rows r0 .. r0+63 and columns c0 .. c0+63 of the row-major n x n source
// into tile[r - r0][c - c0] as FP32, zero outside the matrix (value_checked
// flags into `bad`).  16 bytes per thread and pass when `vec` (16-byte
// aligned rows) and the tile is whole in columns, element loads otherwise.
// 256 threads; `tile` is [64][65]; the caller synchronises before reading.
template <int DT>
__device__ __forceinline__ void tile_load_f32(const void* __restrict__ src, int64_t n,
                                              int64_t lds, int64_t r0, int64_t c0,
                                              float lim, bool vec, float (*tile)[65],
                                              bool& bad) {
    using T = typename Elem<DT>::T;
    constexpr int V = 16 / (int)sizeof(T);     // elements per 16-byte load
    constexpr int TPR = 64 / V;                 // threads per tile row
    constexpr int RPP = 256 / TPR;              // tile rows per pass
    constexpr int P = 64 / RPP;                 // passes
    const int tid = threadIdx.x;
    const int lc = (tid % TPR) * V, lr = tid / TPR;
    const T* s = static_cast<const T*>(src);
    if (vec && c0 + 64 <= n) {
        uint4 q[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int64_t r = r0 + lr + RPP * p;
            q[p] = r < n ? *reinterpret_cast<const uint4*>(s + r * lds + c0 + lc)
                         : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const T* e = reinterpret_cast<const T*>(&q[p]);
#pragma unroll
            for (int t = 0; t < V; ++t) tile[lr + RPP * p][lc + t] = value_checked<DT>(e[t], lim, bad);
        }
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int64_t r = r0 + lr + RPP * p;
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int64_t c = c0 + lc + t;
                tile[lr + RPP * p][lc + t] =
                    (r < n && c < n) ? value_checked<DT>(s[r * lds + c], lim, bad) : 0.f;
            }
        }
    }
}

// Check bits of a converted value: kBadRange (not exact in the operand type
// or beyond its limit), and for Rep-factors (Sec. 2 types: non-negative
// integers) kBadNegative and kBadNonInteger (NaN and infinities included).
constexpr int kBadRange = 1, kBadNegative = 2, kBadNonInteger = 4;

__device__ __forceinline__ int rep_bits(float v) {
    return (v < 0.f ? kBadNegative : 0) | ((!isfinite(v) || truncf(v) != v) ? kBadNonInteger : 0);
}

// The status code of a set of check bits (0 when none is set): a negative
// Rep-factor first, then a non-integer one, then a range error.
__device__ __forceinline__ int bad_status(int bits) {
    return (bits & kBadNegative) ? (int)AFMM_ERR_NEGATIVE_REP
           : (bits & kBadNonInteger) ? (int)AFMM_ERR_NONINTEGER_REP
           : bits ? (int)AFMM_ERR_OVERFLOW_RISK : 0;
}

// Two values as S BF16 slices (or, H16, one FP16 value each, S = 1) packed
// into w[sl]; the check bits as in tile_store_transposed.
template <int S, bool EXACT, bool H16>
__device__ __forceinline__ int convert_pair(float v0, float v1, float lim, bool rep,
                                            uint32_t (&w)[S]) {
    int bits = 0;
    if constexpr (H16) {
        static_assert(S == 1 && EXACT, "FP16 output: exact values, one slice");
        const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
        if (__half2float(h0) != v0 || __half2float(h1) != v1 || fabsf(v0) > lim ||
            fabsf(v1) > lim)
            bits |= kBadRange;
        w[0] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
    } else {
        __nv_bfloat16 o0[S], o1[S];
        split_bf16<S>(v0, o0);
        split_bf16<S>(v1, o1);
        if (EXACT && (__bfloat162float(o0[0]) != v0 || __bfloat162float(o1[0]) != v1 ||
                      fabsf(v0) > lim || fabsf(v1) > lim))
            bits |= kBadRange;
#pragma unroll
        for (int sl = 0; sl < S; ++sl) w[sl] = pack2(o0[sl], o1[sl]);
    }
    if (rep) bits |= rep_bits(v0) | rep_bits(v1);
    return bits;
}

// The store half of tile_transpose_convert: tile[r - r0][c - c0] (FP32,
// filled and synchronised by the caller) becomes rows c (K-major) of the
// destination, dst[(s * n + c) * ldk + r] = slice s of the value, for S
// BF16 slices; four threads write one 128-byte segment of an output row per
// slice.  Returns the check bits of the values this thread converted:
// kBadRange (EXACT: not exact in BF16 or |v| > lim) and, with `rep`, the
// Rep-factor checks (rep_bits).  H16: FP16 instead of BF16 (S = 1, EXACT).
// 256 threads; `tile` is [64][65].
template <int S, bool EXACT, bool H16 = false>
__device__ __forceinline__ int tile_store_transposed(const float (*tile)[65], int64_t n,
                                                     int64_t r0, int64_t c0,
                                                     __nv_bfloat16* __restrict__ dst,
                                                     int64_t ldk, float lim, bool rep) {
    const int tid = threadIdx.x;
    int bits = 0;
    const int cc = tid >> 2, qq = tid & 3;
    const int64_t c = c0 + cc, r = r0 + 16 * qq;
    if (c < n && r < ldk) {
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = tile[16 * qq + e][cc];
        const int cnt = (int)((ldk - r) < 16 ? (ldk - r) : 16);   // 8 or 16
        uint32_t w[S][8];
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
            uint32_t q[S];
            bits |= convert_pair<S, EXACT, H16>(v[e], v[e + 1], lim, rep, q);
#pragma unroll
            for (int sl = 0; sl < S; ++sl) w[sl][e / 2] = q[sl];
        }
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            __nv_bfloat16* o = dst + ((int64_t)sl * n + c) * ldk + r;
            *reinterpret_cast<uint4*>(o) = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
            if (cnt == 16)
                *reinterpret_cast<uint4*>(o + 8) =
                    make_uint4(w[sl][4], w[sl][5], w[sl][6], w[sl][7]);
        }
    }
    return bits;
}

// Rows r0 .. r0+63 and columns c0 .. c0+63 of the row-major n x n source
// become rows c (K-major) of the destination: dst[(s * n + c) * ldk + r] =
// slice s of src[r][c], for S BF16 slices.  S = 1 and EXACT: the value must
// be exact in BF16 and |v| <= lim, else kBadRange is returned; `rep` adds
// the Rep-factor checks (rep_bits) of every value in the matrix.
// Loads: tile_load_f32; the tile goes through shared memory as FP32;
// stores: tile_store_transposed.  256 threads; `tile` is [64][65].
template <int DT, int S, bool EXACT, bool H16 = false>
__device__ __forceinline__ int tile_transpose_convert(const void* __restrict__ src,
                                                      int64_t n, int64_t lds, int64_t r0,
                                                      int64_t c0,
                                                      __nv_bfloat16* __restrict__ dst,
                                                      int64_t ldk, float lim, bool vec,
                                                      float (*tile)[65], bool rep = false) {
    bool bad = false;
    tile_load_f32<DT>(src, n, lds, r0, c0, lim, vec, tile, bad);
    __syncthreads();
    const int bits = tile_store_transposed<S, EXACT, H16>(tile, n, r0, c0, dst, ldk, lim, rep);
    return bits | ((EXACT && bad) ? kBadRange : 0);
}

// Store half for one-byte sources, with a bank-conflict-free read of the
// tile (row stride 65 floats: element (r, c) sits in bank (r + c) mod 32):
// thread (column cc, quarter qq) takes rows 8 qq + e and 32 + 8 qq + e
// (e = 0 .. 7), so the 32 lanes of a warp (8 columns x 4 quarters) read 32
// different banks; each run of 8 rows becomes one 16-byte store per slice,
// and the four quarters of a column still fill its 128-byte output row.
template <int S, bool EXACT, bool H16 = false>
__device__ __forceinline__ int tile_store_transposed_il(const float (*tile)[65], int64_t n,
                                                        int64_t r0, int64_t c0,
                                                        __nv_bfloat16* __restrict__ dst,
                                                        int64_t ldk, float lim, bool rep) {
    const int tid = threadIdx.x;
    const int cc = tid >> 2, qq = tid & 3;
    const int64_t c = c0 + cc;
    int bits = 0;
    if (c >= n) return 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int tr = 32 * half + 8 * qq;             // first tile row of this run
        const int64_t r = r0 + tr;
        if (r >= ldk) continue;                        // ldk is a multiple of 8
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = tile[tr + e][cc];
        uint32_t w[S][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint32_t q[S];
            bits |= convert_pair<S, EXACT, H16>(v[e], v[e + 1], lim, rep, q);
#pragma unroll
            for (int sl = 0; sl < S; ++sl) w[sl][e / 2] = q[sl];
        }
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
            *reinterpret_cast<uint4*>(dst + ((int64_t)sl * n + c) * ldk + r) =
                make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
    }
    return bits;
}

// Two vertically adjacent 64 x 64 tiles (rows r0 .. r0+127) of a source of
// one-byte elements, both loaded before either is converted (two 16-byte
// loads in flight per thread).  Load mapping, per tile: warps 2b and 2b+1
// cover tile rows 16b .. 16b+15; lane l takes the 16 columns q = l / 8 of
// row 16b + (l mod 8) + 8 * ((q / 2) xor (warp mod 2)), so the 32 lanes of a
// warp write 32 different banks of the stride-65 tile (the rows and
// quarters they take differ by 0, 8, 16, 24 in bank).  Store half:
// tile_store_transposed_il.  `vec` as in tile_load_f32; `tile` is
// [2][64][65].  Returns the check bits of both tiles.
template <int DT, int S, bool EXACT, bool H16 = false>
__device__ __forceinline__ int tile2_transpose_convert_u8(const void* __restrict__ src,
                                                          int64_t n, int64_t lds, int64_t r0,
                                                          int64_t c0,
                                                          __nv_bfloat16* __restrict__ dst,
                                                          int64_t ldk, float lim, bool vec,
                                                          float (*tile)[64][65], bool rep) {
    using T = typename Elem<DT>::T;
    static_assert(sizeof(T) == 1, "one-byte elements");
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int q = l >> 3;
    const int lr = 16 * (warp >> 1) + (l & 7) + 8 * ((q >> 1) ^ (warp & 1));
    const int lc = 16 * q;
    const T* s = static_cast<const T*>(src);
    bool bad = false;
    if (vec && c0 + 64 <= n) {
        uint4 v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = r0 + 64 * h + lr;
            v[h] = r < n ? *reinterpret_cast<const uint4*>(s + r * lds + c0 + lc)
                         : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T* e = reinterpret_cast<const T*>(&v[h]);
#pragma unroll
            for (int t = 0; t < 16; ++t) tile[h][lr][lc + t] = value_checked<DT>(e[t], lim, bad);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = r0 + 64 * h + lr;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int64_t c = c0 + lc + t;
                tile[h][lr][lc + t] =
                    (r < n && c < n) ? value_checked<DT>(s[r * lds + c], lim, bad) : 0.f;
            }
        }
    }
    __syncthreads();
    int bits = (EXACT && bad) ? kBadRange : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (r0 + 64 * h < ldk)
            bits |= tile_store_transposed_il<S, EXACT, H16>(tile[h], n, r0 + 64 * h, c0, dst,
                                                            ldk, lim, rep);
    return bits;
}

// Whether rows of a dtype-dt source start 16-byte aligned.
__host__ __device__ inline bool rows_aligned16(const void* p, int64_t ld, int64_t es) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (ld * es) % 16 == 0;
}

}  // namespace afmm
