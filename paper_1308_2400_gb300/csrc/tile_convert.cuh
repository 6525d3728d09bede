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

// One-byte sources transposed through shared memory as raw bytes.  A block
// of 256 threads takes rows r0 .. r0+RB-1 and columns c0 .. c0+63 of the
// row-major source into tile[RB][64] (16-byte aligned), each row's four
// 16-byte pieces stored at piece p ^ ((row / 8) mod 4):
//   - loads (tile_bytes_load): thread t copies piece t mod 4 of rows t / 4 +
//     64 i (16-byte cp.async copies, all RB / 64 in flight); the 8 lanes of
//     a store phase write two 64-byte rows, 32 different banks.  Rows past n
//     are zero (they pad K up to ldk); `vec`: 16-byte aligned rows (element
//     loads otherwise, and for a tile cut by the last column);
//   - stores: thread (column cc = t / 4, quarter qq = t mod 4) reads the
//     bytes of rows 32 h + 8 qq + e (e = 0 .. 7) of its column, whose pieces
//     sit at (cc / 16) ^ qq: the four quarters of a warp read four different
//     16-byte slots of rows of one parity, 8 banks, no conflict.  Each run
//     of 8 rows is one store, and the quarters fill a column's output row.
//     Rows at or past ldk (a multiple of 8) are not stored.
template <int RB>
__device__ __forceinline__ void tile_bytes_load(const uint8_t* __restrict__ s, int64_t n,
                                                int64_t lds, int64_t r0, int64_t c0, bool vec,
                                                uint8_t (*tile)[64]) {
    static_assert(RB % 64 == 0, "whole 64-row passes");
    constexpr int P = RB / 64;
    const int lr = threadIdx.x >> 2, piece = threadIdx.x & 3;
    if (vec && c0 + 64 <= n) {
        // Asynchronous 16-byte copies straight into the tile (no registers
        // held while they are in flight); rows past n are zero-filled
        // (source size 0, the address stays in row r0).
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int row = 64 * i + lr;
            const int64_t r = r0 + row;
            const uint8_t* g = s + (r < n ? r : r0) * lds + c0 + 16 * piece;
            const uint32_t d =
                (uint32_t)__cvta_generic_to_shared(&tile[row][16 * (piece ^ ((row >> 3) & 3))]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(g),
                         "r"(r < n ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    } else {
        // Unaligned rows or the last, cut column tile: element loads.
#pragma unroll 1
        for (int i = 0; i < P; ++i) {
            const int row = 64 * i + lr;
            const int64_t r = r0 + row;
            uint8_t* d = &tile[row][16 * (piece ^ ((row >> 3) & 3))];
            for (int t = 0; t < 16; ++t) {
                const int64_t c = c0 + 16 * piece + t;
                d[t] = (r < n && c < n) ? s[r * lds + c] : (uint8_t)0;
            }
        }
    }
}

// The byte of tile row `row` in this thread's column (slot from
// tile_bytes_slot).
__device__ __forceinline__ int tile_bytes_slot(int cc, int qq) {
    return 16 * ((cc >> 4) ^ qq) + (cc & 15);
}

// Store half through a table: a byte has 256 possible values, each
// converted once per block into lut[code] = the OB-byte result (low bits)
// | check bits << 16.  Output row c = c0 + cc gets dst[c * ldk + r] for
// OB-byte elements (OB = 2: 16-byte stores of 8 values; OB = 1: 8-byte
// stores).  Returns the OR of the table entries used (check bits << 16).
template <int RB, int OB>
__device__ __forceinline__ uint32_t tile_bytes_store_lut(const uint8_t (*tile)[64],
                                                         const uint32_t* lut, int64_t n,
                                                         int64_t r0, int64_t c0,
                                                         void* __restrict__ dst, int64_t ldk) {
    static_assert(OB == 1 || OB == 2, "one- or two-byte results");
    const int cc = threadIdx.x >> 2, qq = threadIdx.x & 3;
    const int64_t c = c0 + cc;
    if (c >= n) return 0;
    const int slot = tile_bytes_slot(cc, qq);
    uint32_t acc = 0;
#pragma unroll 2
    for (int h = 0; h < RB / 32; ++h) {
        const int tr = 32 * h + 8 * qq;
        const int64_t r = r0 + tr;
        if (r >= ldk) continue;
        uint32_t e[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            e[u] = lut[tile[tr + u][slot]];
            acc |= e[u];
        }
        if constexpr (OB == 2) {
            *reinterpret_cast<uint4*>(static_cast<uint16_t*>(dst) + c * ldk + r) =
                make_uint4(__byte_perm(e[0], e[1], 0x5410), __byte_perm(e[2], e[3], 0x5410),
                           __byte_perm(e[4], e[5], 0x5410), __byte_perm(e[6], e[7], 0x5410));
        } else {
            // Low bytes of e[0..3] and e[4..7]: pairs, then pairs of pairs.
            const uint32_t lo = __byte_perm(__byte_perm(e[0], e[1], 0x0040),
                                            __byte_perm(e[2], e[3], 0x0040), 0x5410);
            const uint32_t hi = __byte_perm(__byte_perm(e[4], e[5], 0x0040),
                                            __byte_perm(e[6], e[7], 0x0040), 0x5410);
            *reinterpret_cast<uint2*>(static_cast<uint8_t*>(dst) + c * ldk + r) =
                make_uint2(lo, hi);
        }
    }
    return acc;
}

// Rows r0 .. r0+RB-1 and columns c0 .. c0+63 of a source of one-byte
// elements become rows c (K-major) of the destination, dst[(s * n + c) *
// ldk + r] = slice s of src[r][c], with the checks of tile_store_transposed
// (tile_bytes_load, then the stores described there).  S = 1 and EXACT
// (Rep-factors): through the table of tile_bytes_store_lut, built here
// into `lut` (256 entries).
template <int DT, int S, bool EXACT, bool H16, int RB>
__device__ __forceinline__ int tile_bytes_transpose_convert(const void* __restrict__ src,
                                                            int64_t n, int64_t lds, int64_t r0,
                                                            int64_t c0,
                                                            __nv_bfloat16* __restrict__ dst,
                                                            int64_t ldk, float lim, bool vec,
                                                            uint8_t (*tile)[64], bool rep,
                                                            uint32_t* lut) {
    using T = typename Elem<DT>::T;
    static_assert(sizeof(T) == 1, "one-byte elements");
    constexpr bool LUT = S == 1 && EXACT;
    const int tid = threadIdx.x;
    if constexpr (LUT) {
        // 256 threads, one code each.
        const uint8_t code = (uint8_t)tid;
        T x;
        __builtin_memcpy(&x, &code, 1);
        bool bad = false;
        const float v = value_checked<DT>(x, lim, bad);
        uint32_t q[1];
        int b = convert_pair<1, true, H16>(v, 0.f, lim, rep, q);
        if (bad) b |= kBadRange;
        lut[tid] = (q[0] & 0xFFFFu) | ((uint32_t)b << 16);
    }
    tile_bytes_load<RB>(static_cast<const uint8_t*>(src), n, lds, r0, c0, vec, tile);
    __syncthreads();
    if constexpr (LUT)
        return (int)(tile_bytes_store_lut<RB, 2>(tile, lut, n, r0, c0, dst, ldk) >> 16);
    const int cc = tid >> 2, qq = tid & 3;
    const int64_t c = c0 + cc;
    if (c >= n) return 0;
    const int slot = tile_bytes_slot(cc, qq);
    int bits = 0;
    bool bad = false;
#pragma unroll 2
    for (int h = 0; h < RB / 32; ++h) {
        const int tr = 32 * h + 8 * qq;                // first tile row of this run
        const int64_t r = r0 + tr;
        if (r >= ldk) continue;                        // ldk is a multiple of 8
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            T x;
            const uint8_t byte = tile[tr + e][slot];
            __builtin_memcpy(&x, &byte, 1);
            v[e] = value_checked<DT>(x, lim, bad);
        }
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
    return bits | ((EXACT && bad) ? kBadRange : 0);
}

// Whether rows of a dtype-dt source start 16-byte aligned.
__host__ __device__ inline bool rows_aligned16(const void* p, int64_t ld, int64_t es) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (ld * es) % 16 == 0;
}

}  // namespace afmm
