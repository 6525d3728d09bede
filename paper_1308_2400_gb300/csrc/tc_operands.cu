// Operand conversions for the tensor-core products (tc_gemm.cu): exact
// widening of Rep-factors to BF16 (or FP16, for the FP16 two-slice form)
// and the hi/mid/lo BF16 split of real values, rows kept (K-major A
// operand) or transposed (K-major B operand).
// HBM-bound single passes.
#include <cuda_bf16.h>

#include "afmm_common.cuh"
#include "bf16_split.cuh"
#include "elem.cuh"
#include "tc_gemm.cuh"
#include "tile_convert.cuh"

namespace afmm {
namespace {

// Value of element i as float plus whether it may be represented exactly
// (for Rep-factors): int32 is range-checked in integer arithmetic so values
// beyond 2^24 cannot slip through a float rounding.
template <int DT>
__device__ __forceinline__ float load_checked(const void* p, int64_t i, float lim,
                                              bool& bad) {
    if constexpr (DT == AFMM_I32) {
        const int32_t v = static_cast<const int32_t*>(p)[i];
        bad |= (float)(v < 0 ? -(int64_t)v : (int64_t)v) > lim;
        return (float)v;
    } else if constexpr (DT == AFMM_F64) {
        const double v = static_cast<const double*>(p)[i];
        bad |= (double)(float)v != v;
        return (float)v;
    } else {
        return (float)Elem<DT>::get(p, i);
    }
}

// Rows kept as rows (K-major A operand): dst[(s*n + r)*ldk + c], eight
// columns per thread (one 16-byte store per slice).  EXACT: one slice that
// must equal the source; otherwise OVERFLOW_RISK is recorded.  rep: the
// source holds Rep-factors, which must be non-negative integers (Sec. 2
// types; NEGATIVE_REP / NONINTEGER_REP otherwise).
template <int DT, int S, bool EXACT>
__global__ void __launch_bounds__(256)
widen_rows_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                  __nv_bfloat16* __restrict__ dst, int64_t ldk, int vec,
                  float lim, int* status, int64_t r0, int64_t r1, int rep) {
    const int64_t c = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 8;
    if (c >= ldk) return;
    int bits = 0;
    for (int64_t r = r0 + blockIdx.y; r < r1; r += gridDim.y) {
        uint32_t w[S][4];
        bool done = false;
        if constexpr (DT != AFMM_F32) {
            if (vec && c + 8 <= n) {
                alignas(16) typename Elem<DT>::T e[8];
                load8<DT>(src, r * lds + c, e);
                bool bad = false;
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    __nv_bfloat16 o0[S], o1[S];
                    const float v0 = value_checked<DT>(e[j], lim, bad);
                    const float v1 = value_checked<DT>(e[j + 1], lim, bad);
                    split_bf16<S>(v0, o0);
                    split_bf16<S>(v1, o1);
                    if (EXACT)
                        bad |= __bfloat162float(o0[0]) != v0 || fabsf(v0) > lim ||
                               __bfloat162float(o1[0]) != v1 || fabsf(v1) > lim;
                    if (rep) bits |= rep_bits(v0) | rep_bits(v1);
#pragma unroll
                    for (int s = 0; s < S; ++s) w[s][j / 2] = pack2(o0[s], o1[s]);
                }
                if (EXACT && bad) bits |= kBadRange;
                done = true;
            }
        }
        if constexpr (DT == AFMM_F32) {
            const float* p = static_cast<const float*>(src) + r * lds + c;
            // Aligned rows: two 16-byte loads; rows that start off a 16-byte
            // boundary (lds % 4 != 0): three aligned loads and a shift.
            const bool al = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
            if ((vec && c + 8 <= n) || (al && c + 12 <= n)) {
                float v[8];
                if (vec) {
                    const float4 a = reinterpret_cast<const float4*>(p)[0];
                    const float4 b = reinterpret_cast<const float4*>(p)[1];
                    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                } else {
                    load8_f32_shifted(p, (int)((reinterpret_cast<uintptr_t>(p) & 15u) >> 2), v);
                }
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    __nv_bfloat16 o0[S], o1[S];
                    split_bf16<S>(v[j], o0);
                    split_bf16<S>(v[j + 1], o1);
                    if (EXACT && (__bfloat162float(o0[0]) != v[j] || fabsf(v[j]) > lim ||
                                  __bfloat162float(o1[0]) != v[j + 1] || fabsf(v[j + 1]) > lim))
                        bits |= kBadRange;
                    if (rep) bits |= rep_bits(v[j]) | rep_bits(v[j + 1]);
#pragma unroll
                    for (int s = 0; s < S; ++s) w[s][j / 2] = pack2(o0[s], o1[s]);
                }
                done = true;
            }
        }
#pragma unroll
        for (int j = 0; j < 8 && !done; j += 2) {
            __nv_bfloat16 o[2][S];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int64_t cc = c + j + t;
                if (cc < n) {
                    bool bad = false;
                    const float v = load_checked<DT>(src, r * lds + cc, lim, bad);
                    split_bf16<S>(v, o[t]);
                    if (EXACT && (bad || __bfloat162float(o[t][0]) != v || fabsf(v) > lim))
                        bits |= kBadRange;
                    if (rep) bits |= rep_bits(v);
                } else {
#pragma unroll
                    for (int s = 0; s < S; ++s) o[t][s] = __float2bfloat16_rn(0.0f);
                }
            }
#pragma unroll
            for (int s = 0; s < S; ++s) w[s][j / 2] = pack2(o[0][s], o[1][s]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
            *reinterpret_cast<uint4*>(dst + ((int64_t)s * n + r) * ldk + c) =
                make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

// Rows become columns (K-major B operand from a row-major K x N matrix):
// dst[(s*n + c)*ldk + r] = slice_s(src[r][c]), one 64 x 64 tile per block
// (tile_transpose_convert: 16-byte loads, FP32 tile in shared memory,
// 128-byte output row segments).  FP64 real factors are rounded to FP32
// first (the FP32 target needs no more).
template <int DT, int S, bool EXACT, bool H16 = false>
__global__ void __launch_bounds__(256)
widen_transpose_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                       __nv_bfloat16* __restrict__ dst, int64_t ldk, float lim,
                       int vec, int* status, int rep) {
    __shared__ float tile[64][65];
    const int bits = tile_transpose_convert<DT, S, EXACT, H16>(
        src, n, lds, (int64_t)blockIdx.y * 64, (int64_t)blockIdx.x * 64, dst, ldk, lim,
        vec != 0, tile, rep != 0);
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

// One-byte sources (E4M3, u8, i8): blocks of 256 rows x 64 columns, the
// tile kept as bytes (tile_bytes_transpose_convert), rows 256 * blockIdx.y
// ...
constexpr int U8_TILE_ROWS = 256;

template <int DT, int S, bool EXACT, bool H16 = false>
__global__ void __launch_bounds__(256)
widen_transpose2_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                        __nv_bfloat16* __restrict__ dst, int64_t ldk, float lim, int vec,
                        int* status, int rep) {
    __shared__ alignas(16) uint8_t tile[U8_TILE_ROWS][64];
    __shared__ uint32_t lut[256];
    const int bits = tile_bytes_transpose_convert<DT, S, EXACT, H16, U8_TILE_ROWS>(
        src, n, lds, (int64_t)blockIdx.y * U8_TILE_ROWS, (int64_t)blockIdx.x * 64, dst, ldk,
        lim, vec != 0, tile, rep != 0, lut);
    if (bits) atomicCAS(status, 0, bad_status(bits));
}

template <int S, bool EXACT>
afmm_status launch_widen_rows(const void* src, int dt, int64_t n, int64_t lds,
                              __nv_bfloat16* dst, int64_t ldk, float lim,
                              int* status, cudaStream_t st, int64_t r0, int64_t r1,
                              bool rep) {
    const int64_t per_row = ldk / 8;
    const int64_t rows = r1 - r0;
    if (rows <= 0) return AFMM_OK;
    const dim3 grid((unsigned)((per_row + 255) / 256),
                    (unsigned)(rows < 65535 ? rows : 65535));
    // Vector loads of 8 elements need rows aligned to min(16, 8 * size) bytes.
    const size_t es = dtype_size(dt), va = es * 8 < 16 ? es * 8 : 16;
    const int vec = (lds * es) % va == 0 && (reinterpret_cast<uintptr_t>(src) % va) == 0;
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        widen_rows_kernel<DT, S, EXACT><<<grid, 256, 0, st>>>(src, n, lds, dst, ldk, vec,
                                                              lim, status, r0, r1, rep ? 1 : 0);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

template <int S, bool EXACT, bool H16 = false>
afmm_status launch_widen_transpose(const void* src, int dt, int64_t n,
                                   int64_t lds, __nv_bfloat16* dst, int64_t ldk,
                                   float lim, int* status, cudaStream_t st, bool rep) {
    const int64_t g = (n + 63) / 64;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    const dim3 grid((unsigned)g, (unsigned)g), block(256);
    const int vec = rows_aligned16(src, lds, (int64_t)dtype_size(dt));
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        if constexpr (sizeof(typename Elem<DT>::T) == 1) {
            // Rows (of the source) in blocks of 256: the row tiles a block
            // holds must cover ldk, the destination's padded K extent (n
            // rounded up to 8, so within the last block).
            const dim3 grid2((unsigned)g,
                             (unsigned)((n + U8_TILE_ROWS - 1) / U8_TILE_ROWS));
            widen_transpose2_kernel<DT, S, EXACT, H16><<<grid2, block, 0, st>>>(
                src, n, lds, dst, ldk, lim, vec, status, rep ? 1 : 0);
        } else {
            widen_transpose_kernel<DT, S, EXACT, H16><<<grid, block, 0, st>>>(
                src, n, lds, dst, ldk, lim, vec, status, rep ? 1 : 0);
        }
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace

afmm_status tc_widen_rows(int slices, bool exact, const void* src, int dt, int64_t n,
                          int64_t lds, void* dst, int64_t ldk, float lim, int* status,
                          cudaStream_t st, int64_t r0, int64_t r1, bool rep) {
    auto* d = static_cast<__nv_bfloat16*>(dst);
    if (r1 < 0) r1 = n;
    if (exact && slices == 1)
        return launch_widen_rows<1, true>(src, dt, n, lds, d, ldk, lim, status, st, r0, r1, rep);
    if (!exact && slices == 3)
        return launch_widen_rows<3, false>(src, dt, n, lds, d, ldk, lim, status, st, r0, r1, rep);
    if (!exact && slices == 2)
        return launch_widen_rows<2, false>(src, dt, n, lds, d, ldk, lim, status, st, r0, r1, rep);
    return AFMM_ERR_INVALID_ARG;
}

afmm_status tc_widen_transpose_h16(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                                   int64_t ldk, float lim, int* status, cudaStream_t st,
                                   bool rep) {
    return launch_widen_transpose<1, true, true>(src, dt, n, lds,
                                                 static_cast<__nv_bfloat16*>(dst), ldk, lim,
                                                 status, st, rep);
}

afmm_status tc_widen_transpose(int slices, bool exact, const void* src, int dt, int64_t n,
                               int64_t lds, void* dst, int64_t ldk, float lim, int* status,
                               cudaStream_t st, bool rep) {
    auto* d = static_cast<__nv_bfloat16*>(dst);
    if (exact && slices == 1)
        return launch_widen_transpose<1, true>(src, dt, n, lds, d, ldk, lim, status, st, rep);
    if (!exact && slices == 3)
        return launch_widen_transpose<3, false>(src, dt, n, lds, d, ldk, lim, status, st, rep);
    if (!exact && slices == 2)
        return launch_widen_transpose<2, false>(src, dt, n, lds, d, ldk, lim, status, st, rep);
    return AFMM_ERR_INVALID_ARG;
}

}  // namespace afmm
