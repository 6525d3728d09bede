// K1, dense regime: the plain FP32 CUDA-core product C = A * B for Base
// factors with few zeros.  There the zero-skip of simt_gemm.cu saves
// nothing (a 4-row group of Base values is all zero with probability
// (1 - d)^4, under 1% at d = 0.7), and its 4 x 8 outputs per thread leave
// that kernel bound by instruction issue.
//
// Each term is still one exact product added once (Sec. 2.1: the result is
// X * Y).  Sums are K-blocked: a fresh partial per 128-wide k block, its
// first term a plain product, then added to the running sum, so an entry's
// rounding error stays within (min(n, 128) + ceil(n / 128)) u sum|x y| to
// first order.
//
// Design (every choice measured at n = 8192 on GB300):
// * A reaches the kernel k-major (A^T, written by the converting transpose
//   below, one extra pass over X), so both operand tiles are plain cp.async
//   copies of 16 k-rows x 128 columns; staging A through registers and
//   transposing it in shared memory cost 15% of the kernel.
// * 128 x 128 output tiles, 256 threads, 8 x 8 outputs per thread: each
//   warp owns a 32 x 64 sub-tile; lane (lm, ln) = (lane / 8, lane % 8) holds
//   rows 4 lm .. 4 lm + 3 and 16 + 4 lm .. of it and columns 4 ln .. and
//   32 + 4 ln .., read per k with four 16-byte shared-memory loads for 64
//   FMAs, the next k's fragments loaded while the current k's FMAs issue.
// * The running sums live in shared memory (64 KiB per CTA, each thread
//   its own conflict-free column), touched once per 128 k, so the partials
//   and fragments fit 128 registers and two CTAs (16 warps) share an SM.
// * Three cp.async stages of 16 k.
#include <cstdint>

#include "afmm_common.cuh"
#include "elem.cuh"

namespace afmm {

namespace {

constexpr int DM = 128, DN = 128, DK = 16;
constexpr int DTHREADS = 256;
constexpr int DSTAGES = 3;
constexpr int KBLOCK = 128;                 // k per FP32 partial sum
constexpr int TILE_F = DK * DM;             // floats per operand tile
constexpr int ACC_F = 64 * DTHREADS;        // running sums, floats
constexpr int DSMEM = (2 * DSTAGES * TILE_F + ACC_F) * 4;   // 112 KiB
constexpr int RO = 16, CO = 32;             // second row / column group

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)),
                 "l"(src));
}
// 4-byte copy; when !ok nothing is read and the destination is zeroed.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(ok ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Rows k0 .. k0+15 (k < K), columns c0 .. c0+127 (c < C) of a row-major
// matrix into S[k][c]; zero outside.  512 chunks of 4 floats, two per thread.
__device__ __forceinline__ void load_tile(float* S, const float* __restrict__ G, int64_t ld,
                                          int64_t K, int64_t C, int64_t k0, int64_t c0,
                                          bool vec) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = threadIdx.x + h * DTHREADS;
        const int k = q >> 5, cc = (q & 31) * 4;
        const int64_t gk = k0 + k, gc = c0 + cc;
        float* dst = S + k * DN + cc;
        if (vec && gk < K && gc + 3 < C) {
            cp_async16(dst, G + gk * ld + gc);
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool ok = gk < K && gc + t < C;
                cp_async4(dst + t, ok ? (const void*)(G + gk * ld + gc + t) : (const void*)G, ok);
            }
        }
    }
}

// The same tile when it lies inside the matrix and 16-byte copies are
// allowed: no predicates.
__device__ __forceinline__ void load_tile_full(float* S, const float* __restrict__ G,
                                               int64_t ld, int64_t k0, int64_t c0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = threadIdx.x + h * DTHREADS;
        const int k = q >> 5, cc = (q & 31) * 4;
        cp_async16(S + k * DN + cc, G + (k0 + k) * ld + c0 + cc);
    }
}

// The 8 A and 8 B values of one k for this thread.
__device__ __forceinline__ void fragments(float (&a)[8], float (&b)[8], const float* as,
                                          const float* bs, int k, int r0, int c0) {
    const float4 a0 = *reinterpret_cast<const float4*>(as + k * DM + r0);
    const float4 a1 = *reinterpret_cast<const float4*>(as + k * DM + RO + r0);
    const float4 b0 = *reinterpret_cast<const float4*>(bs + k * DN + c0);
    const float4 b1 = *reinterpret_cast<const float4*>(bs + k * DN + CO + c0);
    a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
    a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
    b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
    b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
}

// p += a b^T over the 8 x 8 block (FIRST: p = a b^T), row by row with the
// column order reversed on odd rows, so consecutive FMAs share an operand
// (measured 8% faster than plain row order).
template <bool FIRST>
__device__ __forceinline__ void outer8(float (&p)[8][8], const float (&a)[8], const float (&b)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int j = (i & 1) ? 7 - v : v;
            p[i][j] = FIRST ? a[i] * b[j] : fmaf(a[i], b[j], p[i][j]);
        }
}

// The K loop of one 128 x 128 tile, its running sums left in Acc (returns
// false when K is empty).  FULL: the tile lies inside M and N, K is a
// multiple of 16 and B allows 16-byte copies, so no load is predicated.
template <bool FULL>
__device__ __forceinline__ bool dense_tile(const float* __restrict__ AT, int64_t ldat,
                                           const float* __restrict__ B, int64_t ldb,
                                           int64_t M, int64_t N, int64_t K, int64_t m0,
                                           int64_t n0, bool vec_b, float* dsm) {
    float* As = dsm;                                // [DSTAGES][DK][DM]
    float* Bs = dsm + DSTAGES * TILE_F;             // [DSTAGES][DK][DN]
    float* Acc = dsm + 2 * DSTAGES * TILE_F;        // [64][DTHREADS]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = (w & 3) * 32 + (lane >> 3) * 4;
    const int c0 = (w >> 2) * 64 + (lane & 7) * 4;
    const auto load_stage = [&](int st, int64_t kb) {
        if (FULL) {
            load_tile_full(As + st * TILE_F, AT, ldat, kb * DK, m0);
            load_tile_full(Bs + st * TILE_F, B, ldb, kb * DK, n0);
        } else {
            load_tile(As + st * TILE_F, AT, ldat, K, M, kb * DK, m0, true);
            load_tile(Bs + st * TILE_F, B, ldb, K, N, kb * DK, n0, vec_b);
        }
    };

    float part[8][8];
    bool summed = false;
    const int64_t nk = (K + DK - 1) / DK;
#pragma unroll
    for (int q = 0; q < DSTAGES - 1; ++q) {
        if (q < nk) load_stage(q, q);
        cp_async_commit();
    }
    int s = 0, sn = DSTAGES - 1;                    // stage read / stage refilled
    int kbi = 0;                                    // k block within the sum block
    for (int64_t t = 0; t < nk; ++t) {
        cp_async_wait<DSTAGES - 2>();
        __syncthreads();                            // stage s landed; stage sn free
        if (t + DSTAGES - 1 < nk) load_stage(sn, t + DSTAGES - 1);
        cp_async_commit();
        const float* as = As + s * TILE_F;
        const float* bs = Bs + s * TILE_F;
        const bool fresh = kbi == 0;
        float a[2][8], b[2][8];
        fragments(a[0], b[0], as, bs, 0, r0, c0);
#pragma unroll
        for (int k = 0; k < DK; ++k) {
            const int c = k & 1;
            if (k + 1 < DK) fragments(a[c ^ 1], b[c ^ 1], as, bs, k + 1, r0, c0);
            if (k == 0 && fresh) outer8<true>(part, a[c], b[c]);
            else outer8<false>(part, a[c], b[c]);
        }
        if (++kbi == KBLOCK / DK || t + 1 == nk) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float* q = Acc + (i * 8 + j) * DTHREADS + threadIdx.x;
                    *q = summed ? *q + part[i][j] : part[i][j];
                }
            summed = true;
            kbi = 0;
        }
        s = s + 1 == DSTAGES ? 0 : s + 1;
        sn = sn + 1 == DSTAGES ? 0 : sn + 1;
    }
    return summed;
}

// C (M x N) = A (M x K) * B (K x N); AT = A^T (K x M, row stride ldat, a
// multiple of 4 floats, 16-byte aligned), B row-major (vec_b: 16-byte
// copies allowed), C row-major (vec_c: 16-byte stores allowed).
__global__ void __launch_bounds__(DTHREADS, 2)
simt_dense_kernel(const float* __restrict__ AT, int64_t ldat, const float* __restrict__ B,
                  int64_t ldb, float* __restrict__ C, int64_t ldc, int64_t M, int64_t N,
                  int64_t K, int vec_b, int vec_c) {
    extern __shared__ __align__(16) float dsm[];
    const float* Acc = dsm + 2 * DSTAGES * TILE_F;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = (w & 3) * 32 + (lane >> 3) * 4;
    const int c0 = (w >> 2) * 64 + (lane & 7) * 4;
    const int64_t m0 = (int64_t)blockIdx.y * DM, n0 = (int64_t)blockIdx.x * DN;
    const bool full = vec_b && m0 + DM <= M && n0 + DN <= N && K % DK == 0;
    const bool summed = full ? dense_tile<true>(AT, ldat, B, ldb, M, N, K, m0, n0, true, dsm)
                             : dense_tile<false>(AT, ldat, B, ldb, M, N, K, m0, n0,
                                                 vec_b != 0, dsm);

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gm = m0 + r0 + (i < 4 ? i : RO + i - 4);
        if (gm >= M) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gn = n0 + c0 + h * CO;
            float v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                v[c] = summed ? Acc[(i * 8 + 4 * h + c) * DTHREADS + threadIdx.x] : 0.f;
            float* dst = C + gm * ldc + gn;
            if (vec_c && gn + 3 < N) {
                *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (gn + c < N) dst[c] = v[c];
            }
        }
    }
}

// dst (ldd floats per row) = src^T converted to FP32: dst[c][r] = src[r][c]
// for r, c < n.  32 x 32 tiles through shared memory, both sides coalesced.
template <int DT>
__global__ void to_f32_transposed_kernel(const void* __restrict__ src, int64_t n, int64_t lds,
                                         float* __restrict__ dst, int64_t ldd) {
    __shared__ float tile[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t gr = by + r, gc = bx + threadIdx.x;
        tile[r][threadIdx.x] = (gr < n && gc < n) ? (float)Elem<DT>::get(src, gr * lds + gc) : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t gr = bx + r, gc = by + threadIdx.x;
        if (gr < n && gc < n) dst[gr * ldd + gc] = tile[threadIdx.x][r];
    }
}

}  // namespace

afmm_status launch_to_f32_transposed(const void* src, int dtype, int64_t n, int64_t lds,
                                     float* dst, int64_t ldd, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    const int64_t g = (n + 31) / 32;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        to_f32_transposed_kernel<DT><<<dim3((unsigned)g, (unsigned)g), dim3(32, 8), 0, st>>>(
            src, n, lds, dst, ldd);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_simt_f32_dense(const float* AT, int64_t ldat, const float* B, int64_t ldb,
                                  float* C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                                  cudaStream_t st) {
    if (M <= 0 || N <= 0) return AFMM_OK;
    const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (ldat % 4 != 0 || !al(AT)) return AFMM_ERR_INVALID_ARG;
    const int vec_b = (ldb % 4 == 0) && al(B);
    const int vec_c = (ldc % 4 == 0) && al(C);
    const int64_t gx = (N + DN - 1) / DN, gy = (M + DM - 1) / DM;
    if (gy > 65535) return AFMM_ERR_UNSUPPORTED;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(simt_dense_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, DSMEM));
    main_kernel_begin(st);
    simt_dense_kernel<<<dim3((unsigned)gx, (unsigned)gy), DTHREADS, DSMEM, st>>>(
        AT, ldat, B, ldb, C, ldc, M, N, K, vec_b, vec_c);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, (int)(gx * gy));
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
