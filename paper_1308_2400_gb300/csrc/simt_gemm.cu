// K1: CUDA-core AFMM product with zero-skipping.
//
// The paper's loop (Sec. 2, Case-A) reads Base = X[i,k] and skips the whole
// J loop when it is zero.  Here one warp owns 4 rows of a 64 x 256 output
// tile and all 256 columns, so the Base values X[i..i+3, k] it needs are the
// same for every lane: the zero test is warp-uniform and a k whose 4 Base
// values are all zero is skipped by the whole warp at no divergence cost.
// The term Rep * Base is formed with one FMA (FP32) or one 4-way int8 dot
// product (exact integers) instead of Rep additions: the same value, formed
// exactly before the accumulation rounds (Sec. 2.1: the result is X * Y).
//
// Layout: A (M x K) and B (K x N) row-major in global memory, staged by
// cp.async into shared memory (A as [64][32], B as [32][256] elements of
// 4 bytes, two stages).  Each of the 16 warps' threads accumulates 4 rows x
// 8 columns; FP32 sums are K-blocked (a fresh partial per 32-wide k tile,
// added to the running sum afterwards) to keep the rounding error of long
// sums low.  The running sums and the partials of 4 rows fit 128 registers,
// so the CTA runs 16 warps.
#include <cstdint>

#include "afmm_common.cuh"

namespace afmm {

namespace {

constexpr int BM = 64, BN = 256, BK = 32;
constexpr int RW = 4;                       // rows of the tile per warp
constexpr int THREADS = BM / RW * 32;       // 16 warps
constexpr int SMEM_BYTES = 2 * (BM * BK + BK * BN) * 4;
constexpr int64_t kMaskMaxKTiles = 16384;   // live flags in shared memory (16 KB)

struct OpF32 {
    using Elt = float;
    using Acc = float;
    static constexpr bool kBlocked = true;
    static __device__ __forceinline__ Acc mac(Elt a, Elt b, Acc c) {
        return fmaf(a, b, c);
    }
    static __device__ __forceinline__ bool nz(Elt a) { return a != 0.0f; }
};

// One element = 4 consecutive k of int8; mac = 4 products + 1 add, exact.
struct OpDp4a {
    using Elt = int32_t;
    using Acc = int32_t;
    static constexpr bool kBlocked = false;
    static __device__ __forceinline__ Acc mac(Elt a, Elt b, Acc c) {
        return __dp4a(a, b, c);
    }
    static __device__ __forceinline__ bool nz(Elt a) { return a != 0; }
};

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
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::);
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename Elt>
__device__ __forceinline__ void load_tiles(Elt* As, Elt* Bs, const Elt* A,
                                           int64_t lda, const Elt* B,
                                           int64_t ldb, int64_t M, int64_t N,
                                           int64_t K, int64_t m0, int64_t n0,
                                           int64_t k0, bool vec) {
    // A tile: 64 rows x 32 elements = 512 chunks of 4.
    for (int c = threadIdx.x; c < BM * BK / 4; c += THREADS) {
        const int m = c / (BK / 4), kc = (c % (BK / 4)) * 4;
        const int64_t gm = m0 + m, gk = k0 + kc;
        Elt* dst = As + m * BK + kc;
        if (vec && gm < M && gk + 3 < K) {
            cp_async16(dst, A + gm * lda + gk);
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool ok = gm < M && gk + t < K;
                cp_async4(dst + t, ok ? (const void*)(A + gm * lda + gk + t)
                                      : (const void*)A, ok);
            }
        }
    }
    // B tile: 32 rows x 256 elements = 2048 chunks of 4.
    for (int c = threadIdx.x; c < BK * BN / 4; c += THREADS) {
        const int k = c / (BN / 4), nc = (c % (BN / 4)) * 4;
        const int64_t gk = k0 + k, gn = n0 + nc;
        Elt* dst = Bs + k * BN + nc;
        if (vec && gk < K && gn + 3 < N) {
            cp_async16(dst, B + gk * ldb + gn);
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool ok = gk < K && gn + t < N;
                cp_async4(dst + t, ok ? (const void*)(B + gk * ldb + gn + t)
                                      : (const void*)B, ok);
            }
        }
    }
}

template <typename V, typename E>
__device__ __forceinline__ E comp(const V& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// One 64 x 256 output tile C[m0.., n0..] of C = A * B.  With LIVE, `live`
// (shared memory, one byte per 32-wide k tile) flags the k tiles to load
// and multiply; the others would add exact zeros.
template <class Op, bool LIVE = false>
__device__ __forceinline__ void simt_tile(const typename Op::Elt* __restrict__ A,
                                          int64_t lda,
                                          const typename Op::Elt* __restrict__ B,
                                          int64_t ldb, typename Op::Acc* __restrict__ C,
                                          int64_t ldc, int64_t M, int64_t N, int64_t K,
                                          int vec, int64_t m0, int64_t n0,
                                          unsigned char* smem_raw, bool accumulate = false,
                                          const uint8_t* live = nullptr) {
    using Elt = typename Op::Elt;
    using Acc = typename Op::Acc;
    using V4 = typename std::conditional<std::is_same<Elt, float>::value,
                                         float4, int4>::type;
    using A4 = typename std::conditional<std::is_same<Acc, float>::value,
                                         float4, int4>::type;
    Elt* As = reinterpret_cast<Elt*>(smem_raw);          // [2][BM][BK]
    Elt* Bs = As + 2 * BM * BK;                          // [2][BK][BN]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = warp * RW;

    Acc acc[RW][8];
    Acc part[RW][8];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[r][c] = Acc(0);
            part[r][c] = Acc(0);
        }

    const int64_t ntiles = (K + BK - 1) / BK;
    // One k tile from stage s: the Base zero test, the products, the flush.
    const auto tile_product = [&](int s) {
            const Elt* as = As + s * BM * BK + row0 * BK;
            const Elt* bs = Bs + s * BK * BN;

            // Which k of this tile have a non-zero Base in the warp's rows.
            bool any = false;
#pragma unroll
            for (int r = 0; r < RW; ++r) any |= Op::nz(as[r * BK + lane]);
            const unsigned mask = __ballot_sync(0xffffffffu, any);

            if (__popc(mask) >= 24) {
                // Nearly dense: run all 32 k; zero Base values add exact zeros.
#pragma unroll
                for (int kq = 0; kq < BK / 4; ++kq) {
                    V4 y[4][2];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const Elt* row = bs + (kq * 4 + kk) * BN;
                        y[kk][0] = *reinterpret_cast<const V4*>(row + lane * 4);
                        y[kk][1] = *reinterpret_cast<const V4*>(row + 128 + lane * 4);
                    }
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        const V4 xv = *reinterpret_cast<const V4*>(as + r * BK + kq * 4);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const Elt x = comp<V4, Elt>(xv, kk);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                part[r][c] = Op::mac(x, comp<V4, Elt>(y[kk][0], c), part[r][c]);
                                part[r][4 + c] = Op::mac(x, comp<V4, Elt>(y[kk][1], c), part[r][4 + c]);
                            }
                        }
                    }
                }
            } else {
                // Sparse: visit only the k whose Base group is non-zero.
                unsigned msk = mask;
                while (msk) {
                    const int k = __ffs(msk) - 1;
                    msk &= msk - 1;
                    const Elt* row = bs + k * BN;
                    const V4 y0 = *reinterpret_cast<const V4*>(row + lane * 4);
                    const V4 y1 = *reinterpret_cast<const V4*>(row + 128 + lane * 4);
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        const Elt x = as[r * BK + k];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            part[r][c] = Op::mac(x, comp<V4, Elt>(y0, c), part[r][c]);
                            part[r][4 + c] = Op::mac(x, comp<V4, Elt>(y1, c), part[r][4 + c]);
                        }
                    }
                }
            }
            if (Op::kBlocked) {
#pragma unroll
                for (int r = 0; r < RW; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        acc[r][c] += part[r][c];
                        part[r][c] = Acc(0);
                    }
            }
    };
    if constexpr (!LIVE) {
        if (ntiles > 0) {
            load_tiles<Elt>(As, Bs, A, lda, B, ldb, M, N, K, m0, n0, 0, vec != 0);
            cp_async_commit();
        }
        for (int64_t t = 0; t < ntiles; ++t) {
            const int s = (int)(t & 1);
            if (t + 1 < ntiles) {
                load_tiles<Elt>(As + (s ^ 1) * BM * BK, Bs + (s ^ 1) * BK * BN, A,
                                lda, B, ldb, M, N, K, m0, n0, (t + 1) * BK,
                                vec != 0);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            tile_product(s);
            __syncthreads();
        }
    } else {
        // Only the live k tiles, in increasing k.
        const auto next_live = [&](int64_t t) -> int64_t {
            while (t < ntiles && !live[t]) ++t;
            return t;
        };
        int64_t t = next_live(0);
        if (t < ntiles) {
            load_tiles<Elt>(As, Bs, A, lda, B, ldb, M, N, K, m0, n0, t * BK, vec != 0);
            cp_async_commit();
        }
        for (int s = 0; t < ntiles; s ^= 1) {
            const int64_t tn = next_live(t + 1);
            if (tn < ntiles) {
                load_tiles<Elt>(As + (s ^ 1) * BM * BK, Bs + (s ^ 1) * BK * BN, A,
                                lda, B, ldb, M, N, K, m0, n0, tn * BK,
                                vec != 0);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            tile_product(s);
            __syncthreads();
            t = tn;
        }
    }
    if (!Op::kBlocked) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = part[r][c];
    }

    // Epilogue: rows m0+row0+r, columns n0 + lane*4 (+128).  With
    // `accumulate` (integer K splits) the sums are added into C atomically,
    // which is exact in any order.
    if constexpr (std::is_same<Acc, int32_t>::value) {
        if (accumulate) {
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int64_t gm = m0 + row0 + r;
                if (gm >= M) break;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t gn = n0 + h * 128 + lane * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (gn + c < N) atomicAdd(C + gm * ldc + gn + c, acc[r][4 * h + c]);
                }
            }
            return;
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int64_t gm = m0 + row0 + r;
        if (gm >= M) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gn = n0 + h * 128 + lane * 4;
            Acc* dst = C + gm * ldc + gn;
            if (vec && gn + 3 < N) {
                A4 v;
                v.x = acc[r][4 * h + 0];
                v.y = acc[r][4 * h + 1];
                v.z = acc[r][4 * h + 2];
                v.w = acc[r][4 * h + 3];
                *reinterpret_cast<A4*>(dst) = v;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (gn + c < N) dst[c] = acc[r][4 * h + c];
            }
        }
    }
}

// xm, ym (optional, one K split only): the K0 tile masks of A (BM x BK
// tiles, row-major over [M / BM][nkb]) and of B (BK x BN tiles, [nkb][N /
// BN]).  A k tile is live for a CTA when both its A and its B tile hold a
// non-zero.  With masks this kernel runs only the CTAs whose k tiles are
// all live (simt_masked_kernel runs the others), and adds their k tiles to
// *ktiles.
template <class Op>
__global__ void __launch_bounds__(THREADS, 1)
simt_gemm_kernel(const typename Op::Elt* __restrict__ A, int64_t lda,
                 const typename Op::Elt* __restrict__ B, int64_t ldb,
                 typename Op::Acc* __restrict__ C, int64_t ldc, int64_t M,
                 int64_t N, int64_t K, int vec, int64_t kchunk,
                 const uint8_t* __restrict__ xm, const uint8_t* __restrict__ ym,
                 unsigned long long* ktiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (xm != nullptr) {
        const int64_t nkb = (K + BK - 1) / BK, nnb = (N + BN - 1) / BN;
        const uint8_t* xr = xm + (int64_t)blockIdx.y * nkb;
        int dead = 0;
        for (int64_t t = threadIdx.x; t < nkb; t += THREADS)
            dead |= !(xr[t] & ym[t * nnb + blockIdx.x]);
        if (__syncthreads_or(dead)) return;
        if (ktiles != nullptr && threadIdx.x == 0) atomicAdd(ktiles, (unsigned long long)nkb);
    }
    // blockIdx.z: the K split [k0, k0 + kchunk) (one split: all of K).
    const int64_t k0 = (int64_t)blockIdx.z * kchunk;
    const int64_t kn = K - k0 < kchunk ? K - k0 : kchunk;
    simt_tile<Op>(A + k0, lda, B + k0 * ldb, ldb, C, ldc, M, N, kn, vec,
                  (int64_t)blockIdx.y * BM, (int64_t)blockIdx.x * BN, smem_raw,
                  gridDim.z > 1);
}

// The CTAs with a dead k tile (FP32, one K split): live flags in shared
// memory after the stages, only the live k tiles loaded and multiplied.
__global__ void __launch_bounds__(THREADS, 1)
simt_masked_kernel(const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
                   int64_t ldb, float* __restrict__ C, int64_t ldc, int64_t M, int64_t N,
                   int64_t K, int vec, const uint8_t* __restrict__ xm,
                   const uint8_t* __restrict__ ym, unsigned long long* ktiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t nkb = (K + BK - 1) / BK, nnb = (N + BN - 1) / BN;
    uint8_t* live = smem_raw + SMEM_BYTES;
    const uint8_t* xr = xm + (int64_t)blockIdx.y * nkb;
    int mine = 0, dead = 0;
    for (int64_t t = threadIdx.x; t < nkb; t += THREADS) {
        live[t] = xr[t] & ym[t * nnb + blockIdx.x];
        mine += live[t];
        dead |= !live[t];
    }
    if (!__syncthreads_or(dead)) return;
    if (ktiles != nullptr) {
        __shared__ int total;
        if (threadIdx.x == 0) total = 0;
        __syncthreads();
        if (mine) atomicAdd(&total, mine);
        __syncthreads();
        if (threadIdx.x == 0 && total) atomicAdd(ktiles, (unsigned long long)total);
    }
    simt_tile<OpF32, true>(A, lda, B, ldb, C, ldc, M, N, K, vec, (int64_t)blockIdx.y * BM,
                           (int64_t)blockIdx.x * BN, smem_raw, false, live);
}

// K0 tile masks: mask[tr][tc] = 1 when the tr x tc tile (TR x TC elements)
// of the FP32 matrix G (rows x cols, row stride ld) holds a non-zero
// (NaN counts as non-zero), else 0.  A CTA scans TR rows x 8 tiles.
template <int TR, int TC>
__global__ void __launch_bounds__(256)
tile_mask_kernel(const float* __restrict__ G, int64_t ld, int64_t rows, int64_t cols,
                 int vec, uint8_t* __restrict__ mask, int64_t ntc) {
    __shared__ int any[8];
    if (threadIdx.x < 8) any[threadIdx.x] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.y * TR, c0 = (int64_t)blockIdx.x * 8 * TC;
    constexpr int W4 = 8 * TC / 4;                  // 4-element pieces per row
    for (int q = threadIdx.x; q < TR * W4; q += 256) {
        const int r = q / W4, p = q % W4;
        const int64_t gr = r0 + r, gc = c0 + (int64_t)p * 4;
        if (gr >= rows || gc >= cols) continue;
        const float* src = G + gr * ld + gc;
        bool nz;
        if (vec && gc + 3 < cols) {
            const float4 v = *reinterpret_cast<const float4*>(src);
            nz = !(v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f);
        } else {
            nz = false;
            for (int t = 0; t < 4 && gc + t < cols; ++t) nz |= !(src[t] == 0.f);
        }
        if (nz) any[(p * 4) / TC] = 1;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int64_t tc = (int64_t)blockIdx.x * 8 + threadIdx.x;
        if (tc < ntc) mask[(int64_t)blockIdx.y * ntc + tc] = (uint8_t)any[threadIdx.x];
    }
}

// Grouped form: block b runs tile b - tile_prefix[j] of job j, where
// tile_prefix is the exclusive prefix sum of the jobs' tile counts.
__global__ void __launch_bounds__(THREADS, 1)
simt_grouped_kernel(const SimtJob* __restrict__ jobs,
                    const int* __restrict__ tile_prefix, int njobs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {                       // last j with tile_prefix[j] <= b
        const int mid = (lo + hi + 1) >> 1;
        if (tile_prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const SimtJob& j = jobs[lo];
    const int t = b - tile_prefix[lo];
    const int tn = t % j.tiles_n, tm = t / j.tiles_n;
    simt_tile<OpF32>(j.A, j.lda, j.B, j.ldb, j.C, j.ldc, j.M, j.N, j.K, j.vec,
                     (int64_t)tm * BM, (int64_t)tn * BN, smem_raw);
}

inline bool aligned16(const void* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

template <class Op>
afmm_status launch_simt(const typename Op::Elt* A, int64_t lda,
                        const typename Op::Elt* B, int64_t ldb,
                        typename Op::Acc* C, int64_t ldc, int64_t M, int64_t N,
                        int64_t K, cudaStream_t st, const uint8_t* xm = nullptr,
                        const uint8_t* ym = nullptr, unsigned long long* ktiles = nullptr) {
    if (M <= 0 || N <= 0) return AFMM_OK;
    const int64_t nkb = (K + BK - 1) / BK;
    if (nkb > kMaskMaxKTiles || !std::is_same<Op, OpF32>::value) xm = ym = nullptr;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(
        simt_gemm_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    const int vec = (lda % 4 == 0) && (ldb % 4 == 0) && (ldc % 4 == 0) &&
                    aligned16(A) && aligned16(B) && aligned16(C);
    const int64_t gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM;
    if (gy > 65535) return AFMM_ERR_UNSUPPORTED;
    // Integer products with fewer tiles than SMs split K (partial sums
    // added atomically into a zeroed C; exact, so the order does not show).
    int64_t kchunk = K > 0 ? K : 1, splits = 1;
    if constexpr (std::is_same<typename Op::Acc, int32_t>::value) {
        DeviceProps dp;
        AFMM_TRY(device_props(&dp));
        const int64_t tiles = gx * gy, ktiles = (K + BK - 1) / BK;
        if (tiles < dp.sm_count && ktiles > 1) {
            int64_t want = (2 * (int64_t)dp.sm_count + tiles - 1) / tiles;
            if (want > ktiles) want = ktiles;
            kchunk = (ktiles + want - 1) / want * BK;
            splits = (K + kchunk - 1) / kchunk;
        }
    }
    if (splits > 1) {
        xm = ym = nullptr;                  // masks index whole-K tiles
        AFMM_CUDA_TRY(cudaMemset2DAsync(C, ldc * sizeof(typename Op::Acc), 0,
                                        N * sizeof(typename Op::Acc), M, st));
    }
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)splits);
    main_kernel_begin(st);
    simt_gemm_kernel<Op><<<grid, THREADS, SMEM_BYTES, st>>>(A, lda, B, ldb, C, ldc, M, N, K,
                                                            vec, kchunk, xm, ym, ktiles);
    AFMM_CUDA_TRY(cudaGetLastError());
    if constexpr (std::is_same<Op, OpF32>::value) {
        if (xm != nullptr) {
            // The same grid; CTAs without a dead k tile return at once.
            const int smem = SMEM_BYTES + (int)((nkb + 15) / 16 * 16);
            AFMM_CUDA_TRY(cudaFuncSetAttribute(
                simt_masked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            simt_masked_kernel<<<grid, THREADS, smem, st>>>(A, lda, B, ldb, C, ldc, M, N, K,
                                                            vec, xm, ym, ktiles);
            AFMM_CUDA_TRY(cudaGetLastError());
            count_launches(1);
        }
    }
    main_kernel_end(st, (int)(gx * gy));
    count_launches(1);
    return AFMM_OK;
}

}  // namespace

afmm_status launch_simt_f32(const float* A, int64_t lda, const float* B,
                            int64_t ldb, float* C, int64_t ldc, int64_t M,
                            int64_t N, int64_t K, cudaStream_t st, const uint8_t* xm,
                            const uint8_t* ym, unsigned long long* ktiles) {
    return launch_simt<OpF32>(A, lda, B, ldb, C, ldc, M, N, K, st, xm, ym, ktiles);
}

size_t simt_mask_bytes(int64_t M, int64_t N, int64_t K, size_t* ym_offset) {
    const int64_t nkb = (K + BK - 1) / BK;
    const size_t xb = (size_t)((M + BM - 1) / BM) * (size_t)nkb;
    const size_t yb = (size_t)nkb * (size_t)((N + BN - 1) / BN);
    if (ym_offset) *ym_offset = (xb + 15) / 16 * 16;
    return (xb + 15) / 16 * 16 + yb;
}

afmm_status launch_tile_masks(const float* A, int64_t lda, const float* B, int64_t ldb,
                              int64_t M, int64_t N, int64_t K, uint8_t* xm, uint8_t* ym,
                              cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return AFMM_OK;
    const int64_t nkb = (K + BK - 1) / BK, nnb = (N + BN - 1) / BN;
    const int64_t gya = (M + BM - 1) / BM;
    if (gya > 65535 || nkb > 65535) return AFMM_ERR_UNSUPPORTED;
    const int va = (lda % 4 == 0) && aligned16(A);
    const int vb = (ldb % 4 == 0) && aligned16(B);
    tile_mask_kernel<BM, BK><<<dim3((unsigned)((nkb + 7) / 8), (unsigned)gya), 256, 0, st>>>(
        A, lda, M, K, va, xm, nkb);
    AFMM_CUDA_TRY(cudaGetLastError());
    tile_mask_kernel<BK, BN><<<dim3((unsigned)((nnb + 7) / 8), (unsigned)nkb), 256, 0, st>>>(
        B, ldb, K, N, vb, ym, nnb);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFMM_OK;
}

afmm_status launch_simt_dp4a(const int8_t* A, int64_t lda, const int32_t* W,
                             int64_t ldw, int32_t* C, int64_t ldc, int64_t M,
                             int64_t N, int64_t K, cudaStream_t st) {
    if (lda % 4 != 0) return AFMM_ERR_INVALID_ARG;
    // K counted in 4-byte words of packed int8.
    return launch_simt<OpDp4a>(reinterpret_cast<const int32_t*>(A), lda / 4,
                               W, ldw, C, ldc, M, N, (K + 3) / 4, st);
}

int simt_tiles(int64_t M, int64_t N) {
    return (int)(((M + BM - 1) / BM) * ((N + BN - 1) / BN));
}
int simt_tiles_n(int64_t N) { return (int)((N + BN - 1) / BN); }

afmm_status launch_simt_f32_grouped(const SimtJob* jobs, const int* tile_prefix,
                                    int njobs, int total_tiles, cudaStream_t st) {
    if (njobs <= 0 || total_tiles <= 0) return AFMM_OK;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(simt_grouped_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES));
    simt_grouped_kernel<<<total_tiles, THREADS, SMEM_BYTES, st>>>(jobs, tile_prefix,
                                                                 njobs);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
