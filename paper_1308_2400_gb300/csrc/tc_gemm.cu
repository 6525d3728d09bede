// Tensor-core AFMM product on sm_103a: tcgen05 MMA with TMEM accumulators,
// operands brought in by TMA, warp-specialised persistent kernels.
//
// The AFMM term Rep * Base (Sec. 2: Base added Rep-factor times) is an exact
// integer multiple of the Base value.  On the tensor cores it is formed as a
// product of BF16 operands accumulated in FP32:
//  - Rep-factors are small non-negative integers, exact in BF16 (all
//    integers up to 256);
//  - the real Base factor is split into S BF16 slices, hi + mid + lo, each
//    the round-to-nearest BF16 of the previous residual, so that for S = 3 the
//    slices sum exactly to an FP32 value;
//  - the slices are always the A operand: Case A multiplies X's slices by
//    Y, Case B computes Z^T = Y^T X^T with Y's slices and stores the tiles
//    transposed; the Rep-factor tile of a k step is loaded once and used by
//    the S MMAs.
// The same kernel runs the FP8 form (F8: four E4M3 slices of the row-scaled
// real factor, kind::f8f6f4, tc_fp8.cu / fp8_split.cuh) and the real x real
// product (no Rep-factor: three BF16 slices of both factors, six of the nine
// slice products).
//
// tc_gemm_kernel (split form; one CTA per SM, persistent over 128 x 256
// output tiles):
//   warp 0      TMA producer: K steps of 32 (64-byte swizzled rows) of every
//               slice of A and of B into a ring of shared-memory stages;
//   warp 1      allocates 512 TMEM columns and issues the MMAs
//               (128 x 256 x 16): the hi slice's products into columns
//               [0,256), the smaller slices' into [256,512), so that a small
//               product is never added into a much larger sum;
//   warps 2..9  epilogue: TMEM -> registers (the two sums added with one
//               rounding) -> Z; the next tile's MMAs start as soon as the
//               TMEM has been read, while the stores are in flight.
// tc_exact2_kernel (exact form; 256 x 256 tiles): see there.
// Every wait on an mbarrier is bounded (2 s); a wait that runs out records
// AFMM_ERR_TIMEOUT in the status word, stops the other roles, lets copies
// and MMAs in flight finish (bounded) and frees TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "afmm_common.cuh"
#include "elem.cuh"
#include "fp16_split.cuh"
#include "fp8_split.cuh"
#include "ptx_sm100.cuh"
#include "tc_gemm.cuh"

namespace afmm {

namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 32;
constexpr int TC_EPI_THREADS = 256;              // 8 epilogue warps
constexpr int TC_THREADS = 64 + TC_EPI_THREADS;
constexpr uint32_t TMEM_COLS = 512;
constexpr int A_TILE_BYTES = TC_BM * TC_BK * 2;   // 8 KiB
constexpr int B_TILE_BYTES = TC_BN * TC_BK * 2;   // 16 KiB
constexpr int SMEM_OPTIN = 232448;                // 227 KiB per CTA
constexpr int GROUP_M = 10;                       // tile raster band
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;
// k-blocks per chunk of the hi sum (0: one chunk per tile): FP8 form
// (blocks of 64), real x real form (blocks of 32).
constexpr int kF8ChunkKb = 16;
constexpr int kRealChunkKb = 12;
constexpr int MAX_STAGES = 16;                    // mbarrier pairs in the barrier block
constexpr int BARS_BYTES = 512;                   // barrier block after the stages

template <int SA, int SB>
struct TcCfg {
    static constexpr int STAGE_BYTES = SA * A_TILE_BYTES + SB * B_TILE_BYTES;
    static constexpr int STAGES_FIT = (SMEM_OPTIN - 2048) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + BARS_BYTES;
    // Both factors sliced (three slices each: the real x real form) or one.
    static constexpr bool BOTH = SA > 1 && SB > 1;
    // MMAs per 32-byte K step: one per slice, or six slice pairs.
    static constexpr int P = BOTH ? 6 : (SA > SB ? SA : SB);
    static_assert(!BOTH || (SA == 3 && SB == 3), "both sides: three slices each");
    static_assert(STAGES >= 2, "pipeline needs two stages");
    static_assert(SMEM <= SMEM_OPTIN, "shared memory");
};

struct TcBars {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(TcBars) <= BARS_BYTES, "barrier block");

// (A slice, B slice) of product p.  One-sided forms pair slice p with the
// other side's only tile.  With three BF16 slices on both sides (a real x
// real product) the six pairs whose products reach down to 2^-16 of the hi
// product: (0,0), (0,1), (1,0), (0,2), (1,1), (2,0); the pairs left out,
// (1,2), (2,1), (2,2), are below 2^-23 of it.
template <int SA, int SB>
__device__ __forceinline__ constexpr int slice_a(int p) {
    return SA > 1 && SB > 1 ? (p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0)) : (SA > 1 ? p : 0);
}
template <int SA, int SB>
__device__ __forceinline__ constexpr int slice_b(int p) {
    return SA > 1 && SB > 1 ? (p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0)) : (SB > 1 ? p : 0);
}

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n,
                                            int& tm, int& tn) {
    const int per_group = GROUP_M * tiles_n;
    const int g = tile / per_group;
    const int first_m = g * GROUP_M;
    const int gm = min(tiles_m - first_m, GROUP_M);
    const int r = tile % per_group;
    tm = first_m + r % gm;
    tn = r / gm;
}

__device__ __forceinline__ void raise_abort(TcBars* b, int* status) {
    b->abort = 1;
    __threadfence_block();
    atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
}

// TOUT: the product computed is Z^T (A = the operand whose rows are Z's
// columns); the epilogue stores tile element (m, n) at Z[n][m].
// F8: E4M3 operands (kind::f8f6f4), SA = 4 slices of the row-scaled real
// factor (tc_fp8.cu): slices 1-3 accumulate into the hi sum, slice 4 (cut
// from the residual times 2^12) into the small sum; amax[m] holds the bits
// of A row m's largest |value|, from which f8_row_shift() gives the power
// of two the row was scaled by, undone in the epilogue.  The tensor pipe
// adds E4M3 products into its FP32 accumulator less precisely than BF16
// ones, an error that grows with the number of additions; so the hi sum is
// closed every kbpc k-blocks (kbpc > 0) and handed to the epilogue, which
// adds the chunks in FP32 registers (round to nearest) while the MMAs wait.
template <int SA, int SB, bool TOUT = false, bool F8 = false, bool H16 = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
               const __grid_constant__ CUtensorMap tmB, float* __restrict__ Z,
               int64_t ldz, int m0, int M, int n0, int N, int K, int vec, int* status,
               const uint32_t* __restrict__ amax, int kbpc) {
    using Cfg = TcCfg<SA, SB>;
    // Elements per 64-byte K block; slices whose products go to the hi sum.
    constexpr int BK = F8 ? 64 : TC_BK;
    constexpr int HI = F8 ? 3 : 1;
    static_assert(!F8 || (SA == 4 && SB == 1), "FP8 form: four A slices");
    static_assert(!H16 || (SA == 2 && SB == 1 && !F8), "FP16 form: two A slices");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    uint8_t* tiles = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    TcBars* bars = reinterpret_cast<TcBars*>(tiles + Cfg::STAGES * Cfg::STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Product rows [m0, M) and columns [n0, N): tile (tm, tn) covers rows
    // m0 + tm*BM .. and columns n0 + tn*BN ..
    const int tiles_m = (M - m0 + TC_BM - 1) / TC_BM, tiles_n = (N - n0 + TC_BN - 1) / TC_BN;
    const int num_tiles = tiles_m * tiles_n;
    const int num_kb = (K + BK - 1) / BK;
    // k-blocks per chunk of the hi sum, and chunks per tile.
    // The FP8 and real x real forms close their hi sum every kbpc k-blocks.
    constexpr bool CH = F8 || Cfg::BOTH;
    const int kc = (CH && kbpc > 0 && kbpc < num_kb) ? kbpc : num_kb;
    const int nch = (num_kb + kc - 1) / kc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            ptx::mbar_init(&bars->full[s], 1);
            ptx::mbar_init(&bars->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(&bars->tfull[a], 1);
            ptx::mbar_init(&bars->tempty[a], TC_EPI_THREADS);
        }
        ptx::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        ptx::tmem_alloc(&bars->tmem_base, TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[8];
            for (int s = 0; s < 8; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
                int tm, tn;
                tile_coords(tile, tiles_m, tiles_n, tm, tn);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&bars->empty[stage], phase ^ 1u, abort,
                                                WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&bars->full[stage], Cfg::STAGE_BYTES);
                    uint8_t* st = tiles + stage * Cfg::STAGE_BYTES;
#pragma unroll
                    for (int s = 0; s < SA; ++s)
                        ptx::tma_load_3d(st + s * A_TILE_BYTES, &tmA, &bars->full[stage],
                                         kb * BK, m0 + tm * TC_BM, s);
#pragma unroll
                    for (int s = 0; s < SB; ++s)
                        ptx::tma_load_3d(st + SA * A_TILE_BYTES + s * B_TILE_BYTES, &tmB,
                                         &bars->full[stage], kb * BK, n0 + tn * TC_BN, s);
                    issued_phase[stage] = (int)phase;
                    if (++stage == Cfg::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                raise_abort(bars, status);
                // Let this CTA's copies in flight land before it exits.
                volatile int never = 0;
                for (int s = 0; s < Cfg::STAGES; ++s)
                    if (issued_phase[s] >= 0)
                        ptx::mbar_wait_bounded(&bars->full[s], (uint32_t)issued_phase[s],
                                               &never, WAIT_LIMIT_NS);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = F8    ? ptx::idesc_e4m3_f32(TC_BM, TC_BN)
                                       : H16 ? ptx::idesc_f16_f32(TC_BM, TC_BN)
                                             : ptx::idesc_bf16_f32(TC_BM, TC_BN);
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            // Split form: per tile two 128 x 256 FP32 accumulators in
            // TMEM, columns [0,256) for the products of the hi slice(s) and
            // [256,512) for those of the smaller slices, so a small
            // product is never added into a sum of much larger
            // magnitude.  The epilogue adds the two.
            uint32_t tphase = 0;
            for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
                if (!ptx::mbar_wait_bounded(&bars->tempty[0], tphase ^ 1u, abort,
                                            WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                for (int kb = 0; kb < num_kb; ++kb) {
                    const bool chunk0 = kb % kc == 0;
                    if (kb > 0 && chunk0) {
                        // Chunk boundary: the epilogue takes the hi sum;
                        // the next chunk overwrites it once it has.
                        ptx::mma_commit(&bars->tfull[0]);
                        tphase ^= 1u;
                        if (!ptx::mbar_wait_bounded(&bars->tempty[0], tphase ^ 1u, abort,
                                                    WAIT_LIMIT_NS)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                    }
                    if (!ptx::mbar_wait_bounded(&bars->full[stage], phase, abort,
                                                WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t s0 = ptx::smem_addr(tiles + stage * Cfg::STAGE_BYTES);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {     // two 32-byte MMA steps
#pragma unroll
                        for (int p = Cfg::P - 1; p >= 0; --p) {
                            const uint32_t a_addr =
                                s0 + slice_a<SA, SB>(p) * A_TILE_BYTES + ks * 32;
                            const uint32_t b_addr = s0 + SA * A_TILE_BYTES +
                                                    slice_b<SA, SB>(p) * B_TILE_BYTES +
                                                    ks * 32;
                            // Products are issued from the last (smallest):
                            // the first MMA into each accumulator overwrites it.
                            const bool first =
                                ks == 0 && ((chunk0 && p == HI - 1) ||
                                            (kb == 0 && p == Cfg::P - 1));
                            const uint32_t d = tmem + (p < HI ? 0u : (uint32_t)TC_BN);
                            if constexpr (F8)
                                ptx::mma_f8(d, ptx::sdesc_kmajor_sw64(a_addr),
                                            ptx::sdesc_kmajor_sw64(b_addr), IDESC,
                                            first ? 0u : 1u);
                            else
                                ptx::mma_f16(d, ptx::sdesc_kmajor_sw64(a_addr),
                                             ptx::sdesc_kmajor_sw64(b_addr), IDESC,
                                             first ? 0u : 1u);
                        }
                    }
                    ptx::mma_commit(&bars->empty[stage]);
                    if (++stage == Cfg::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                ptx::mma_commit(&bars->tfull[0]);
                tphase ^= 1u;
            }
            if (!ok) raise_abort(bars, status);
            // Every MMA issued above completes before TMEM is released.
            ptx::mma_commit(&bars->drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(&bars->drain, 0u, &never, WAIT_LIMIT_NS);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue
        // 8 warps: warp w reads TMEM lanes 32*(w%4).. (its rows) and half
        // h of the 256 columns, 128 values per thread.
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128);
        uint32_t tphase = 0;
        for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
            int tm, tn;
            tile_coords(tile, tiles_m, tiles_n, tm, tn);
            float sum[128];
            bool got = true;
            // F8, chunks before the last: add the hi sum into sum[].
            for (int ch = 0; CH && ch + 1 < nch; ++ch) {
                got = __all_sync(0xffffffffu, ptx::mbar_wait_bounded(&bars->tfull[0], tphase,
                                                                      abort, WAIT_LIMIT_NS));
                if (!got) break;
                ptx::tc_fence_after();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t r0[16];
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(c * 16), r0);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        sum[c * 16 + j] = ch == 0 ? __uint_as_float(r0[j])
                                                  : sum[c * 16 + j] + __uint_as_float(r0[j]);
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(&bars->tempty[0]);
                tphase ^= 1u;
            }
            // TMEM loads below are warp-collective: decide as a warp.
            if (got)
                got = __all_sync(0xffffffffu, ptx::mbar_wait_bounded(&bars->tfull[0], tphase,
                                                                      abort, WAIT_LIMIT_NS));
            if (!got) {
                if (lane == 0) raise_abort(bars, status);
                break;
            }
            ptx::tc_fence_after();
            const int64_t m = (int64_t)m0 + (int64_t)tm * TC_BM + row;
            // F8, H16: row m was scaled by 2^sh; 2^-sh as two exact factors.
            float f1 = 1.f, f2 = 1.f;
            if constexpr (F8 || H16) {
                const int sh = m < M ? (F8 ? f8_row_shift(amax[m]) : h16_row_shift(amax[m])) : 0;
                const int e1 = max(-sh, -126);
                f1 = f8_pow2(e1);
                f2 = f8_pow2(-sh - e1);
            }
            if constexpr (H16) {
                // hi sum plus the lo sum times 2^-8 (one rounding), times
                // the row's scale (exact).
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t r0[16], r1[16];
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(c * 16), r0);
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(TC_BN + c * 16), r1);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        sum[c * 16 + j] = fmaf(__uint_as_float(r1[j]), 0x1p-8f,
                                               __uint_as_float(r0[j])) * f1 * f2;
                }
            } else if constexpr (F8) {
                // Last chunk of the hi sum plus the small sum times 2^-12
                // (one rounding), times the row's scale (exact); 16 columns
                // per load, so sum[] and the loads fit the registers.
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t r0[16], r1[16];
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(c * 16), r0);
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(TC_BN + c * 16), r1);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float hi = nch > 1 ? sum[c * 16 + j] + __uint_as_float(r0[j])
                                                 : __uint_as_float(r0[j]);
                        sum[c * 16 + j] =
                            fmaf(__uint_as_float(r1[j]), 0x1p-12f, hi) * f1 * f2;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    // hi-slice sum (its last chunk added to the earlier ones)
                    // + small-slice sum, one rounding.
                    uint32_t r0[16], r1[16];
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(c * 16), r0);
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(TC_BN + c * 16), r1);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float hi = CH && nch > 1
                                             ? sum[c * 16 + j] + __uint_as_float(r0[j])
                                             : __uint_as_float(r0[j]);
                        sum[c * 16 + j] = hi + __uint_as_float(r1[j]);
                    }
                }
            }
            // TMEM is free again before the stores below.
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars->tempty[0]);
            tphase ^= 1u;
            const int col0 = n0 + tn * TC_BN + h * 128;
            if (TOUT && m < M) {
                // Element (m, col0 + j) of Z^T is Z[col0 + j][m]: the lanes of
                // a warp hold consecutive m, so each store writes one
                // 128-byte segment of a row of Z.
                float* zc = Z + m;
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (col0 + j < N) zc[(int64_t)(col0 + j) * ldz] = sum[j];
            } else if (m < M) {
                float* zr = Z + m * ldz + col0;
                if (vec && col0 + 128 <= N) {
#pragma unroll
                    for (int j = 0; j < 128; j += 4)
                        *reinterpret_cast<float4*>(zr + j) =
                            make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (col0 + j < N) zr[j] = sum[j];
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// --------------------------------------------------- two-SM split form
// tc_pair_kernel: the split form of tc_gemm_kernel (S BF16 slices of the real
// factor on the A side, one Rep-factor tile on the B side, hi and small sums
// in two TMEM accumulators) computed by clusters of two CTAs on the two SMs
// of a pair with tcgen05 cta_group::2.  A pair owns a 256 x 256 output tile:
// CTA r holds A rows [128 r, 128 r + 128) of the tile's slices and B rows
// (product columns) [128 r, 128 r + 128) in its shared memory, and the
// accumulator rows [128 r, 128 r + 128) x all 256 columns in its TMEM.  The
// even CTA issues every MMA (M = 256, N = 256, K = 16), whose B operand
// is read from both CTAs' halves, so each SM stages and reads half the B
// bytes per flop of the one-CTA kernel: per 32-wide K step a CTA receives
// S x 8 KiB + 8 KiB instead of S x 8 KiB + 16 KiB, and its tensor core reads
// 4 + 4 KiB per MMA instead of 4 + 8 KiB.
//   - Both CTAs' TMA copies of a stage complete on the even CTA's `full`
//     barrier (cta_group::2 copies), which expects both CTAs' bytes.
//   - The MMA commits free a stage in both CTAs and hand a finished tile to
//     both CTAs' epilogues (multicast commits).
//   - Each epilogue warp of either CTA arrives on the even CTA's `tempty`
//     barrier (16 arrivals) once it has read its TMEM lanes.
// Every wait is bounded; an abort raised in one CTA is written into the
// peer's flag too, and both CTAs meet at cluster barriers at the start
// (barriers initialised) and before releasing TMEM.
constexpr int PR_BM = 256, PR_BN = 256;           // pair tile
constexpr int PR_HALF = 128;                       // rows of A and of B per CTA
constexpr int PR_GROUP_M = 5;                      // tile raster band (tile rows)
constexpr int PR_EPI_WARPS = 2 * (TC_EPI_THREADS / 32);   // tempty arrivals

// A stage holds SUB consecutive K blocks of RB-byte operand rows (64: a
// 64-byte swizzle, 128: a 128-byte swizzle), each laid out as its SA A
// tiles (128 rows) then its B tile (128 rows).  SUB = 2 halves the stage
// hand-overs per MMA; 128-byte rows move the same stage in half as many
// TMA row requests as two 64-byte blocks.
template <int SA, int SUB = 1, int RB = 64>
struct PairCfg {
    static constexpr int A_BYTES = PR_HALF * RB;     // one A slice tile
    static constexpr int B_BYTES = PR_HALF * RB;     // this CTA's half of B
    static constexpr int SUB_BYTES = SA * A_BYTES + B_BYTES;
    static constexpr int STAGE_BYTES = SUB * SUB_BYTES;
    static constexpr int STAGES_FIT = (SMEM_OPTIN - 1024 - BARS_BYTES) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT > MAX_STAGES ? MAX_STAGES : STAGES_FIT;
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + BARS_BYTES;
    static_assert(STAGES >= 2, "pipeline needs two stages");
    static_assert(SMEM <= SMEM_OPTIN, "shared memory");
};

__device__ __forceinline__ void pair_tile_coords(int tile, int tiles_m, int tiles_n, int& tm,
                                                 int& tn) {
    const int per_group = PR_GROUP_M * tiles_n;
    const int g = tile / per_group;
    const int first_m = g * PR_GROUP_M;
    const int gm = min(tiles_m - first_m, PR_GROUP_M);
    const int r = tile % per_group;
    tm = first_m + r % gm;
    tn = r / gm;
}

__device__ __forceinline__ void raise_abort_pair(TcBars* b, uint32_t peer_abort, int* status) {
    b->abort = 1;
    ptx::st_shared_cluster_u32(peer_abort, 1u);
    __threadfence_block();
    atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
}

// Work unit u of a pair: the first `whole` units are whole 256 x 256
// tiles; the units after them cut each of the last tiles into `split`
// column parts of 256 / split columns (256 x 128 for split = 2), so that a
// last round with fewer tiles than pairs still spreads over all pairs.
struct PairUnit {
    int tm, tn;       // pair tile
    int col;          // first column of the part inside the tile
    int width;        // columns of the part: 256, or 128
};
__device__ __forceinline__ PairUnit pair_unit(int u, int whole, int split, int tiles_m,
                                              int tiles_n) {
    PairUnit w;
    int tile = u, part = 0;
    w.width = PR_BN;
    if (u >= whole) {
        tile = whole + (u - whole) / split;
        part = (u - whole) % split;
        w.width = PR_BN / split;
    }
    pair_tile_coords(tile, tiles_m, tiles_n, w.tm, w.tn);
    w.col = part * w.width;
    return w;
}

// Modes of the pair kernel: the split-BF16 form, the FP16 two-slice form,
// and the exact form on E4M3 digits (A = two digit slices h, l of integer
// values x = 16 h + l, B = E4M3 Rep-factors; every partial sum is an exact
// integer below 2^24, and the epilogue writes 16 acc_h + acc_l as int32).
constexpr int PM_SPLIT = 0, PM_H16 = 1, PM_X8 = 2;

template <int SA, bool TOUT, int MODE = PM_SPLIT, int SUB = 1, int RB = 64>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_pair_kernel(const __grid_constant__ CUtensorMap tmA,
               const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmB64, float* __restrict__ Z, int64_t ldz,
               int m0, int M, int n0, int N, int K, int vec, int split, int* status,
               const uint32_t* __restrict__ amax) {
    using Cfg = PairCfg<SA, SUB, RB>;
    constexpr bool H16 = MODE == PM_H16, X8 = MODE == PM_X8;
    static_assert((!H16 && !X8) || SA == 2, "FP16 and digit forms: two A slices");
    static_assert(RB == 64 || RB == 128, "64- or 128-byte operand rows");
    // Elements per RB-byte row of a K block; 32-byte MMA K steps per row.
    constexpr int BKE = X8 ? RB : RB / 2;
    constexpr int KSTEPS = RB / 32;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    uint8_t* tiles = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    TcBars* bars = reinterpret_cast<TcBars*>(tiles + Cfg::STAGES * Cfg::STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = ptx::cluster_ctarank();
    const bool leader = rank == 0;
    const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
    const int tiles_m = (M - m0 + PR_BM - 1) / PR_BM, tiles_n = (N - n0 + PR_BN - 1) / PR_BN;
    const int num_tiles = tiles_m * tiles_n;
    const int num_kb = (K + BKE - 1) / BKE;
    // The tiles of the last, partial round are split when split > 1.
    const int rem = split > 1 ? num_tiles % npairs : 0;
    const int whole = num_tiles - rem;
    const int num_units = whole + split * rem;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            ptx::mbar_init(&bars->full[s], 1);
            ptx::mbar_init(&bars->empty[s], 1);
        }
        ptx::mbar_init(&bars->tfull[0], 1);
        ptx::mbar_init(&bars->tempty[0], PR_EPI_WARPS);
        ptx::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        ptx::prefetch_tmap(&tmB64);
    }
    if (warp == 1) {
        ptx::tmem_alloc_pair(&bars->tmem_base, TMEM_COLS);
        ptx::tmem_relinquish_pair();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();           // both CTAs' barriers exist before any remote use
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;
    const uint32_t peer_abort = ptx::mapa_shared(ptx::smem_addr(&bars->abort), rank ^ 1u);

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[MAX_STAGES];
            for (int s = 0; s < MAX_STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int u = pair; ok && u < num_units; u += npairs) {
                const PairUnit w = pair_unit(u, whole, split, tiles_m, tiles_n);
                const int arow = m0 + w.tm * PR_BM + (int)rank * PR_HALF;
                // Each CTA holds half of the unit's B rows (128, or 64).
                const int bhalf = w.width / 2;
                const int brow = n0 + w.tn * PR_BN + w.col + (int)rank * bhalf;
                const CUtensorMap* mb = w.width == PR_BN ? &tmB : &tmB64;
                const uint32_t bytes = SA * Cfg::A_BYTES + (uint32_t)bhalf * RB;
                for (int kb0 = 0; kb0 < num_kb; kb0 += SUB) {
                    if (!ptx::mbar_wait_cluster_bounded(&bars->empty[stage], phase ^ 1u, abort,
                                                        WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    // K blocks of this stage (the last stage may hold fewer).
                    const int nsub = num_kb - kb0 < SUB ? num_kb - kb0 : SUB;
                    // The even CTA's barrier counts both CTAs' bytes.
                    if (leader)
                        ptx::mbar_arrive_expect_tx(&bars->full[stage], 2 * bytes * (uint32_t)nsub);
                    const uint32_t full0 =
                        ptx::mapa_shared(ptx::smem_addr(&bars->full[stage]), 0u);
#pragma unroll
                    for (int q = 0; q < SUB; ++q) {
                        if (q >= nsub) break;
                        const int kb = kb0 + q;
                        uint8_t* st = tiles + stage * Cfg::STAGE_BYTES + q * Cfg::SUB_BYTES;
#pragma unroll
                        for (int s = 0; s < SA; ++s)
                            ptx::tma_load_3d_pair(st + s * Cfg::A_BYTES, &tmA, full0, kb * BKE,
                                                  arow, s);
                        ptx::tma_load_3d_pair(st + SA * Cfg::A_BYTES, mb, full0, kb * BKE, brow,
                                              0);
                    }
                    issued_phase[stage] = (int)phase;
                    if (++stage == Cfg::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                raise_abort_pair(bars, peer_abort, status);
                // Let copies in flight land before this CTA can exit: the
                // even CTA waits for the phases it expected; both wait a
                // bounded while for the rest (copies take microseconds).
                volatile int never = 0;
                if (leader)
                    for (int s = 0; s < Cfg::STAGES; ++s)
                        if (issued_phase[s] >= 0)
                            ptx::mbar_wait_cluster_bounded(&bars->full[s],
                                                           (uint32_t)issued_phase[s], &never,
                                                           WAIT_LIMIT_NS);
                const uint64_t t0 = ptx::globaltimer_ns();
                while (ptx::globaltimer_ns() - t0 < 2000000ull) {
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0 && leader) {
            int stage = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            for (int u = pair; ok && u < num_units; u += npairs) {
                const int width = u < whole ? PR_BN : PR_BN / split;
                const uint32_t IDESC = X8    ? ptx::idesc_e4m3_f32(PR_BM, width)
                                       : H16 ? ptx::idesc_f16_f32(PR_BM, width)
                                             : ptx::idesc_bf16_f32(PR_BM, width);
                if (!ptx::mbar_wait_cluster_bounded(&bars->tempty[0], tphase ^ 1u, abort,
                                                    WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                for (int kb0 = 0; kb0 < num_kb; kb0 += SUB) {
                    if (!ptx::mbar_wait_cluster_bounded(&bars->full[stage], phase, abort,
                                                        WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int nsub = num_kb - kb0 < SUB ? num_kb - kb0 : SUB;
#pragma unroll
                    for (int q = 0; q < SUB; ++q) {
                        if (q >= nsub) break;
                        const uint32_t s0 = ptx::smem_addr(tiles + stage * Cfg::STAGE_BYTES) +
                                            (uint32_t)(q * Cfg::SUB_BYTES);
#pragma unroll
                        for (int ks = 0; ks < KSTEPS; ++ks) {     // 32-byte MMA steps
#pragma unroll
                            for (int p = SA - 1; p >= 0; --p) {
                                const uint32_t a_addr = s0 + p * Cfg::A_BYTES + ks * 32;
                                const uint32_t b_addr = s0 + SA * Cfg::A_BYTES + ks * 32;
                                const uint64_t a_desc = RB == 128
                                                            ? ptx::sdesc_kmajor_sw128(a_addr)
                                                            : ptx::sdesc_kmajor_sw64(a_addr);
                                const uint64_t b_desc = RB == 128
                                                            ? ptx::sdesc_kmajor_sw128(b_addr)
                                                            : ptx::sdesc_kmajor_sw64(b_addr);
                                // Issued from the smallest slice: the first MMA
                                // into each accumulator overwrites it.
                                const bool first =
                                    kb0 + q == 0 && ks == 0 && (p == 0 || p == SA - 1);
                                if constexpr (X8)
                                    ptx::mma_f8_pair(tmem + (p == 0 ? 0u : (uint32_t)PR_BN),
                                                     a_desc, b_desc, IDESC, first ? 0u : 1u);
                                else
                                    ptx::mma_f16_pair(tmem + (p == 0 ? 0u : (uint32_t)PR_BN),
                                                      a_desc, b_desc, IDESC, first ? 0u : 1u);
                            }
                        }
                    }
                    ptx::mma_commit_pair_mc(&bars->empty[stage], (uint16_t)3u);
                    if (++stage == Cfg::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                ptx::mma_commit_pair_mc(&bars->tfull[0], (uint16_t)3u);
                tphase ^= 1u;
            }
            if (!ok) raise_abort_pair(bars, peer_abort, status);
            // Every MMA issued above completes before either CTA frees TMEM.
            ptx::mma_commit_pair_mc(&bars->drain, (uint16_t)3u);
        }
        if (lane == 0) {
            volatile int never = 0;
            ptx::mbar_wait_cluster_bounded(&bars->drain, 0u, &never, WAIT_LIMIT_NS);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue
        // Warp w reads TMEM lanes 32*(w%4).. (its rows of this CTA's half)
        // and half h of the 256 columns, 128 values per thread.
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128);
        const uint32_t tempty0 = ptx::mapa_shared(ptx::smem_addr(&bars->tempty[0]), 0u);
        uint32_t tphase = 0;
        for (int u = pair; u < num_units; u += npairs) {
            const PairUnit w = pair_unit(u, whole, split, tiles_m, tiles_n);
            const bool got = __all_sync(
                0xffffffffu,
                ptx::mbar_wait_cluster_bounded(&bars->tfull[0], tphase, abort, WAIT_LIMIT_NS));
            if (!got) {
                if (lane == 0) raise_abort_pair(bars, peer_abort, status);
                break;
            }
            ptx::tc_fence_after();
            // A 128-wide part has columns for the h = 0 warps only.
            const bool live = h * 128 < w.width;
            const int64_t m = (int64_t)m0 + (int64_t)w.tm * PR_BM + (int64_t)rank * PR_HALF + row;
            float sum[128];
            if (live) {
                // H16: row m was scaled by 2^sh; 2^-sh as two exact factors.
                float f1 = 1.f, f2 = 1.f;
                if constexpr (H16) {
                    const int sh = m < M ? h16_row_shift(amax[m]) : 0;
                    const int e1 = max(-sh, -126);
                    f1 = f8_pow2(e1);
                    f2 = f8_pow2(-sh - e1);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    // hi-slice sum + small-slice sum (H16: times 2^-8), one
                    // rounding; H16 then the row's scale (exact).
                    uint32_t r0[16], r1[16];
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(c * 16), r0);
                    ptx::tmem_ld_16cols(lane_base + (uint32_t)(PR_BN + c * 16), r1);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if constexpr (X8)    // int32 bits, stored as they are
                            sum[c * 16 + j] = __int_as_float(
                                16 * __float2int_rn(__uint_as_float(r0[j])) +
                                __float2int_rn(__uint_as_float(r1[j])));
                        else if constexpr (H16)
                            sum[c * 16 + j] = fmaf(__uint_as_float(r1[j]), 0x1p-8f,
                                                   __uint_as_float(r0[j])) * f1 * f2;
                        else
                            sum[c * 16 + j] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
                    }
                }
            }
            // This warp's TMEM lanes are free again before the stores.
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive_cluster(tempty0);
            tphase ^= 1u;
            if (!live) continue;
            const int col0 = n0 + w.tn * PR_BN + w.col + h * 128;
            if (TOUT && m < M) {
                // Element (m, col0 + j) of Z^T is Z[col0 + j][m]: a warp's
                // lanes hold consecutive m, one 128-byte segment per store.
                float* zc = Z + m;
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (col0 + j < N) zc[(int64_t)(col0 + j) * ldz] = sum[j];
            } else if (m < M) {
                float* zr = Z + m * ldz + col0;
                if (vec && col0 + 128 <= N) {
#pragma unroll
                    for (int j = 0; j < 128; j += 4)
                        *reinterpret_cast<float4*>(zr + j) =
                            make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (col0 + j < N) zr[j] = sum[j];
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();           // no remote access to either CTA after this
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc_pair(tmem, TMEM_COLS);
    }
}

// --------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

// 3-D map over a stack of `slices` matrices of `rows` x `cols` (K) es-byte
// elements with leading dimension `ld`; box = row_bytes (64 or 128, with a
// swizzle of that width) of K x box_rows x 1.
afmm_status tc_encode_map(void* out, void* base, int64_t cols, int64_t rows,
                       int64_t ld, int slices, int box_rows, int es, int row_bytes) {
    auto fn = get_encode_fn();
    if (!fn || (es != 1 && es != 2) || (row_bytes != 64 && row_bytes != 128))
        return AFMM_ERR_CUDA;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(ld * es * rows)};
    cuuint32_t box[3] = {(cuuint32_t)(row_bytes / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(out),
                    es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                    3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? AFMM_OK : AFMM_ERR_CUDA;
}

namespace {

// Exact form with 256 x 256 output tiles: the two 128-row halves of a tile
// share each B tile, so one 32-wide K step moves 2 x 8 KiB of A and 16 KiB
// of B through shared memory for two 128 x 256 x 32 MMAs, two thirds of the
// bytes per flop of a 128 x 256 tile (whose load path, not the tensor pipe,
// bounds it).  The halves accumulate into TMEM columns [0,256) and
// [256,512).  K is cut into chunks of kb_per_chunk k-blocks whose FP32
// partial sums are exact integers; the epilogue converts each chunk to
// int32 and stores it (first chunk) or adds it into Z (later chunks, exact).
// Roles, bounded waits and the abort path are those of tc_gemm_kernel.
constexpr int X2_BM = 256, X2_BN = 256;
constexpr int X2_STAGE = 2 * A_TILE_BYTES + B_TILE_BYTES;   // 32 KiB
constexpr int X2_STAGES = 7;
constexpr int X2_SMEM = 1024 + X2_STAGES * X2_STAGE + BARS_BYTES;
static_assert(X2_SMEM <= SMEM_OPTIN, "shared memory");
static_assert(X2_STAGES <= MAX_STAGES, "barrier block");

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_exact2_kernel(const __grid_constant__ CUtensorMap tmA,
                 const __grid_constant__ CUtensorMap tmB, int32_t* __restrict__ Z,
                 int64_t ldz, int M, int N, int K, int kb_per_chunk, int vec, int* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    uint8_t* tiles = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    TcBars* bars = reinterpret_cast<TcBars*>(tiles + X2_STAGES * X2_STAGE);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + X2_BM - 1) / X2_BM, tiles_n = (N + X2_BN - 1) / X2_BN;
    const int num_tiles = tiles_m * tiles_n;
    const int num_kb = (K + TC_BK - 1) / TC_BK;
    const int kbpc = kb_per_chunk > 0 ? kb_per_chunk : num_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < X2_STAGES; ++s) {
            ptx::mbar_init(&bars->full[s], 1);
            ptx::mbar_init(&bars->empty[s], 1);
        }
        ptx::mbar_init(&bars->tfull[0], 1);
        ptx::mbar_init(&bars->tempty[0], TC_EPI_THREADS);
        ptx::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        ptx::tmem_alloc(&bars->tmem_base, TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[X2_STAGES];
            for (int s = 0; s < X2_STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
                int tm, tn;
                tile_coords(tile, tiles_m, tiles_n, tm, tn);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&bars->empty[stage], phase ^ 1u, abort,
                                                WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&bars->full[stage], X2_STAGE);
                    uint8_t* st = tiles + stage * X2_STAGE;
                    ptx::tma_load_3d(st, &tmA, &bars->full[stage], kb * TC_BK, tm * X2_BM, 0);
                    ptx::tma_load_3d(st + A_TILE_BYTES, &tmA, &bars->full[stage], kb * TC_BK,
                                     tm * X2_BM + TC_BM, 0);
                    ptx::tma_load_3d(st + 2 * A_TILE_BYTES, &tmB, &bars->full[stage],
                                     kb * TC_BK, tn * X2_BN, 0);
                    issued_phase[stage] = (int)phase;
                    if (++stage == X2_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                raise_abort(bars, status);
                // Let this CTA's copies in flight land before it exits.
                volatile int never = 0;
                for (int s = 0; s < X2_STAGES; ++s)
                    if (issued_phase[s] >= 0)
                        ptx::mbar_wait_bounded(&bars->full[s], (uint32_t)issued_phase[s],
                                               &never, WAIT_LIMIT_NS);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = ptx::idesc_bf16_f32(TC_BM, TC_BN);
            int stage = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
                for (int kb0 = 0; ok && kb0 < num_kb; kb0 += kbpc) {
                    // Both halves' accumulators are read out before a chunk starts.
                    if (!ptx::mbar_wait_bounded(&bars->tempty[0], tphase ^ 1u, abort,
                                                WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int kb1 = min(kb0 + kbpc, num_kb);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!ptx::mbar_wait_bounded(&bars->full[stage], phase, abort,
                                                    WAIT_LIMIT_NS)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t s0 = ptx::smem_addr(tiles + stage * X2_STAGE);
                        const uint32_t b0 = s0 + 2 * A_TILE_BYTES;
#pragma unroll
                        for (int ks = 0; ks < TC_BK / 16; ++ks) {
#pragma unroll
                            for (int h = 0; h < 2; ++h)
                                ptx::mma_f16(tmem + (uint32_t)(h * TC_BN),
                                             ptx::sdesc_kmajor_sw64(s0 + h * A_TILE_BYTES +
                                                                    ks * 32),
                                             ptx::sdesc_kmajor_sw64(b0 + ks * 32), IDESC,
                                             (kb != kb0 || ks != 0) ? 1u : 0u);
                        }
                        ptx::mma_commit(&bars->empty[stage]);
                        if (++stage == X2_STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    ptx::mma_commit(&bars->tfull[0]);
                    tphase ^= 1u;
                }
            }
            if (!ok) raise_abort(bars, status);
            // Every MMA issued above completes before TMEM is released.
            ptx::mma_commit(&bars->drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(&bars->drain, 0u, &never, WAIT_LIMIT_NS);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue
        // Warp w reads TMEM lanes 32*(w%4).. of half h = (w-2)/4: tile row
        // h*128 + 32*(w%4) + lane, 256 columns in two passes of 128.
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * TC_BN);
        uint32_t tphase = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
            int tm, tn;
            tile_coords(tile, tiles_m, tiles_n, tm, tn);
            const int64_t m = (int64_t)tm * X2_BM + h * TC_BM + q * 32 + lane;
            for (int kb0 = 0; kb0 < num_kb; kb0 += kbpc) {
                const bool got = ptx::mbar_wait_bounded(&bars->tfull[0], tphase, abort,
                                                        WAIT_LIMIT_NS);
                // TMEM loads below are warp-collective: decide as a warp.
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) raise_abort(bars, status);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const bool first = kb0 == 0;
#pragma unroll 1
                for (int ch = 0; ch < 2; ++ch) {
                    int32_t v[128];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint32_t r[32];
                        ptx::tmem_ld_32cols(lane_base + (uint32_t)(ch * 128 + c * 32), r);
                        ptx::tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[c * 32 + j] = __float2int_rn(__uint_as_float(r[j]));
                    }
                    const int col0 = tn * X2_BN + ch * 128;
                    if (m < M) {
                        int32_t* zr = Z + m * ldz + col0;
                        if (vec && col0 + 128 <= N) {
#pragma unroll
                            for (int j = 0; j < 128; j += 4) {
                                int4 o = make_int4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                                if (!first) {
                                    const int4 z = *reinterpret_cast<const int4*>(zr + j);
                                    o.x += z.x;
                                    o.y += z.y;
                                    o.z += z.z;
                                    o.w += z.w;
                                }
                                *reinterpret_cast<int4*>(zr + j) = o;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 128; ++j)
                                if (col0 + j < N) zr[j] = first ? v[j] : zr[j] + v[j];
                        }
                    }
                }
                // TMEM is free again.
                ptx::tc_fence_before();
                ptx::mbar_arrive(&bars->tempty[0]);
                tphase ^= 1u;
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
}

template <int SA, int SB, bool TOUT = false, bool F8 = false, bool H16 = false>
afmm_status launch_tc(const TcPlan* t, float* Z, int64_t ldz, int* status, cudaStream_t st,
                      int m0 = 0, int m1 = -1, int n0 = 0, int n1 = -1) {
    using Cfg = TcCfg<SA, SB>;
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    const int n = (int)t->n;
    if (m1 < 0) m1 = n;
    if (n1 < 0) n1 = n;
    const int tiles = ((m1 - m0 + TC_BM - 1) / TC_BM) * ((n1 - n0 + TC_BN - 1) / TC_BN);
    const int grid = tiles < dp.sm_count ? tiles : dp.sm_count;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<SA, SB, TOUT, F8, H16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg::SMEM));
    const int vec = (ldz % 4 == 0) && ((reinterpret_cast<uintptr_t>(Z) & 15u) == 0);
    CUtensorMap ma, mb;
    std::memcpy(&ma, TOUT ? t->tmap_at : t->tmap_a, sizeof ma);
    std::memcpy(&mb, TOUT ? t->tmap_bt : t->tmap_b, sizeof mb);
    main_kernel_begin(st);
    tc_gemm_kernel<SA, SB, TOUT, F8, H16><<<grid, TC_THREADS, Cfg::SMEM, st>>>(
        ma, mb, Z, ldz, m0, m1, n0, n1, n, vec, status, t->amax, t->chunk_kb);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, grid);
    count_launches(1);
    return AFMM_OK;
}

// Clusters of two CTAs (one per SM of a pair) that fit at once, for the
// pair kernel's persistent grid; 0 when the device cannot co-schedule any.
template <int SA, bool TOUT, int MODE, int SUB, int RB>
int pair_clusters(int smem) {
    static int cached[64];
    static std::once_flag once;
    std::call_once(once, [] { std::fill(cached, cached + 64, -1); });
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    int& c = cached[dev];
    if (c >= 0) return c;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tc_pair_kernel<SA, TOUT, MODE, SUB, RB>, &cfg) !=
        cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    c = n;
    return n;
}

// The two-SM split product over rows [m0, m1) and columns [n0, n1) of the
// product (Z^T's when TOUT).
template <int SA, bool TOUT, int MODE, int SUB, int RB>
afmm_status launch_tc_pair_sub(const TcPlan* t, float* Z, int64_t ldz, int* status,
                               cudaStream_t st, int m0, int m1, int n0, int n1) {
    using Cfg = PairCfg<SA, SUB, RB>;
    const int n = (int)t->n;
    if (m1 < 0) m1 = n;
    if (n1 < 0) n1 = n;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(tc_pair_kernel<SA, TOUT, MODE, SUB, RB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg::SMEM));
    const int tiles = ((m1 - m0 + PR_BM - 1) / PR_BM) * ((n1 - n0 + PR_BN - 1) / PR_BN);
    const int cap = pair_clusters<SA, TOUT, MODE, SUB, RB>(Cfg::SMEM);
    if (cap < 1) return AFMM_ERR_UNSUPPORTED;
    const int clusters = tiles < cap ? tiles : cap;
    const int vec = (ldz % 4 == 0) && ((reinterpret_cast<uintptr_t>(Z) & 15u) == 0);
    CUtensorMap ma, mb, mb64;
    if constexpr (RB == 128) {
        std::memcpy(&ma, TOUT ? t->tmap_atw : t->tmap_aw, sizeof ma);
        std::memcpy(&mb, TOUT ? t->tmap_bt2w : t->tmap_b2w, sizeof mb);
        std::memcpy(&mb64, TOUT ? t->tmap_bt3w : t->tmap_b3w, sizeof mb64);
    } else {
        std::memcpy(&ma, TOUT ? t->tmap_at : t->tmap_a, sizeof ma);
        std::memcpy(&mb, TOUT ? t->tmap_bt2 : t->tmap_b2, sizeof mb);
        std::memcpy(&mb64, TOUT ? t->tmap_bt3 : t->tmap_b3, sizeof mb64);
    }
    // A last round with at most half as many tiles as pairs is run as
    // 256 x 128 halves.
    const int rem = tiles % clusters;
    const int split = (rem > 0 && 2 * rem <= clusters) ? 2 : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)Cfg::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    main_kernel_begin(st);
    AFMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_pair_kernel<SA, TOUT, MODE, SUB, RB>, ma, mb, mb64, Z,
                                     ldz, m0, m1, n0, n1, n, vec, split, status,
                                     (const uint32_t*)t->amax));
    main_kernel_end(st, 2 * clusters);
    count_launches(1);
    return AFMM_OK;
}

// Pair-kernel stage layout (read once from the environment): one K block
// of 128-byte operand rows per stage (default), or with AFMM_TC_ROW=64
// 64-byte rows, two K blocks per stage (AFMM_TC_KSUB=1: one).  Measured at
// n = 8192 / 16384 with 64-byte rows, two blocks per stage against one:
// split BF16 kernel 1.54 against 1.55 ms, FP16 two slices 1.07 against
// 1.11 ms, E4M3 digits 4.26 against 4.39 ms; three blocks (the two-slice
// forms, three 72 KiB stages) 1-2% slower than two.
inline int pair_layout() {
    static const int v = [] {
        const char* r = std::getenv("AFMM_TC_ROW");
        if (!(r && std::atoi(r) == 64)) return 128;
        const char* e = std::getenv("AFMM_TC_KSUB");
        return e && std::atoi(e) == 1 ? 1 : 2;
    }();
    return v;
}

template <int SA, bool TOUT = false, int MODE = PM_SPLIT>
afmm_status launch_tc_pair(const TcPlan* t, float* Z, int64_t ldz, int* status,
                           cudaStream_t st, int m0 = 0, int m1 = -1, int n0 = 0, int n1 = -1) {
    switch (pair_layout()) {
        case 128:
            return launch_tc_pair_sub<SA, TOUT, MODE, 1, 128>(t, Z, ldz, status, st, m0, m1,
                                                              n0, n1);
        case 2:
            return launch_tc_pair_sub<SA, TOUT, MODE, 2, 64>(t, Z, ldz, status, st, m0, m1, n0,
                                                             n1);
        default:
            return launch_tc_pair_sub<SA, TOUT, MODE, 1, 64>(t, Z, ldz, status, st, m0, m1, n0,
                                                             n1);
    }
}

// The split product with S = t->slices BF16 slices: the two-SM kernel when
// the plan chose it (t->pair), else the one-CTA kernel.
template <bool TOUT>
afmm_status split_product(const TcPlan* t, float* Z, int64_t ldz, int* status,
                          cudaStream_t st, int m0 = 0, int m1 = -1, int n0 = 0, int n1 = -1) {
    if (t->h16) {
        // FP16 two-slice form (Case A).
        if (t->pair) {
            const afmm_status rc =
                launch_tc_pair<2, TOUT, PM_H16>(t, Z, ldz, status, st, m0, m1, n0, n1);
            if (rc != AFMM_ERR_UNSUPPORTED) return rc;
        }
        return launch_tc<2, 1, TOUT, false, true>(t, Z, ldz, status, st, m0, m1, n0, n1);
    }
    if (t->pair) {
        const afmm_status rc =
            t->slices == 3 ? launch_tc_pair<3, TOUT>(t, Z, ldz, status, st, m0, m1, n0, n1)
                           : launch_tc_pair<2, TOUT>(t, Z, ldz, status, st, m0, m1, n0, n1);
        if (rc != AFMM_ERR_UNSUPPORTED) return rc;
    }
    return t->slices == 3 ? launch_tc<3, 1, TOUT>(t, Z, ldz, status, st, m0, m1, n0, n1)
                          : launch_tc<2, 1, TOUT>(t, Z, ldz, status, st, m0, m1, n0, n1);
}

afmm_status launch_exact2(const TcPlan* t, void* Z, int64_t ldz, int kb_per_chunk,
                          int* status, cudaStream_t st) {
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    const int n = (int)t->n;
    const int tiles = ((n + X2_BM - 1) / X2_BM) * ((n + X2_BN - 1) / X2_BN);
    const int grid = tiles < dp.sm_count ? tiles : dp.sm_count;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(tc_exact2_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, X2_SMEM));
    const int vec = (ldz % 4 == 0) && ((reinterpret_cast<uintptr_t>(Z) & 15u) == 0);
    CUtensorMap ma, mb;
    std::memcpy(&ma, t->tmap_a, sizeof ma);
    std::memcpy(&mb, t->tmap_b, sizeof mb);
    main_kernel_begin(st);
    tc_exact2_kernel<<<grid, TC_THREADS, X2_SMEM, st>>>(ma, mb, static_cast<int32_t*>(Z), ldz,
                                                         n, n, n, kb_per_chunk, vec, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, grid);
    count_launches(1);
    return AFMM_OK;
}

// One thread waits on a barrier that is never completed; the bounded wait
// must give up and record AFMM_ERR_TIMEOUT.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int* status) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        abort = 0;
        ptx::fence_barrier_init();
        if (!ptx::mbar_wait_bounded(&bar, 0u, &abort, limit_ns))
            atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
    }
}

}  // namespace

afmm_status tc_selftest_bounded_wait(uint64_t limit_ns, cudaStream_t st) {
    if (limit_ns > WAIT_LIMIT_NS) limit_ns = WAIT_LIMIT_NS;
    int* d = nullptr;
    AFMM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(int), st));
    afmm_status rc = AFMM_OK;
    int h = 0;
    if (cudaMemsetAsync(d, 0, sizeof(int), st) != cudaSuccess) rc = AFMM_ERR_CUDA;
    if (rc == AFMM_OK) {
        bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, d);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = AFMM_ERR_CUDA;
    }
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
    return rc != AFMM_OK ? rc : static_cast<afmm_status>(h);
}

bool tc_available() {
    DeviceProps dp;
    if (device_props(&dp) != AFMM_OK) return false;
    return dp.cc_major == 10 && dp.cc_minor == 3 && dp.smem_optin >= (size_t)SMEM_OPTIN;
}

int tc_exact_chunk_k(double amax, double bmax) {
    const double per = (amax < 1.0 ? 1.0 : amax) * (bmax < 1.0 ? 1.0 : bmax);
    const double k = std::floor(16777215.0 / per);
    return (int)(std::floor(k / TC_BK) * TC_BK);
}

namespace {
double dtype_bound(int dt) {
    switch (dt) {
        case AFMM_I8: return 128.0;
        case AFMM_U8: return 255.0;
        default: return 256.0;      // BF16-exact integers checked on device
    }
}
}  // namespace

void tc_layout(TcPlan* t, const afmm_desc& d, int slices, bool f8, bool h16, bool x8) {
    t->n = d.n;
    t->slices = slices;
    t->sliced_a = d.kase != AFMM_CASE_B;
    t->both = d.kase == AFMM_CASE_REAL;
    t->f8 = f8;
    t->h16 = h16;
    t->x8 = x8;
    if (x8) {
        // One byte per element: 16-byte aligned rows; two digit slices of
        // the integer Base factor (the a buffer in Case A, b in Case B),
        // one Rep-factor operand; the two-SM kernel.
        t->ld_a = t->ld_b = (d.n + 15) / 16 * 16;
        t->rows_a = t->rows_b = d.n;
        t->a_bytes = (size_t)(t->sliced_a ? 2 : 1) * d.n * t->ld_a;
        t->b_bytes = (size_t)(t->sliced_a ? 1 : 2) * d.n * t->ld_b;
        t->pair = true;
        return;
    }
    t->ld_a = t->ld_b = (d.n + 7) / 8 * 8;
    if (f8) {
        // E4M3 operands: 16-byte aligned rows of one-byte elements; the
        // row maxima of the sliced operand.
        t->ld_a = t->ld_b = (d.n + 15) / 16 * 16;
        t->chunk_kb = kF8ChunkKb;
        if (const char* e = std::getenv("AFMM_TC_CHUNK_KB")) t->chunk_kb = std::atoi(e);
        const int sa = t->sliced_a ? slices : 1, sb = t->sliced_a ? 1 : slices;
        t->rows_a = t->rows_b = d.n;
        t->a_bytes = (size_t)sa * d.n * t->ld_a;
        t->b_bytes = (size_t)sb * d.n * t->ld_b;
        t->s_bytes = (size_t)d.n * sizeof(uint32_t);
        const int64_t ldz = d.ldz ? d.ldz : d.n;
        if (t->sliced_a && ldz % 4 != 0) {
            t->ld_z = (d.n + 3) / 4 * 4;
            t->z_bytes = (size_t)d.n * t->ld_z * 4;
        }
        return;
    }
    if (slices == 0) {
        // Exact form: A = X, B = Y^T, one BF16 operand each.
        const int rep_dt = d.kase == AFMM_CASE_A ? d.y_dtype : d.x_dtype;
        const int base_dt = d.kase == AFMM_CASE_A ? d.x_dtype : d.y_dtype;
        double rb = dtype_bound(rep_dt), bb = dtype_bound(base_dt);
        if (d.rep_max >= 0.0 && d.rep_max < rb) rb = d.rep_max;
        if (d.base_max >= 0.0 && d.base_max < bb) bb = d.base_max;
        const double amax = d.kase == AFMM_CASE_A ? bb : rb;
        const double bmax = d.kase == AFMM_CASE_A ? rb : bb;
        t->lim_a = (float)amax;
        t->lim_b = (float)bmax;
        t->kb_per_chunk = tc_exact_chunk_k(amax, bmax) / TC_BK;
        t->a_bytes = (size_t)d.n * t->ld_a * 2;
        t->b_bytes = (size_t)d.n * t->ld_b * 2;
        return;
    }
    const int sa = t->sliced_a ? slices : 1, sb = t->sliced_a && !t->both ? 1 : slices;
    // The two-SM kernel for the one-sided split form from n = 512 up (a
    // pair tile is 256 x 256); AFMM_TC_PAIR=0 in the environment keeps the
    // one-CTA kernel.
    t->pair = !t->both && d.n >= 512;
    if (const char* e = std::getenv("AFMM_TC_PAIR")) t->pair = t->pair && std::atoi(e) != 0;
    if (t->both) {
        t->chunk_kb = kRealChunkKb;
        if (const char* e = std::getenv("AFMM_TC_CHUNK_KB")) t->chunk_kb = std::atoi(e);
    }
    t->rows_a = d.n;
    t->rows_b = d.n;
    t->a_bytes = (size_t)sa * d.n * t->ld_a * 2;
    t->b_bytes = (size_t)sb * d.n * t->ld_b * 2;
    if (h16) t->s_bytes = (size_t)d.n * sizeof(uint32_t);    // row maxima of X
    const int64_t ldz = d.ldz ? d.ldz : d.n;
    if (t->sliced_a && ldz % 4 != 0) {
        t->ld_z = (d.n + 3) / 4 * 4;
        t->z_bytes = (size_t)d.n * t->ld_z * 4;
    }
}

afmm_status tc_bind_workspace(TcPlan* t, void* a, void* b, void* z, void* s) {
    t->a = a;
    t->b = b;
    t->z = t->z_bytes ? z : nullptr;
    t->amax = t->s_bytes ? static_cast<uint32_t*>(s) : nullptr;
    t->maps_ready = false;
    if (t->n <= 0) return AFMM_OK;
    const int sl = t->slices > 0 ? t->slices : 1;
    const int sa = t->sliced_a ? sl : 1, sb = t->sliced_a && !t->both ? 1 : sl;
    const int es = (t->f8 || t->x8) ? 1 : 2;
    AFMM_TRY(tc_encode_map(t->tmap_a, a, t->n, t->n, t->ld_a, sa, TC_BM, es));
    AFMM_TRY(tc_encode_map(t->tmap_b, b, t->n, t->n, t->ld_b, sb, TC_BN, es));
    // B side with 128-row boxes: each CTA of a pair loads half of a B tile.
    AFMM_TRY(tc_encode_map(t->tmap_b2, b, t->n, t->n, t->ld_b, sb, PR_HALF, es));
    AFMM_TRY(tc_encode_map(t->tmap_b3, b, t->n, t->n, t->ld_b, sb, PR_HALF / 2, es));
    const bool caseb = !t->sliced_a && t->slices > 0;
    if (caseb) {
        // Case B as Z^T = Y^T X^T: the sliced Y^T rows are the A side.
        AFMM_TRY(tc_encode_map(t->tmap_at, b, t->n, t->n, t->ld_b, sb, TC_BM, es));
        AFMM_TRY(tc_encode_map(t->tmap_bt, a, t->n, t->n, t->ld_a, sa, TC_BN, es));
        AFMM_TRY(tc_encode_map(t->tmap_bt2, a, t->n, t->n, t->ld_a, sa, PR_HALF, es));
        AFMM_TRY(tc_encode_map(t->tmap_bt3, a, t->n, t->n, t->ld_a, sa, PR_HALF / 2, es));
    }
    if (t->pair) {
        // The same maps with 128-byte rows for the pair kernel.
        AFMM_TRY(tc_encode_map(t->tmap_aw, a, t->n, t->n, t->ld_a, sa, PR_HALF, es, 128));
        AFMM_TRY(tc_encode_map(t->tmap_b2w, b, t->n, t->n, t->ld_b, sb, PR_HALF, es, 128));
        AFMM_TRY(tc_encode_map(t->tmap_b3w, b, t->n, t->n, t->ld_b, sb, PR_HALF / 2, es, 128));
        if (caseb) {
            AFMM_TRY(tc_encode_map(t->tmap_atw, b, t->n, t->n, t->ld_b, sb, PR_HALF, es, 128));
            AFMM_TRY(tc_encode_map(t->tmap_bt2w, a, t->n, t->n, t->ld_a, sa, PR_HALF, es, 128));
            AFMM_TRY(
                tc_encode_map(t->tmap_bt3w, a, t->n, t->n, t->ld_a, sa, PR_HALF / 2, es, 128));
        }
    }
    t->maps_ready = true;
    return AFMM_OK;
}

afmm_status tc_run_split(TcPlan* t, const afmm_desc& d, const void* X,
                         const void* Y, void* Z, int* status, cudaStream_t st) {
    if (!t->maps_ready) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d.n;
    auto* A = static_cast<__nv_bfloat16*>(t->a);
    auto* B = static_cast<__nv_bfloat16*>(t->b);
    float* Zf = static_cast<float*>(Z);
    if (d.kase == AFMM_CASE_A && t->slices == 3 && tc_fused_usable(d, X)) {
        // B = Rep-factors Y transposed; X is split inside the product kernel.
        AFMM_TRY((tc_widen_transpose(1, true, Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                  256.f, status, st, true)));
        return tc_run_fused_caseA(t, d, X, Z, status, st);
    }
    if (d.kase == AFMM_CASE_A) {
        // A = slices of the real X (rows), B = Rep-factors Y transposed.
        if (t->slices == 3)
            AFMM_TRY((tc_widen_rows(3, false, X, d.x_dtype, n, d.ldx, A, t->ld_a,
                                                  0.f, status, st)));
        else
            AFMM_TRY((tc_widen_rows(2, false, X, d.x_dtype, n, d.ldx, A, t->ld_a,
                                                  0.f, status, st)));
        AFMM_TRY((tc_widen_transpose(1, true, Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                  256.f, status, st, true)));
        if (t->z) {
            // Rows of Z off 16-byte boundaries: product into the aligned
            // buffer, then one 2-D copy.
            float* zt = static_cast<float*>(t->z);
            AFMM_TRY((split_product<false>(t, zt, t->ld_z, status, st)));
            AFMM_CUDA_TRY(cudaMemcpy2DAsync(Zf, d.ldz * sizeof(float), zt,
                                            t->ld_z * sizeof(float), n * sizeof(float), n,
                                            cudaMemcpyDeviceToDevice, st));
            return AFMM_OK;
        }
        return split_product<false>(t, Zf, d.ldz, status, st);
    }
    // Case B: A = Rep-factors X (rows), B = slices of the real Y transposed.
    AFMM_TRY((tc_widen_rows(1, true, X, d.x_dtype, n, d.ldx, A, t->ld_a, 256.f,
                                         status, st, 0, -1, true)));
    if (t->slices == 3)
        AFMM_TRY((tc_widen_transpose(3, false, Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                   0.f, status, st)));
    else
        AFMM_TRY((tc_widen_transpose(2, false, Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                   0.f, status, st)));
    // Computed as Z^T = Y^T X^T: the slices on the A side, as in Case A, so
    // a stage holds S + 1 tiles of 8 + 16 KiB instead of 1 + S of 8 + 16 x S.
    return split_product<true>(t, Zf, d.ldz, status, st);
}

afmm_status tc_run_real(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                        void* Z, int* status, cudaStream_t st) {
    if (!t->maps_ready || !t->both) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d.n;
    float* Zf = static_cast<float*>(Z);
    // A = three slices of X (rows), B = three slices of Y transposed.
    AFMM_TRY((tc_widen_rows(3, false, X, d.x_dtype, n, d.ldx, t->a, t->ld_a, 0.f, status,
                            st)));
    AFMM_TRY((tc_widen_transpose(3, false, Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, 0.f,
                                 status, st)));
    if (t->z) {
        float* zt = static_cast<float*>(t->z);
        AFMM_TRY((launch_tc<3, 3>(t, zt, t->ld_z, status, st)));
        AFMM_CUDA_TRY(cudaMemcpy2DAsync(Zf, d.ldz * sizeof(float), zt,
                                        t->ld_z * sizeof(float), n * sizeof(float), n,
                                        cudaMemcpyDeviceToDevice, st));
        return AFMM_OK;
    }
    return launch_tc<3, 3>(t, Zf, d.ldz, status, st);
}

afmm_status tc_run_fp8(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                       void* Z, int* status, cudaStream_t st) {
    if (!t->maps_ready || !t->f8) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d.n;
    float* Zf = static_cast<float*>(Z);
    if (d.kase == AFMM_CASE_A) {
        // A = four slices of the real X (rows), B = Rep-factors Y transposed.
        AFMM_TRY(tc_f8_rows(false, X, d.x_dtype, n, d.ldx, t->a, t->ld_a, t->amax, status, st));
        AFMM_TRY(tc_f8_transpose(true, Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, t->amax, status,
                                 st));
        if (t->z) {
            float* zt = static_cast<float*>(t->z);
            AFMM_TRY((launch_tc<4, 1, false, true>(t, zt, t->ld_z, status, st)));
            AFMM_CUDA_TRY(cudaMemcpy2DAsync(Zf, d.ldz * sizeof(float), zt,
                                            t->ld_z * sizeof(float), n * sizeof(float), n,
                                            cudaMemcpyDeviceToDevice, st));
            return AFMM_OK;
        }
        return launch_tc<4, 1, false, true>(t, Zf, d.ldz, status, st);
    }
    // Case B as Z^T = Y^T X^T: A = four slices of Y^T (Y's columns), B = X.
    AFMM_TRY(tc_f8_rows(true, X, d.x_dtype, n, d.ldx, t->a, t->ld_a, t->amax, status, st));
    AFMM_TRY(tc_f8_transpose(false, Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, t->amax, status,
                             st));
    return launch_tc<4, 1, true, true>(t, Zf, d.ldz, status, st);
}

afmm_status tc_run_h16(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                       void* Z, int* status, cudaStream_t st) {
    if (!t->maps_ready || !t->h16) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d.n;
    float* Zf = static_cast<float*>(Z);
    if (d.kase == AFMM_CASE_B) {
        // As Z^T = Y^T X^T: A = two column-scaled FP16 slices of Y^T (the
        // b buffer), B = the Rep-factors X as FP16 rows.
        AFMM_TRY(tc_h16_rep_rows(X, d.x_dtype, n, d.ldx, t->a, t->ld_a, 2048.f, status, st));
        AFMM_TRY(tc_h16_transpose(Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, t->amax, status, st));
        return split_product<true>(t, Zf, d.ldz, status, st);
    }
    // A = two row-scaled FP16 slices of X, B = Rep-factors Y transposed,
    // FP16, exact up to 2048.
    AFMM_TRY(tc_h16_rows(X, d.x_dtype, n, d.ldx, t->a, t->ld_a, t->amax, status, st));
    AFMM_TRY(tc_widen_transpose_h16(Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, 2048.f, status, st,
                                    true));
    if (t->z) {
        float* zt = static_cast<float*>(t->z);
        AFMM_TRY((split_product<false>(t, zt, t->ld_z, status, st)));
        AFMM_CUDA_TRY(cudaMemcpy2DAsync(Zf, d.ldz * sizeof(float), zt,
                                        t->ld_z * sizeof(float), n * sizeof(float), n,
                                        cudaMemcpyDeviceToDevice, st));
        return AFMM_OK;
    }
    return split_product<false>(t, Zf, d.ldz, status, st);
}

afmm_status tc_run_exact_x8(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                            void* Z, int* status, cudaStream_t st) {
    if (!t->maps_ready || !t->x8) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d.n;
    if (d.kase == AFMM_CASE_B) {
        // A = two digit slices of Y^T (the b buffer), B = X's Rep-factors;
        // tiles of Z^T, stored transposed.
        AFMM_TRY(tc_x8_rep_rows(X, d.x_dtype, n, d.ldx, t->a, t->ld_a, status, st));
        AFMM_TRY(tc_x8_digit_transpose(Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, status, st));
        return launch_tc_pair<2, true, PM_X8>(t, static_cast<float*>(Z), d.ldz, status, st);
    }
    AFMM_TRY(tc_x8_digit_rows(X, d.x_dtype, n, d.ldx, t->a, t->ld_a, status, st));
    AFMM_TRY(tc_x8_rep_transpose(Y, d.y_dtype, n, d.ldy, t->b, t->ld_b, status, st));
    // The kernel writes int32 bit patterns through its float pointer.
    return launch_tc_pair<2, false, PM_X8>(t, static_cast<float*>(Z), d.ldz, status, st);
}

afmm_status tc_run_exact(TcPlan* t, const afmm_desc& d, const void* X,
                         const void* Y, void* Z, int* status, cudaStream_t st) {
    if (!t->maps_ready) return AFMM_ERR_INVALID_ARG;
    if (t->kb_per_chunk < 1) return AFMM_ERR_OVERFLOW_RISK;
    const int64_t n = d.n;
    auto* A = static_cast<__nv_bfloat16*>(t->a);
    auto* B = static_cast<__nv_bfloat16*>(t->b);
    AFMM_TRY((tc_widen_rows(1, true, X, d.x_dtype, n, d.ldx, A, t->ld_a, t->lim_a,
                                         status, st, 0, -1, d.kase == AFMM_CASE_B)));
    AFMM_TRY((tc_widen_transpose(1, true, Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                              t->lim_b, status, st, d.kase == AFMM_CASE_A)));
    return launch_exact2(t, Z, d.ldz, t->kb_per_chunk, status, st);
}

afmm_status tc_split_prepare_b(TcPlan* t, const afmm_desc& d, const void* Y, int* status,
                               cudaStream_t st) {
    if (!t->maps_ready) return AFMM_ERR_INVALID_ARG;
    const int sl = t->slices;
    if (t->f8)
        return tc_f8_transpose(d.kase == AFMM_CASE_A, Y, d.y_dtype, d.n, d.ldy, t->b, t->ld_b,
                               t->amax, status, st);
    if (d.kase == AFMM_CASE_A)        // B = Rep-factors Y transposed
        return tc_widen_transpose(1, true, Y, d.y_dtype, d.n, d.ldy, t->b, t->ld_b, 256.f,
                                  status, st, true);
    return tc_widen_transpose(sl, false, Y, d.y_dtype, d.n, d.ldy, t->b, t->ld_b, 0.f,
                              status, st);
}

afmm_status tc_split_convert_rows(TcPlan* t, const afmm_desc& d, const void* X, int64_t r0,
                                  int64_t r1, int* status, cudaStream_t st) {
    if (!t->maps_ready) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d.n;
    if (t->f8)
        return tc_f8_rows(d.kase == AFMM_CASE_B, X, d.x_dtype, n, d.ldx, t->a, t->ld_a,
                          t->amax, status, st, r0, r1);
    if (d.kase == AFMM_CASE_A)
        return tc_widen_rows(t->slices, false, X, d.x_dtype, n, d.ldx, t->a, t->ld_a, 0.f,
                             status, st, r0, r1);
    return tc_widen_rows(1, true, X, d.x_dtype, n, d.ldx, t->a, t->ld_a, 256.f, status, st,
                         r0, r1, true);
}

afmm_status tc_split_product_rows(TcPlan* t, const afmm_desc& d, void* Z, int64_t r0,
                                  int64_t r1, int* status, cudaStream_t st) {
    if (!t->maps_ready) return AFMM_ERR_INVALID_ARG;
    const int m0 = (int)r0, m1 = (int)r1;
    float* Zf = static_cast<float*>(Z);
    if (t->f8)
        return d.kase == AFMM_CASE_A
                   ? launch_tc<4, 1, false, true>(t, Zf, d.ldz, status, st, m0, m1)
                   : launch_tc<4, 1, true, true>(t, Zf, d.ldz, status, st, 0, -1, m0, m1);
    if (d.kase == AFMM_CASE_A) return split_product<false>(t, Zf, d.ldz, status, st, m0, m1);
    // Case B (Z^T = Y^T X^T): rows [r0, r1) of Z are columns of the product.
    return split_product<true>(t, Zf, d.ldz, status, st, 0, -1, m0, m1);
}

afmm_status tc_split_rows(TcPlan* t, const afmm_desc& d, const void* X, void* Z,
                          int64_t r0, int64_t r1, int* status, cudaStream_t st) {
    AFMM_TRY(tc_split_convert_rows(t, d, X, r0, r1, status, st));
    return tc_split_product_rows(t, d, Z, r0, r1, status, st);
}

int tc_pipe_blocks(int64_t n, int sms, int64_t* bounds, int max_blocks, bool caseb,
                   bool pair) {
    // Tile extent along Z's rows and tiles per tile row of the kernel that
    // multiplies the blocks; `sms` becomes the number of CTA pairs when the
    // two-SM kernel (256 x 256 tiles on pairs of SMs) runs them.
    const int64_t unit_rows = pair ? PR_BM : (caseb ? TC_BN : TC_BM);
    const int64_t tm = (n + unit_rows - 1) / unit_rows,
                  tn = pair ? (n + PR_BN - 1) / PR_BN
                            : (caseb ? (n + TC_BM - 1) / TC_BM : (n + TC_BN - 1) / TC_BN);
    if (pair) sms = std::max(1, sms / 2);
    // First and last blocks of about one wave of tiles: the first product
    // starts after Y and a small piece of X have arrived, and the last
    // block's product and copy-out are short.  Middle blocks fill whole
    // waves where they can.
    const int64_t edge = std::max<int64_t>(1, sms / tn);
    const int64_t mid = tm - 2 * edge;
    if (mid < 1 || max_blocks < 3)
        return tc_row_blocks(n, pair ? 2 * sms : sms, bounds, max_blocks, caseb, pair);
    int64_t g = sms, b = tn;
    while (b) { const int64_t r = g % b; g = b; b = r; }
    int64_t unit = std::max<int64_t>(1, sms / g);        // tile rows of whole waves
    if (pair) {
        // Smaller middle blocks whose tiles come to nearly whole rounds (at
        // least 95% of their last round busy): a block's rows arrive in a
        // fraction of its product time, so the products, not the copies,
        // set the pace.  (At n = 8192: 7 bands, 224 tiles, 2.95 rounds of
        // 76 pairs, against 19 bands for exactly whole rounds.)
        for (int64_t k = 2; 4 * k <= mid && k < unit; ++k) {
            const int64_t tiles = k * tn;
            const int64_t rounds = (tiles + sms - 1) / sms;
            if (20 * tiles >= 19 * rounds * sms) {
                unit = k;
                break;
            }
        }
    }
    while (mid / unit + (mid % unit ? 1 : 0) > max_blocks - 2) unit *= 2;
    int k = 0;
    bounds[k++] = 0;
    int64_t r = edge;
    bounds[k++] = r * unit_rows;
    for (int64_t left = mid; left > 0;) {                // whole-wave blocks, then the rest
        const int64_t take = std::min(unit, left);
        r += take;
        left -= take;
        bounds[k++] = std::min<int64_t>(r * unit_rows, n);
    }
    bounds[k] = n;
    return k;                                            // number of blocks
}

int tc_row_blocks(int64_t n, int sms, int64_t* bounds, int max_blocks, bool caseb,
                  bool pair) {
    // Rows of Z are product rows (tiles of TC_BM) in Case A and product
    // columns (tiles of TC_BN) in Case B; pair tiles are 256 x 256 on
    // sms / 2 pairs.
    const int64_t unit_rows = pair ? PR_BM : (caseb ? TC_BN : TC_BM);
    const int64_t tm = (n + unit_rows - 1) / unit_rows,
                  tn = pair ? (n + PR_BN - 1) / PR_BN
                            : (caseb ? (n + TC_BM - 1) / TC_BM : (n + TC_BN - 1) / TC_BN);
    if (pair) sms = std::max(1, sms / 2);
    // Smallest number of tile rows whose tiles fill whole waves.
    int64_t g = sms, b = tn;
    while (b) { const int64_t r = g % b; g = b; b = r; }
    int64_t unit = sms / g;
    if (unit < 1) unit = 1;
    int64_t per = unit * std::max<int64_t>(1, (tm / 4 + unit / 2) / unit);
    if (per >= tm) per = (tm + 1) / 2;                   // at least two blocks
    int k = 0;
    bounds[k++] = 0;
    for (int64_t r = per; r < tm && k < max_blocks; r += per) bounds[k++] = r * unit_rows;
    bounds[k] = n;
    return k;                                            // number of blocks
}

}  // namespace afmm
