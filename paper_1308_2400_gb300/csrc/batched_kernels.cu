// Batched AFMM products: many independent instances (Sec. 2 problems of
// different n, Case A or B) in one call.
//
// Per batch signature (the array of descriptors) the library builds once:
//  - a route per instance: the tcgen05 split-BF16 form or the CUDA-core
//    zero-skip form (desc.variant when forced, else the planner's rule);
//  - operand buffers for all instances in one workspace, with two TMA
//    descriptors per tensor-core instance kept in device memory;
//  - per-CTA tile lists for one persistent grouped tensor-core launch,
//    balanced by longest-processing-time-first over 128 x 256 tiles
//    (a tile's cost is its number of 32-wide K steps);
//  - a CUDA graph: grouped conversions -> grouped tensor-core product, and
//    grouped FP32 widening -> grouped CUDA-core product on a parallel
//    branch.
// Every call copies the instances' X, Y, Z pointers into a device table and
// launches the graph on the caller's stream.  This file holds the kernels
// and their launchers; batched.cpp holds the planning and the graph.
#include <cuda.h>
#include <cuda_bf16.h>

#include "afmm_common.cuh"
#include "batched.cuh"
#include "bf16_split.cuh"
#include "ptx_sm100.cuh"
#include "tc_gemm.cuh"
#include "tile_convert.cuh"

namespace afmm {
namespace {

constexpr int GB_EPI = 256;
constexpr int GB_THREADS = 64 + GB_EPI;
constexpr uint32_t GB_TMEM_COLS = 512;
constexpr int GB_A_TILE = GB_BM * GB_BK * 2;      // 8 KiB
constexpr int GB_B_TILE = GB_BN * GB_BK * 2;      // 16 KiB
// Every tile is computed with the three slices on the A side (Case B as
// Z^T = Y^T X^T), so a stage is 3 A tiles + 1 B tile.
constexpr int GB_STAGE = 3 * GB_A_TILE + GB_B_TILE;
constexpr int GB_STAGES = 4;
constexpr int GB_EPI_SMEM = 8 * 32 * 33 * 4;         // per-warp 32 x 33 floats
constexpr int GB_SMEM = 1024 + GB_STAGES * GB_STAGE + 256 + GB_EPI_SMEM;
constexpr uint64_t GB_WAIT_NS = 2000000000ull;
static_assert(GB_SMEM <= 232448, "shared memory");


struct GBars {
    uint64_t full[GB_STAGES];
    uint64_t empty[GB_STAGES];
    uint64_t tfull, tempty, drain;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ int find_job(const int* prefix, int n, int b) {
    int lo = 0, hi = n - 1;               // last j with prefix[j] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ----------------------------------------------------------- conversions
// The instance's dtype is read once per block and selects a specialised
// body, so the inner loops hold no per-element dtype switch.
#define G_DTYPE_SWITCH(dt, BODY)                                   \
    switch (dt) {                                                  \
        case AFMM_F64: { constexpr int DT = AFMM_F64; BODY; } break;   \
        case AFMM_F32: { constexpr int DT = AFMM_F32; BODY; } break;   \
        case AFMM_BF16: { constexpr int DT = AFMM_BF16; BODY; } break; \
        case AFMM_E4M3: { constexpr int DT = AFMM_E4M3; BODY; } break; \
        case AFMM_I32: { constexpr int DT = AFMM_I32; BODY; } break;   \
        case AFMM_I8: { constexpr int DT = AFMM_I8; BODY; } break;     \
        default: { constexpr int DT = AFMM_U8; BODY; } break;          \
    }

// One row of the A operand: Case A (KIND 0) slices a row of the real X into
// 3 BF16 rows; Case B (KIND 1) widens a row of the Rep-factors X to BF16
// (values must be exact, |v| <= 256, else the instance's flag is set and
// its Z becomes NaN).  Eight columns per thread and step (vector loads when
// the rows are aligned), one 16-byte store per slice; the row's threads are
// t0, t0 + 1, .. (nt of them).
template <int DT, int KIND>
__device__ __forceinline__ void g_row_body(const GInst& g, int64_t r, int* flags, int* status,
                                           int t0, int nt) {
    using T = typename Elem<DT>::T;
    const int64_t n = g.n, ldk = g.ldk;
    const int64_t va = sizeof(T) * 8 < 16 ? sizeof(T) * 8 : 16;
    const bool vec = (reinterpret_cast<uintptr_t>(g.X) % va) == 0 &&
                     (g.ldx * (int64_t)sizeof(T)) % va == 0;
    const T* x = static_cast<const T*>(g.X) + r * g.ldx;
    bool bad = false;
    int bits = 0;
    for (int64_t c = 8 * (int64_t)t0; c < ldk; c += 8 * (int64_t)nt) {
        float v[8];
        // FP32 rows that start off a 16-byte boundary: aligned loads and a shift.
        constexpr bool kF32 = DT == AFMM_F32;
        const bool shifted = kF32 && !vec && (reinterpret_cast<uintptr_t>(g.X) & 15u) == 0 &&
                             c + 12 <= n;
        if (vec && c + 8 <= n) {
            alignas(16) T e[8];
            load8<DT>(x, c, e);
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = value_checked<DT>(e[t], 256.f, bad);
        } else if (shifted) {
            const float* p = reinterpret_cast<const float*>(x) + c;
            load8_f32_shifted(p, (int)((reinterpret_cast<uintptr_t>(p) & 15u) >> 2), v);
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                v[t] = c + t < n ? value_checked<DT>(x[c + t], 256.f, bad) : 0.f;
        }
        if constexpr (KIND == 0) {
            uint32_t w[3][4];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                __nv_bfloat16 o0[3], o1[3];
                split_bf16<3>(v[t], o0);
                split_bf16<3>(v[t + 1], o1);
#pragma unroll
                for (int s = 0; s < 3; ++s) w[s][t / 2] = pack2(o0[s], o1[s]);
            }
#pragma unroll
            for (int s = 0; s < 3; ++s)
                *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(g.A) +
                                          ((int64_t)s * n + r) * ldk + c) =
                    make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
        } else {
            uint32_t w[4];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                bits |= rep_bits(v[t]) | rep_bits(v[t + 1]);
                const __nv_bfloat16 b0 = __float2bfloat16_rn(v[t]);
                const __nv_bfloat16 b1 = __float2bfloat16_rn(v[t + 1]);
                bad |= __bfloat162float(b0) != v[t] || __bfloat162float(b1) != v[t + 1] ||
                       fabsf(v[t]) > 256.f || fabsf(v[t + 1]) > 256.f;
                w[t / 2] = pack2(b0, b1);
            }
            *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(g.A) + r * ldk + c) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    if (KIND == 1 && bad) bits |= kBadRange;
    if (KIND == 1 && bits) {
        atomicExch(&flags[g.flag], 1);
        atomicCAS(status, 0, bad_status(bits));
    }
}

// Warp w of block b converts row q = 8 b + w (of all instances' A rows in
// order): row q - row_prefix[j] of instance j = row_job[q].  A warp per row
// keeps eight rows' loads in flight per block (instances' rows are short:
// n <= 2048).
constexpr int G_ROWS_PER_BLOCK = 8;
__global__ void __launch_bounds__(32 * G_ROWS_PER_BLOCK)
g_rows_kernel(const GInst* __restrict__ inst, const int* __restrict__ row_prefix,
              const int* __restrict__ row_job, int rows_total, int* __restrict__ flags,
              int* __restrict__ status) {
    const int q = blockIdx.x * G_ROWS_PER_BLOCK + (threadIdx.x >> 5);
    if (q >= rows_total) return;
    const int lane = threadIdx.x & 31;
    const int j = row_job[q];
    const GInst& g = inst[j];
    const int64_t r = q - row_prefix[j];
    if (g.kind == 0) {
        G_DTYPE_SWITCH(g.x_dtype, (g_row_body<DT, 0>(g, r, flags, status, lane, 32)))
    } else {
        G_DTYPE_SWITCH(g.x_dtype, (g_row_body<DT, 1>(g, r, flags, status, lane, 32)))
    }
}

// The byte-tile path of g_transpose_kernel, kept out of line so that its
// registers are allocated apart from the FP32-tile paths.
__device__ __noinline__ int g_transpose_bytes(const GInst& g, int64_t r0, int64_t c0,
                                              uint8_t (*bt)[64], uint32_t* lut) {
    auto* B = static_cast<__nv_bfloat16*>(g.B);
    const bool vec = rows_aligned16(g.Y, g.ldy, 1);
    switch (g.y_dtype) {
        case AFMM_E4M3:
            return tile_bytes_transpose_convert<AFMM_E4M3, 1, true, false, GB_U8_ROWS>(
                g.Y, g.n, g.ldy, r0, c0, B, g.ldk, 256.f, vec, bt, true, lut);
        case AFMM_I8:
            return tile_bytes_transpose_convert<AFMM_I8, 1, true, false, GB_U8_ROWS>(
                g.Y, g.n, g.ldy, r0, c0, B, g.ldk, 256.f, vec, bt, true, lut);
        default:
            return tile_bytes_transpose_convert<AFMM_U8, 1, true, false, GB_U8_ROWS>(
                g.Y, g.n, g.ldy, r0, c0, B, g.ldk, 256.f, vec, bt, true, lut);
    }
}

// Block b converts one tile of the B operand (Y transposed to K-major) of
// instance j = tt_job[b]: Case A widens the Rep-factors Y (exact
// non-negative integers, |v| <= 256), one-byte ones in GB_U8_ROWS x 64 byte
// tiles through a per-block table of the 256 codes
// (tile_bytes_transpose_convert), others in 64 x 64 FP32 tiles; Case B
// splits the real Y into 3 slices (64 x 64 FP32 tiles).
__global__ void __launch_bounds__(256, 6)
g_transpose_kernel(const GInst* __restrict__ inst, const int* __restrict__ tt_prefix,
                   const int* __restrict__ tt_job, int* __restrict__ flags,
                   int* __restrict__ status) {
    // The FP32 tile; a byte tile and its code table reuse its first 9 KiB.
    __shared__ alignas(16) float tile[64][65];
    static_assert(GB_U8_ROWS * 64 + 256 * 4 <= 64 * 65 * 4, "byte tile fits");
    const int j = tt_job[blockIdx.x];
    const GInst& g = inst[j];
    const int64_t n = g.n;
    const int64_t tpr = (n + 63) / 64;
    const int64_t t = blockIdx.x - tt_prefix[j];
    auto* B = static_cast<__nv_bfloat16*>(g.B);
    int bits = 0;
    const bool byte_rep =
        g.y_dtype == AFMM_E4M3 || g.y_dtype == AFMM_I8 || g.y_dtype == AFMM_U8;
    if (g.kind == 0 && byte_rep) {
        const int64_t r0 = (t / tpr) * GB_U8_ROWS, c0 = (t % tpr) * 64;
        bits = g_transpose_bytes(g, r0, c0, reinterpret_cast<uint8_t(*)[64]>(&tile[0][0]),
                                 reinterpret_cast<uint32_t*>(&tile[0][0]) + GB_U8_ROWS * 64 / 4);
    } else if (g.kind == 0) {
        const int64_t r0 = (t / tpr) * 64, c0 = (t % tpr) * 64;
        G_DTYPE_SWITCH(g.y_dtype, (bits = tile_transpose_convert<DT, 1, true>(
                                       g.Y, n, g.ldy, r0, c0, B, g.ldk, 256.f,
                                       rows_aligned16(g.Y, g.ldy, sizeof(typename Elem<DT>::T)),
                                       tile, true)))
    } else {
        const int64_t r0 = (t / tpr) * 64, c0 = (t % tpr) * 64;
        G_DTYPE_SWITCH(g.y_dtype, (tile_transpose_convert<DT, 3, false>(
                                       g.Y, n, g.ldy, r0, c0, B, g.ldk, 0.f,
                                       rows_aligned16(g.Y, g.ldy, sizeof(typename Elem<DT>::T)),
                                       tile)))
    }
    if (bits) {
        atomicExch(&flags[g.flag], 1);
        atomicCAS(status, 0, bad_status(bits));
    }
}

// Block b widens one row of one operand to FP32 for the CUDA-core form;
// a Rep-factor operand (w.rep) is checked on the way (non-negative
// integers, else the batch status records the error), and a job without a
// destination (an FP32 Rep-factor operand the kernel reads in place) is
// only checked.
__global__ void __launch_bounds__(256)
g_widen_kernel(const WJob* __restrict__ jobs, const int* __restrict__ prefix, int njobs,
               int* __restrict__ status) {
    const int j = find_job(prefix, njobs, blockIdx.x);
    const WJob& w = jobs[j];
    const int64_t r = blockIdx.x - prefix[j];
    int bits = 0;
    for (int64_t c = threadIdx.x; c < w.n; c += 256) {
        const float v = load_any_f(w.src, r * w.lds + c, w.dtype);
        if (w.rep) bits |= rep_bits(v);
        if (w.dst) w.dst[r * w.n + c] = v;
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits) atomicCAS(status, 0, bad_status(bits));
}

// ----------------------------------------------------------- grouped TC
// Persistent: CTA b runs tiles[cta_off[b] .. cta_off[b+1]) in order; a tile
// is (instance, tm, tn), 128 x bn with the instance's tile width bn: 256, or
// 128 for the narrow-tile route (128 x 128 x 16 MMAs, a 128-row B tile,
// only the h = 0 epilogue warps storing).  Roles as in the single-product
// kernel: warp 0 TMA, warp 1 TMEM + MMA, warps 2..9 epilogue; two
// accumulators per tile (hi slice | smaller slices).  Stage layout: the
// three A slices (8 KiB each) then the B tile (bn x 64 bytes); Case B tiles
// are tiles of Z^T = Y^T X^T and are stored transposed.
__global__ void __launch_bounds__(GB_THREADS, 1)
g_tc_kernel(const GInst* __restrict__ inst, const CUtensorMap* __restrict__ maps,
            const int* __restrict__ cta_off, const int4* __restrict__ tiles,
            const int* __restrict__ flags, int* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    uint8_t* stg = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    GBars* bars = reinterpret_cast<GBars*>(stg + GB_STAGES * GB_STAGE);
    float* epi = reinterpret_cast<float*>(stg + GB_STAGES * GB_STAGE + 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t0 = cta_off[blockIdx.x], t1 = cta_off[blockIdx.x + 1];

    if (threadIdx.x == 0) {
        for (int s = 0; s < GB_STAGES; ++s) {
            ptx::mbar_init(&bars->full[s], 1);
            ptx::mbar_init(&bars->empty[s], 1);
        }
        ptx::mbar_init(&bars->tfull, 1);
        ptx::mbar_init(&bars->tempty, GB_EPI);
        ptx::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
        ptx::fence_proxy_async_smem();
    }
    if (warp == 1) {
        ptx::tmem_alloc(&bars->tmem_base, GB_TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued[GB_STAGES];
            for (int s = 0; s < GB_STAGES; ++s) issued[s] = -1;
            bool ok = true;
            for (int t = t0; ok && t < t1; ++t) {
                const int4 tl = tiles[t];
                const GInst& g = inst[tl.x];
                const CUtensorMap* ma = &maps[2 * tl.x];
                const CUtensorMap* mb = &maps[2 * tl.x + 1];
                constexpr int sa = 3;
                // The B tile is bn rows of 64 bytes (bn = 256 or 128).
                const uint32_t bytes = sa * GB_A_TILE + (uint32_t)g.bn * GB_BK * 2;
                const int nkb = (int)((g.n + GB_BK - 1) / GB_BK);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&bars->empty[stage], phase ^ 1u, abort,
                                                GB_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&bars->full[stage], bytes);
                    uint8_t* st = stg + stage * GB_STAGE;
                    for (int s = 0; s < sa; ++s)
                        ptx::tma_load_3d(st + s * GB_A_TILE, ma, &bars->full[stage],
                                         kb * GB_BK, tl.y * GB_BM, s);
                    ptx::tma_load_3d(st + sa * GB_A_TILE, mb, &bars->full[stage], kb * GB_BK,
                                     tl.z * g.bn, 0);
                    issued[stage] = (int)phase;
                    if (++stage == GB_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                bars->abort = 1;
                atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
                volatile int never = 0;
                for (int s = 0; s < GB_STAGES; ++s)
                    if (issued[s] >= 0)
                        ptx::mbar_wait_bounded(&bars->full[s], (uint32_t)issued[s], &never,
                                               GB_WAIT_NS);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            for (int t = t0; ok && t < t1; ++t) {
                const int4 tl = tiles[t];
                const GInst& g = inst[tl.x];
                const uint32_t IDESC = ptx::idesc_bf16_f32(GB_BM, g.bn);
                constexpr int sa = 3;
                const int nkb = (int)((g.n + GB_BK - 1) / GB_BK);
                if (!ptx::mbar_wait_bounded(&bars->tempty, tphase ^ 1u, abort, GB_WAIT_NS)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&bars->full[stage], phase, abort,
                                                GB_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t s0 = ptx::smem_addr(stg + stage * GB_STAGE);
#pragma unroll
                    for (int ks = 0; ks < GB_BK / 16; ++ks) {
#pragma unroll
                        for (int p = 2; p >= 0; --p) {
                            const uint32_t a_addr = s0 + p * GB_A_TILE + ks * 32;
                            const uint32_t b_addr = s0 + sa * GB_A_TILE + ks * 32;
                            const bool first = kb == 0 && ks == 0 && (p == 0 || p == 2);
                            ptx::mma_f16(tmem + (p == 0 ? 0u : (uint32_t)GB_BN),
                                         ptx::sdesc_kmajor_sw64(a_addr),
                                         ptx::sdesc_kmajor_sw64(b_addr), IDESC,
                                         first ? 0u : 1u);
                        }
                    }
                    ptx::mma_commit(&bars->empty[stage]);
                    if (++stage == GB_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                ptx::mma_commit(&bars->tfull);
                tphase ^= 1u;
            }
            if (!ok) {
                bars->abort = 1;
                atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
            }
            ptx::mma_commit(&bars->drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(&bars->drain, 0u, &never, GB_WAIT_NS);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128);
        uint32_t tphase = 0;
        for (int t = t0; t < t1; ++t) {
            const int4 tl = tiles[t];
            const GInst& g = inst[tl.x];
            const bool got = ptx::mbar_wait_bounded(&bars->tfull, tphase, abort, GB_WAIT_NS);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) {
                    bars->abort = 1;
                    atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
                }
                break;
            }
            ptx::tc_fence_after();
            // A 128-wide tile has columns for the h = 0 warps only; the
            // others still hand the accumulator back.
            const bool live = h * 128 < g.bn;
            float sum[128];
            if (live) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint32_t r0[32], r1[32];
                    ptx::tmem_ld_32cols(lane_base + (uint32_t)(c * 32), r0);
                    ptx::tmem_ld_32cols(lane_base + (uint32_t)(GB_BN + c * 32), r1);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        sum[c * 32 + j] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars->tempty);
            tphase ^= 1u;
            if (!live) continue;
            // Coalesced stores: each 32 x 32 block goes through this warp's
            // shared-memory tile (thread = row on the way in, thread =
            // column on the way out), one 128-byte row segment per store.
            const bool bad = flags[g.flag] != 0;
            float* sm = epi + (warp - 2) * 32 * 33;
            const int64_t mbase = (int64_t)tl.y * GB_BM + q * 32;
            if (g.kind == 1) {
                // Case B: the tile is Z^T, element (m, n) goes to Z[n][m];
                // lanes hold consecutive m, so stores are 128-byte row
                // segments without the shared-memory turn.
                const int64_t m = mbase + lane;
                const int64_t n0 = (int64_t)tl.z * g.bn + h * 128;
                if (m < g.n) {
                    float* zc = g.Z + m;
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (n0 + j < g.n)
                            zc[(n0 + j) * g.ldz] = bad ? __int_as_float(0x7fc00000) : sum[j];
                }
                continue;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int j = 0; j < 32; ++j) sm[lane * 33 + j] = sum[c * 32 + j];
                __syncwarp();
                const int64_t col = (int64_t)tl.z * g.bn + h * 128 + c * 32 + lane;
                if (col < g.n) {
                    for (int rr = 0; rr < 32; ++rr) {
                        const int64_t m = mbase + rr;
                        if (m < g.n)
                            g.Z[m * g.ldz + col] =
                                bad ? __int_as_float(0x7fc00000) : sm[rr * 33 + lane];
                    }
                }
                __syncwarp();
            }
            (void)row;
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, GB_TMEM_COLS);
    }
}

}  // namespace

afmm_status launch_batch_convert(const GInst* inst, const int* row_prefix,
                                 const int* row_job, const int* tt_prefix,
                                 const int* tt_job, int ninst, int rows_total,
                                 int tt_total, int* flags, int* status, cudaStream_t st) {
    if (ninst <= 0) return AFMM_OK;
    AFMM_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * (ninst + 1), st));
    g_rows_kernel<<<(rows_total + G_ROWS_PER_BLOCK - 1) / G_ROWS_PER_BLOCK,
                    32 * G_ROWS_PER_BLOCK, 0, st>>>(inst, row_prefix, row_job, rows_total,
                                                    flags, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    g_transpose_kernel<<<tt_total, 256, 0, st>>>(inst, tt_prefix, tt_job, flags, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFMM_OK;
}

afmm_status launch_batch_tc(const GInst* inst, const void* maps, const int* cta_off,
                            const int* tiles, int grid, const int* flags, int* status,
                            cudaStream_t st) {
    if (grid <= 0) return AFMM_OK;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(g_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       GB_SMEM));
    g_tc_kernel<<<grid, GB_THREADS, GB_SMEM, st>>>(
        inst, static_cast<const CUtensorMap*>(maps), cta_off,
        reinterpret_cast<const int4*>(tiles), flags, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_batch_widen(const WJob* jobs, const int* prefix, int njobs,
                               int rows_total, int* status, cudaStream_t st) {
    if (njobs <= 0) return AFMM_OK;
    g_widen_kernel<<<rows_total, 256, 0, st>>>(jobs, prefix, njobs, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
