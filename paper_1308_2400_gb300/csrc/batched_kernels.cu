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

namespace afmm {
namespace {

constexpr int GB_EPI = 256;
constexpr int GB_THREADS = 64 + GB_EPI;
constexpr uint32_t GB_TMEM_COLS = 512;
constexpr int GB_A_TILE = GB_BM * GB_BK * 2;      // 8 KiB
constexpr int GB_B_TILE = GB_BN * GB_BK * 2;      // 16 KiB
constexpr int GB_STAGE = GB_A_TILE + 3 * GB_B_TILE;   // fits 3A+1B and 1A+3B
constexpr int GB_STAGES = 3;
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
// Block b converts one row of the A operand of one instance: Case A slices
// a row of the real X into 3 BF16 rows; Case B widens a row of the
// Rep-factors X to BF16 (values must be exact, |v| <= 256, else the
// instance's flag is set and its Z becomes NaN).  Eight columns per thread,
// one 16-byte store per slice; FP32 arithmetic throughout.
__global__ void __launch_bounds__(128)
g_rows_kernel(const GInst* __restrict__ inst, const int* __restrict__ row_prefix,
              int ninst, int* __restrict__ flags) {
    const int j = find_job(row_prefix, ninst, blockIdx.x);
    const GInst& g = inst[j];
    const int64_t r = blockIdx.x - row_prefix[j];
    const int64_t n = g.n, ldk = g.ldk;
    const bool vec = g.x_dtype == AFMM_F32 && (g.ldx % 4) == 0 &&
                     ((reinterpret_cast<uintptr_t>(g.X) & 15u) == 0);
    const bool vec8 = (g.x_dtype == AFMM_U8 || g.x_dtype == AFMM_I8 ||
                       g.x_dtype == AFMM_E4M3) &&
                      (g.ldx % 8) == 0 && ((reinterpret_cast<uintptr_t>(g.X) & 7u) == 0);
    for (int64_t c = 8 * threadIdx.x; c < ldk; c += 8 * 128) {
        float v[8];
        if (vec8 && c + 8 <= n) {
            const uint2 w = *reinterpret_cast<const uint2*>(
                static_cast<const uint8_t*>(g.X) + r * g.ldx + c);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const uint8_t byte = (uint8_t)((t < 4 ? w.x : w.y) >> (8 * (t & 3)));
                v[t] = load_any_f(&byte, 0, g.x_dtype);
            }
        } else if (vec && c + 8 <= n) {
            const float4* q = reinterpret_cast<const float4*>(
                static_cast<const float*>(g.X) + r * g.ldx + c);
            const float4 a = q[0], b = q[1];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                v[t] = (c + t < n) ? load_any_f(g.X, r * g.ldx + c + t, g.x_dtype) : 0.f;
        }
        if (g.kind == 0) {
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
            bool bad = false;
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                const __nv_bfloat16 b0 = __float2bfloat16_rn(v[t]);
                const __nv_bfloat16 b1 = __float2bfloat16_rn(v[t + 1]);
                bad |= __bfloat162float(b0) != v[t] || __bfloat162float(b1) != v[t + 1] ||
                       fabsf(v[t]) > 256.f || fabsf(v[t + 1]) > 256.f;
                w[t / 2] = pack2(b0, b1);
            }
            if (bad) atomicExch(&flags[g.flag], 1);
            *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(g.A) + r * ldk + c) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Block b converts one 64 x 64 tile of the B operand (Y transposed to
// K-major): Case A widens the Rep-factors Y; Case B slices the real Y.
// Loads: a thread reads 4 consecutive source values (one 16-byte load for
// FP32, one 4-byte load for one-byte dtypes, when aligned); stores: 4
// threads write one 128-byte output row segment (16 BF16 values each).
__global__ void __launch_bounds__(256)
g_transpose_kernel(const GInst* __restrict__ inst, const int* __restrict__ tt_prefix,
                   int ninst, int* __restrict__ flags) {
    __shared__ float tile[64][65];
    const int j = find_job(tt_prefix, ninst, blockIdx.x);
    const GInst& g = inst[j];
    const int64_t n = g.n, ldk = g.ldk;
    const int64_t tpr = (n + 63) / 64;
    const int64_t t = blockIdx.x - tt_prefix[j];
    const int64_t r0 = (t / tpr) * 64, c0 = (t % tpr) * 64;
    const int tid = threadIdx.x;
    const int dt = g.y_dtype;
    const bool f4 = dt == AFMM_F32 && (g.ldy % 4) == 0 &&
                    ((reinterpret_cast<uintptr_t>(g.Y) & 15u) == 0);
    const bool b4 = (dt == AFMM_U8 || dt == AFMM_I8 || dt == AFMM_E4M3) &&
                    (g.ldy % 4) == 0 && ((reinterpret_cast<uintptr_t>(g.Y) & 3u) == 0);
    // 16 threads per source row (4 values each), 16 rows per pass.
    const int lc = (tid & 15) * 4;
    for (int i = tid >> 4; i < 64; i += 16) {
        const int64_t r = r0 + i, c = c0 + lc;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (r < n) {
            if (f4 && c + 4 <= n) {
                const float4 q = *reinterpret_cast<const float4*>(
                    static_cast<const float*>(g.Y) + r * g.ldy + c);
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else if (b4 && c + 4 <= n) {
                const uint32_t w = *reinterpret_cast<const uint32_t*>(
                    static_cast<const uint8_t*>(g.Y) + r * g.ldy + c);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint8_t byte = (uint8_t)(w >> (8 * e));
                    v[e] = load_any_f(&byte, 0, dt);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (c + e < n) v[e] = load_any_f(g.Y, r * g.ldy + c + e, dt);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) tile[i][lc + e] = v[e];
    }
    __syncthreads();
    // Output row cc (source column), source rows 16*qq .. 16*qq+15.
    const int cc = tid >> 2, qq = tid & 3;
    const int64_t c = c0 + cc, r = r0 + 16 * qq;
    bool bad = false;
    if (c < n && r < ldk) {
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = tile[16 * qq + e][cc];
        // r + 16 <= ldk unless ldk ends inside this group (ldk % 8 == 0).
        const int cnt = (int)((ldk - r) < 16 ? (ldk - r) : 16);
        if (g.kind == 0) {
            uint32_t w[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const __nv_bfloat16 b0 = __float2bfloat16_rn(v[e]);
                const __nv_bfloat16 b1 = __float2bfloat16_rn(v[e + 1]);
                bad |= __bfloat162float(b0) != v[e] || __bfloat162float(b1) != v[e + 1] ||
                       fabsf(v[e]) > 256.f || fabsf(v[e + 1]) > 256.f;
                w[e / 2] = pack2(b0, b1);
            }
            __nv_bfloat16* o = static_cast<__nv_bfloat16*>(g.B) + c * ldk + r;
            *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
            if (cnt == 16) *reinterpret_cast<uint4*>(o + 8) = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
            uint32_t w[3][8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                __nv_bfloat16 o0[3], o1[3];
                split_bf16<3>(v[e], o0);
                split_bf16<3>(v[e + 1], o1);
#pragma unroll
                for (int sl = 0; sl < 3; ++sl) w[sl][e / 2] = pack2(o0[sl], o1[sl]);
            }
#pragma unroll
            for (int sl = 0; sl < 3; ++sl) {
                __nv_bfloat16* o =
                    static_cast<__nv_bfloat16*>(g.B) + ((int64_t)sl * n + c) * ldk + r;
                *reinterpret_cast<uint4*>(o) = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
                if (cnt == 16)
                    *reinterpret_cast<uint4*>(o + 8) =
                        make_uint4(w[sl][4], w[sl][5], w[sl][6], w[sl][7]);
            }
        }
    }
    if (bad) atomicExch(&flags[g.flag], 1);
}

// Block b widens one row of one operand to FP32 for the CUDA-core form.
__global__ void __launch_bounds__(256)
g_widen_kernel(const WJob* __restrict__ jobs, const int* __restrict__ prefix, int njobs) {
    const int j = find_job(prefix, njobs, blockIdx.x);
    const WJob& w = jobs[j];
    const int64_t r = blockIdx.x - prefix[j];
    for (int64_t c = threadIdx.x; c < w.n; c += 256)
        w.dst[r * w.n + c] = load_any_f(w.src, r * w.lds + c, w.dtype);
}

// ----------------------------------------------------------- grouped TC
// Persistent: CTA b runs tiles[cta_off[b] .. cta_off[b+1]) in order; a tile
// is (instance, tm, tn).  Roles as in the single-product kernel: warp 0 TMA,
// warp 1 TMEM + MMA, warps 2..9 epilogue; two accumulators per tile (hi
// slice | smaller slices).  Stage layout: A slices then B slices, 8 KiB per
// A tile and 16 KiB per B tile (3A+1B for Case A, 1A+3B for Case B).
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
                const int sa = g.kind == 0 ? 3 : 1, sb = g.kind == 0 ? 1 : 3;
                const uint32_t bytes = sa * GB_A_TILE + sb * GB_B_TILE;
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
                    for (int s = 0; s < sb; ++s)
                        ptx::tma_load_3d(st + sa * GB_A_TILE + s * GB_B_TILE, mb,
                                         &bars->full[stage], kb * GB_BK, tl.z * GB_BN, s);
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
            constexpr uint32_t IDESC = ptx::idesc_bf16_f32(GB_BM, GB_BN);
            int stage = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            for (int t = t0; ok && t < t1; ++t) {
                const int4 tl = tiles[t];
                const GInst& g = inst[tl.x];
                const int kind = g.kind;
                const int sa = kind == 0 ? 3 : 1;
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
                            const uint32_t a_addr =
                                s0 + (kind == 0 ? p : 0) * GB_A_TILE + ks * 32;
                            const uint32_t b_addr =
                                s0 + sa * GB_A_TILE + (kind == 1 ? p : 0) * GB_B_TILE + ks * 32;
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
            float sum[128];
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
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars->tempty);
            tphase ^= 1u;
            // Coalesced stores: each 32 x 32 block goes through this warp's
            // shared-memory tile (thread = row on the way in, thread =
            // column on the way out), one 128-byte row segment per store.
            const bool bad = flags[g.flag] != 0;
            float* sm = epi + (warp - 2) * 32 * 33;
            const int64_t mbase = (int64_t)tl.y * GB_BM + q * 32;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int j = 0; j < 32; ++j) sm[lane * 33 + j] = sum[c * 32 + j];
                __syncwarp();
                const int64_t col = (int64_t)tl.z * GB_BN + h * 128 + c * 32 + lane;
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
                                 const int* tt_prefix, int ninst, int rows_total,
                                 int tt_total, int* flags, cudaStream_t st) {
    if (ninst <= 0) return AFMM_OK;
    AFMM_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * (ninst + 1), st));
    g_rows_kernel<<<rows_total, 128, 0, st>>>(inst, row_prefix, ninst, flags);
    AFMM_CUDA_TRY(cudaGetLastError());
    g_transpose_kernel<<<tt_total, 256, 0, st>>>(inst, tt_prefix, ninst, flags);
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
                               int rows_total, cudaStream_t st) {
    if (njobs <= 0) return AFMM_OK;
    g_widen_kernel<<<rows_total, 256, 0, st>>>(jobs, prefix, njobs);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
