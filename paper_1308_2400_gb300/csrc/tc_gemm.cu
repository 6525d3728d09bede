// Tensor-core AFMM product on sm_103a: tcgen05 MMA with TMEM accumulators,
// operands brought in by TMA, warp-specialised persistent kernel.
//
// The AFMM term Rep * Base (Sec. 2: Base added Rep-factor times) is an exact
// integer multiple of the Base value.  On the tensor cores it is formed as a
// product of BF16 operands accumulated in FP32:
//  - Rep-factors are small non-negative integers, exact in BF16 (all
//    integers up to 256);
//  - the real Base factor is split into S BF16 slices, hi + mid + lo, each
//    the round-to-nearest BF16 of the previous residual, so that for S = 3 the
//    slices sum exactly to an FP32 value;
//  - Z = sum_s X_s * Y (case A) or X * sum_s Y_s (case B): one FP32 TMEM
//    accumulator per output tile takes all S products of every k step, the
//    Rep-factor tile being loaded once and reused for the S slices.
//
// Kernel layout (one CTA per SM, persistent over 128 x 256 output tiles):
//   warp 0      TMA producer: K steps of 32 (64-byte swizzled rows) of every
//               slice of A and B into a ring of shared-memory stages;
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32
//               accumulators) and issues the MMAs (128 x 256 x 16 each);
//   warps 2..5  epilogue: TMEM -> registers -> Z (FP32), overlapping the
//               next tile's MMAs through the second accumulator.
// Every wait on an mbarrier is bounded (2 s); a wait that runs out records
// AFMM_ERR_TIMEOUT in the status word, stops the other roles, lets copies
// and MMAs in flight finish (bounded) and frees TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "afmm_common.cuh"
#include "elem.cuh"
#include "ptx_sm100.cuh"
#include "tc_gemm.cuh"

namespace afmm {

namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 32;
constexpr int TC_THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr int A_TILE_BYTES = TC_BM * TC_BK * 2;   // 8 KiB
constexpr int B_TILE_BYTES = TC_BN * TC_BK * 2;   // 16 KiB
constexpr int SMEM_OPTIN = 232448;                // 227 KiB per CTA
constexpr int GROUP_M = 16;                       // tile raster band
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

template <int SA, int SB>
struct TcCfg {
    static constexpr int STAGE_BYTES = SA * A_TILE_BYTES + SB * B_TILE_BYTES;
    static constexpr int STAGES_FIT = (SMEM_OPTIN - 2048) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + 256;
    static constexpr int P = SA > SB ? SA : SB;   // MMAs per 16-wide k step
    static_assert(SA == 1 || SB == 1, "slices on one side only");
    static_assert(STAGES >= 2, "pipeline needs two stages");
    static_assert(SMEM <= SMEM_OPTIN, "shared memory");
};

struct TcBars {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(TcBars) <= 256, "barrier block");

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

template <int SA, int SB>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
               const __grid_constant__ CUtensorMap tmB, float* __restrict__ Z,
               int64_t ldz, int M, int N, int K, int vec, int* status) {
    using Cfg = TcCfg<SA, SB>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    uint8_t* tiles = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    TcBars* bars = reinterpret_cast<TcBars*>(tiles + Cfg::STAGES * Cfg::STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + TC_BM - 1) / TC_BM, tiles_n = (N + TC_BN - 1) / TC_BN;
    const int num_tiles = tiles_m * tiles_n;
    const int num_kb = (K + TC_BK - 1) / TC_BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            ptx::mbar_init(&bars->full[s], 1);
            ptx::mbar_init(&bars->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(&bars->tfull[a], 1);
            ptx::mbar_init(&bars->tempty[a], 128);
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
        if (lane == 0) {
        // ---------------------------------------------------- TMA producer
        int stage = 0;
        uint32_t phase = 0;
        int issued_phase[8];
        for (int s = 0; s < 8; ++s) issued_phase[s] = -1;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
            int tm, tn;
            tile_coords(tile, tiles_m, tiles_n, tm, tn);
            for (int kb = 0; kb < num_kb; ++kb) {
                if (!ptx::mbar_wait_bounded(&bars->empty[stage], phase ^ 1u,
                                            abort, WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                ptx::mbar_arrive_expect_tx(&bars->full[stage], Cfg::STAGE_BYTES);
                uint8_t* st = tiles + stage * Cfg::STAGE_BYTES;
#pragma unroll
                for (int s = 0; s < SA; ++s)
                    ptx::tma_load_3d(st + s * A_TILE_BYTES, &tmA, &bars->full[stage],
                                     kb * TC_BK, tm * TC_BM, s);
#pragma unroll
                for (int s = 0; s < SB; ++s)
                    ptx::tma_load_3d(st + SA * A_TILE_BYTES + s * B_TILE_BYTES, &tmB,
                                     &bars->full[stage], kb * TC_BK, tn * TC_BN, s);
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
        if (lane == 0) {
        // ---------------------------------------------------- MMA issuer
        constexpr uint32_t IDESC = ptx::idesc_bf16_f32(TC_BM, TC_BN);
        int stage = 0;
        uint32_t phase = 0;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
            if (!ptx::mbar_wait_bounded(&bars->tempty[acc], acc_phase ^ 1u, abort,
                                        WAIT_LIMIT_NS)) {
                ok = false;
                break;
            }
            ptx::tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * TC_BN);
            for (int kb = 0; kb < num_kb; ++kb) {
                if (!ptx::mbar_wait_bounded(&bars->full[stage], phase, abort,
                                            WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t s0 = ptx::smem_addr(tiles + stage * Cfg::STAGE_BYTES);
#pragma unroll
                for (int ks = 0; ks < TC_BK / 16; ++ks) {
#pragma unroll
                    for (int p = 0; p < Cfg::P; ++p) {
                        const uint32_t a_addr =
                            s0 + (SA > 1 ? p : 0) * A_TILE_BYTES + ks * 32;
                        const uint32_t b_addr = s0 + SA * A_TILE_BYTES +
                                                (SB > 1 ? p : 0) * B_TILE_BYTES + ks * 32;
                        ptx::mma_f16(d, ptx::sdesc_kmajor_sw64(a_addr),
                                     ptx::sdesc_kmajor_sw64(b_addr), IDESC,
                                     (kb | ks | p) != 0 ? 1u : 0u);
                    }
                }
                ptx::mma_commit(&bars->empty[stage]);
                if (++stage == Cfg::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
            ptx::mma_commit(&bars->tfull[acc]);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
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
        const int q = warp & 3;                 // TMEM lanes 32q .. 32q+31
        const int row = q * 32 + lane;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
            int tm, tn;
            tile_coords(tile, tiles_m, tiles_n, tm, tn);
            const bool got = ptx::mbar_wait_bounded(&bars->tfull[acc], acc_phase,
                                                    abort, WAIT_LIMIT_NS);
            // TMEM loads below are warp-collective: decide as a warp.
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) raise_abort(bars, status);
                break;
            }
            ptx::tc_fence_after();
            const int64_t m = (int64_t)tm * TC_BM + row;
            const int n0 = tn * TC_BN;
#pragma unroll 1
            for (int c = 0; c < TC_BN / 32; ++c) {
                uint32_t r[32];
                ptx::tmem_ld_32cols(tmem + ((uint32_t)(q * 32) << 16) +
                                        (uint32_t)(acc * TC_BN + c * 32), r);
                ptx::tmem_ld_wait();
                if (m < M) {
                    const int col = n0 + c * 32;
                    float* zr = Z + m * ldz + col;
                    if (vec && col + 32 <= N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 v;
                            v.x = __uint_as_float(r[j]);
                            v.y = __uint_as_float(r[j + 1]);
                            v.z = __uint_as_float(r[j + 2]);
                            v.w = __uint_as_float(r[j + 3]);
                            *reinterpret_cast<float4*>(zr + j) = v;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col + j < N) zr[j] = __uint_as_float(r[j]);
                    }
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars->tempty[acc]);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
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

// --------------------------------------------------------------- operands
// Round-to-nearest BF16 slices of v: out[0] = bf16(v), out[s] = bf16 of the
// residual left by out[0..s-1].  Residuals are exact in FP64.
template <int S>
__device__ __forceinline__ void split_bf16(double v, __nv_bfloat16 (&out)[S]) {
    double r = v;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        out[s] = __double2bfloat16(r);
        r -= (double)__bfloat162float(out[s]);
    }
}

// Rows kept as rows (K-major A operand): dst[(s*n + r)*ldk + c].
// EXACT: a single slice that must equal the source (Rep-factors).
template <int DT, int S, bool EXACT>
__global__ void widen_rows_kernel(const void* __restrict__ src, int64_t n,
                                  int64_t lds, __nv_bfloat16* __restrict__ dst,
                                  int64_t ldk, int* status) {
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (c >= ldk) return;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        __nv_bfloat16 o[S];
        if (c < n) {
            const double v = Elem<DT>::get(src, r * lds + c);
            split_bf16<S>(v, o);
            if (EXACT && (double)__bfloat162float(o[0]) != v)
                atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) o[s] = __float2bfloat16(0.0f);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) dst[((int64_t)s * n + r) * ldk + c] = o[s];
    }
}

// Rows become columns (K-major B operand from a row-major K x N matrix):
// dst[(s*n + c)*ldk + r] = slice_s(src[r][c]), 32 x 32 tiles via smem.
template <int DT, int S, bool EXACT>
__global__ void widen_transpose_kernel(const void* __restrict__ src, int64_t n,
                                       int64_t lds, __nv_bfloat16* __restrict__ dst,
                                       int64_t ldk, int* status) {
    __shared__ double tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < n && c < n) ? Elem<DT>::get(src, r * lds + c) : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;   // output row c, col r
        if (c < n && r < ldk) {
            const double v = tile[threadIdx.x][i];
            __nv_bfloat16 o[S];
            split_bf16<S>(v, o);
            if (EXACT && (double)__bfloat162float(o[0]) != v)
                atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
#pragma unroll
            for (int s = 0; s < S; ++s) dst[((int64_t)s * n + c) * ldk + r] = o[s];
        }
    }
}

template <int S, bool EXACT>
afmm_status launch_widen_rows(const void* src, int dt, int64_t n, int64_t lds,
                              __nv_bfloat16* dst, int64_t ldk, int* status,
                              cudaStream_t st) {
    const dim3 grid((unsigned)((ldk + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        widen_rows_kernel<DT, S, EXACT><<<grid, 256, 0, st>>>(src, n, lds, dst, ldk,
                                                              status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

template <int S, bool EXACT>
afmm_status launch_widen_transpose(const void* src, int dt, int64_t n,
                                   int64_t lds, __nv_bfloat16* dst, int64_t ldk,
                                   int* status, cudaStream_t st) {
    const int64_t g = (n + 31) / 32;
    if (g > 65535) return AFMM_ERR_UNSUPPORTED;
    const dim3 grid((unsigned)g, (unsigned)g), block(32, 8);
    afmm_status rc = dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        widen_transpose_kernel<DT, S, EXACT><<<grid, block, 0, st>>>(src, n, lds, dst,
                                                                     ldk, status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
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

// 3-D map over a stack of `slices` BF16 matrices of `rows` x `cols` (K)
// with leading dimension `ld`; box = 32 (K) x box_rows x 1.
afmm_status encode_map(void* out, void* base, int64_t cols, int64_t rows,
                       int64_t ld, int slices, int box_rows) {
    auto fn = get_encode_fn();
    if (!fn) return AFMM_ERR_CUDA;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(ld * 2 * rows)};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                    3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? AFMM_OK : AFMM_ERR_CUDA;
}

template <int SA, int SB>
afmm_status launch_tc(const TcPlan* t, float* Z, int64_t ldz, int* status,
                      cudaStream_t st) {
    using Cfg = TcCfg<SA, SB>;
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    const int n = (int)t->n;
    const int tiles = ((n + TC_BM - 1) / TC_BM) * ((n + TC_BN - 1) / TC_BN);
    const int grid = tiles < dp.sm_count ? tiles : dp.sm_count;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<SA, SB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg::SMEM));
    const int vec = (ldz % 4 == 0) && ((reinterpret_cast<uintptr_t>(Z) & 15u) == 0);
    CUtensorMap ma, mb;
    std::memcpy(&ma, t->tmap_a, sizeof ma);
    std::memcpy(&mb, t->tmap_b, sizeof mb);
    main_kernel_begin(st);
    tc_gemm_kernel<SA, SB><<<grid, TC_THREADS, Cfg::SMEM, st>>>(ma, mb, Z, ldz, n, n, n,
                                                               vec, status);
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

void tc_layout(TcPlan* t, const afmm_desc& d, int slices) {
    t->n = d.n;
    t->slices = slices;
    t->sliced_a = d.kase == AFMM_CASE_A;
    t->ld_a = t->ld_b = (d.n + 7) / 8 * 8;
    const int sa = t->sliced_a ? slices : 1, sb = t->sliced_a ? 1 : slices;
    t->rows_a = d.n;
    t->rows_b = d.n;
    t->a_bytes = (size_t)sa * d.n * t->ld_a * 2;
    t->b_bytes = (size_t)sb * d.n * t->ld_b * 2;
}

afmm_status tc_bind_workspace(TcPlan* t, void* a, void* b) {
    t->a = a;
    t->b = b;
    t->maps_ready = false;
    if (t->n <= 0) return AFMM_OK;
    const int sa = t->sliced_a ? t->slices : 1, sb = t->sliced_a ? 1 : t->slices;
    AFMM_TRY(encode_map(t->tmap_a, a, t->n, t->n, t->ld_a, sa, TC_BM));
    AFMM_TRY(encode_map(t->tmap_b, b, t->n, t->n, t->ld_b, sb, TC_BN));
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
    if (d.kase == AFMM_CASE_A) {
        // A = slices of the real X (rows), B = Rep-factors Y transposed.
        if (t->slices == 3)
            AFMM_TRY((launch_widen_rows<3, false>(X, d.x_dtype, n, d.ldx, A, t->ld_a,
                                                  status, st)));
        else
            AFMM_TRY((launch_widen_rows<2, false>(X, d.x_dtype, n, d.ldx, A, t->ld_a,
                                                  status, st)));
        AFMM_TRY((launch_widen_transpose<1, true>(Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                  status, st)));
        return t->slices == 3 ? launch_tc<3, 1>(t, Zf, d.ldz, status, st)
                              : launch_tc<2, 1>(t, Zf, d.ldz, status, st);
    }
    // Case B: A = Rep-factors X (rows), B = slices of the real Y transposed.
    AFMM_TRY((launch_widen_rows<1, true>(X, d.x_dtype, n, d.ldx, A, t->ld_a, status,
                                         st)));
    if (t->slices == 3)
        AFMM_TRY((launch_widen_transpose<3, false>(Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                   status, st)));
    else
        AFMM_TRY((launch_widen_transpose<2, false>(Y, d.y_dtype, n, d.ldy, B, t->ld_b,
                                                   status, st)));
    return t->slices == 3 ? launch_tc<1, 3>(t, Zf, d.ldz, status, st)
                          : launch_tc<1, 2>(t, Zf, d.ldz, status, st);
}

}  // namespace afmm
