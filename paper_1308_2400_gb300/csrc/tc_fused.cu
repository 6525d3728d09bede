// Case-A split-BF16 product with the split fused into the kernel.
//
// Same product as the three-slice form of tc_gemm.cu (Sec. 2 Case A: X real,
// Y Rep-factors; Z = X * Y with X = hi + mid + lo in BF16 and the hi-slice
// and small-slice products in separate TMEM accumulators), but X is read
// once, as FP32, straight from the caller's matrix: TMA brings 128 x 32 FP32
// tiles (128-byte swizzle) into a small ring, and eight converter warps cut
// each value into its three BF16 slices and write them into the stage in
// the 64-byte-swizzled K-major layout the MMA reads.  The separate split
// pass and its 6 bytes per element of slice traffic disappear.
//
// Warps: 0 TMA (X tiles and B tiles), 1 TMEM + MMA, 2..9 converters (two
// per SMSP, half a row each), 10..13 epilogue (row per thread, 32 columns
// at a time).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "afmm_common.cuh"
#include "bf16_split.cuh"
#include "ptx_sm100.cuh"
#include "tc_gemm.cuh"

namespace afmm {
namespace {

constexpr int FM = 128, FN = 256, FK = 32;
constexpr int F_CONV = 256;                      // 8 converter warps
constexpr int F_THREADS = 64 + F_CONV + 128;      // + 4 epilogue warps
constexpr int F_NX = 3;                          // FP32 X tile ring
constexpr int F_NS = 4;                          // operand stages
constexpr int F_X_BYTES = FM * FK * 4;           // 16 KiB
constexpr int F_A_BYTES = FM * FK * 2;           // 8 KiB per slice
constexpr int F_B_BYTES = FN * FK * 2;           // 16 KiB
constexpr int F_STAGE = 3 * F_A_BYTES + F_B_BYTES;
constexpr int F_SMEM = 1024 + F_NX * F_X_BYTES + F_NS * F_STAGE + 256;
constexpr uint64_t F_WAIT_NS = 2000000000ull;
constexpr int F_GROUP_M = 16;
static_assert(F_SMEM <= 232448, "shared memory");

struct FBars {
    uint64_t x_full[F_NX], x_empty[F_NX];
    uint64_t b_full[F_NS], a_full[F_NS], s_empty[F_NS];
    uint64_t tfull, tempty, drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(FBars) <= 256, "barrier block");

__device__ __forceinline__ void ftile(int tile, int tiles_m, int tiles_n, int& tm, int& tn) {
    const int per = F_GROUP_M * tiles_n;
    const int g = tile / per;
    const int first = g * F_GROUP_M;
    const int gm = min(tiles_m - first, F_GROUP_M);
    const int r = tile % per;
    tm = first + r % gm;
    tn = r / gm;
}

__device__ __forceinline__ void fabort(FBars* b, int* status) {
    b->abort = 1;
    __threadfence_block();
    atomicCAS(status, 0, (int)AFMM_ERR_TIMEOUT);
}

__global__ void __launch_bounds__(F_THREADS, 1)
tc_fused_kernel(const __grid_constant__ CUtensorMap tmX,
                const __grid_constant__ CUtensorMap tmB, float* __restrict__ Z,
                int64_t ldz, int M, int N, int K, int vec, int* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    uint8_t* xbuf = base;                                  // [F_NX][16 KiB]
    uint8_t* stg = base + F_NX * F_X_BYTES;                // [F_NS][40 KiB]
    FBars* bars = reinterpret_cast<FBars*>(stg + F_NS * F_STAGE);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + FM - 1) / FM, tiles_n = (N + FN - 1) / FN;
    const int num_tiles = tiles_m * tiles_n;
    const int num_kb = (K + FK - 1) / FK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < F_NX; ++i) {
            ptx::mbar_init(&bars->x_full[i], 1);
            ptx::mbar_init(&bars->x_empty[i], F_CONV);
        }
        for (int s = 0; s < F_NS; ++s) {
            ptx::mbar_init(&bars->b_full[s], 1);
            ptx::mbar_init(&bars->a_full[s], F_CONV);
            ptx::mbar_init(&bars->s_empty[s], 1);
        }
        ptx::mbar_init(&bars->tfull, 1);
        ptx::mbar_init(&bars->tempty, 128);
        ptx::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmX);
        ptx::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        ptx::tmem_alloc(&bars->tmem_base, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int xs = 0, s = 0;
            uint32_t xph = 0, sph = 0;
            int xiss[F_NX], siss[F_NS];
            for (int i = 0; i < F_NX; ++i) xiss[i] = -1;
            for (int i = 0; i < F_NS; ++i) siss[i] = -1;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
                int tm, tn;
                ftile(tile, tiles_m, tiles_n, tm, tn);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&bars->x_empty[xs], xph ^ 1u, abort, F_WAIT_NS) ||
                        !ptx::mbar_wait_bounded(&bars->s_empty[s], sph ^ 1u, abort, F_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&bars->x_full[xs], F_X_BYTES);
                    ptx::tma_load_3d(xbuf + xs * F_X_BYTES, &tmX, &bars->x_full[xs], kb * FK,
                                     tm * FM, 0);
                    ptx::mbar_arrive_expect_tx(&bars->b_full[s], F_B_BYTES);
                    ptx::tma_load_3d(stg + s * F_STAGE + 3 * F_A_BYTES, &tmB, &bars->b_full[s],
                                     kb * FK, tn * FN, 0);
                    xiss[xs] = (int)xph;
                    siss[s] = (int)sph;
                    if (++xs == F_NX) { xs = 0; xph ^= 1u; }
                    if (++s == F_NS) { s = 0; sph ^= 1u; }
                }
            }
            if (!ok) {
                fabort(bars, status);
                volatile int never = 0;
                for (int i = 0; i < F_NX; ++i)
                    if (xiss[i] >= 0)
                        ptx::mbar_wait_bounded(&bars->x_full[i], (uint32_t)xiss[i], &never, F_WAIT_NS);
                for (int i = 0; i < F_NS; ++i)
                    if (siss[i] >= 0)
                        ptx::mbar_wait_bounded(&bars->b_full[i], (uint32_t)siss[i], &never, F_WAIT_NS);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = ptx::idesc_bf16_f32(FM, FN);
            int s = 0;
            uint32_t sph = 0, tph = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
                if (!ptx::mbar_wait_bounded(&bars->tempty, tph ^ 1u, abort, F_WAIT_NS)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&bars->b_full[s], sph, abort, F_WAIT_NS) ||
                        !ptx::mbar_wait_bounded(&bars->a_full[s], sph, abort, F_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t s0 = ptx::smem_addr(stg + s * F_STAGE);
#pragma unroll
                    for (int ks = 0; ks < FK / 16; ++ks) {
#pragma unroll
                        for (int p = 2; p >= 0; --p) {
                            const uint32_t a = s0 + p * F_A_BYTES + ks * 32;
                            const uint32_t b = s0 + 3 * F_A_BYTES + ks * 32;
                            const bool first = kb == 0 && ks == 0 && (p == 0 || p == 2);
                            ptx::mma_f16(tmem + (p == 0 ? 0u : (uint32_t)FN),
                                         ptx::sdesc_kmajor_sw64(a), ptx::sdesc_kmajor_sw64(b),
                                         IDESC, first ? 0u : 1u);
                        }
                    }
                    ptx::mma_commit(&bars->s_empty[s]);
                    if (++s == F_NS) { s = 0; sph ^= 1u; }
                }
                if (!ok) break;
                ptx::mma_commit(&bars->tfull);
                tph ^= 1u;
            }
            if (!ok) fabort(bars, status);
            ptx::mma_commit(&bars->drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(&bars->drain, 0u, &never, F_WAIT_NS);
        }
        __syncwarp();
    } else if (warp < 2 + F_CONV / 32) {
        // ------------------------------------------------ converters
        // Thread = half hh of row m of the 128-row tile (k 16hh .. 16hh+15).
        // FP32 row m of an X tile sits at m*128 with its 16-byte chunk j
        // stored at chunk j ^ (m & 7) (128-byte swizzle); BF16 row m of a
        // slice tile sits at m*64 with chunk c stored at c ^ ((m >> 1) & 3)
        // (64-byte swizzle).
        const int t = threadIdx.x - 64;
        const int m = t & 127, hh = t >> 7;
        int xs = 0, s = 0;
        uint32_t xph = 0, sph = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
            for (int kb = 0; kb < num_kb; ++kb) {
                if (!ptx::mbar_wait_bounded(&bars->x_full[xs], xph, abort, F_WAIT_NS) ||
                    !ptx::mbar_wait_bounded(&bars->s_empty[s], sph ^ 1u, abort, F_WAIT_NS)) {
                    ok = false;
                    break;
                }
                const uint8_t* xr = xbuf + xs * F_X_BYTES + m * 128;
                uint8_t* ar = stg + s * F_STAGE + m * 64;
#pragma unroll
                for (int c = 2 * hh; c < 2 * hh + 2; ++c) {
                    const float4 f0 = *reinterpret_cast<const float4*>(
                        xr + (((2 * c) ^ (m & 7)) << 4));
                    const float4 f1 = *reinterpret_cast<const float4*>(
                        xr + (((2 * c + 1) ^ (m & 7)) << 4));
                    const float v[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
                    uint32_t w[3][4];
#pragma unroll
                    for (int t = 0; t < 8; t += 2) {
                        __nv_bfloat16 o0[3], o1[3];
                        split_bf16<3>(v[t], o0);
                        split_bf16<3>(v[t + 1], o1);
#pragma unroll
                        for (int sl = 0; sl < 3; ++sl) w[sl][t / 2] = pack2(o0[sl], o1[sl]);
                    }
                    const int pc = (c ^ ((m >> 1) & 3)) << 4;
#pragma unroll
                    for (int sl = 0; sl < 3; ++sl)
                        *reinterpret_cast<uint4*>(ar + sl * F_A_BYTES + pc) =
                            make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
                }
                // Generic-proxy stores become visible to the tensor core's
                // async-proxy reads before the stage is declared ready.
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive(&bars->x_empty[xs]);
                ptx::mbar_arrive(&bars->a_full[s]);
                if (++xs == F_NX) { xs = 0; xph ^= 1u; }
                if (++s == F_NS) { s = 0; sph ^= 1u; }
            }
        }
        if (!ok) fabort(bars, status);
    } else {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t tph = 0;
        for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
            int tm, tn;
            ftile(tile, tiles_m, tiles_n, tm, tn);
            const bool got = ptx::mbar_wait_bounded(&bars->tfull, tph, abort, F_WAIT_NS);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) fabort(bars, status);
                break;
            }
            ptx::tc_fence_after();
            const int64_t m = (int64_t)tm * FM + row;
            const int col0 = tn * FN;
#pragma unroll 1
            for (int c = 0; c < FN / 32; ++c) {
                uint32_t r0[32], r1[32];
                ptx::tmem_ld_32cols(lane_base + (uint32_t)(c * 32), r0);
                ptx::tmem_ld_32cols(lane_base + (uint32_t)(FN + c * 32), r1);
                ptx::tmem_ld_wait();
                if (m < M) {
                    float* zr = Z + m * ldz + col0 + c * 32;
                    const int cl = col0 + c * 32;
                    if (vec && cl + 32 <= N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4*>(zr + j) = make_float4(
                                __uint_as_float(r0[j]) + __uint_as_float(r1[j]),
                                __uint_as_float(r0[j + 1]) + __uint_as_float(r1[j + 1]),
                                __uint_as_float(r0[j + 2]) + __uint_as_float(r1[j + 2]),
                                __uint_as_float(r0[j + 3]) + __uint_as_float(r1[j + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (cl + j < N)
                                zr[j] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
                    }
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars->tempty);
            tph ^= 1u;
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

bool tc_fused_usable(const afmm_desc& d, const void* X) {
    return (d.flags & AFMM_FLAG_FUSED_SPLIT) && d.kase == AFMM_CASE_A &&
           d.x_dtype == AFMM_F32 && d.n >= 32 &&
           (d.ldx ? d.ldx : d.n) % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
}

afmm_status tc_run_fused_caseA(const TcPlan* t, const afmm_desc& d, const void* X,
                               void* Z, int* status, cudaStream_t st) {
    auto fn = encode_fn();
    if (!fn) return AFMM_ERR_CUDA;
    const int64_t n = d.n, ldx = d.ldx ? d.ldx : n;
    // FP32 X as a 3-D map with one slice: dims {K = n, rows = n, 1}.
    alignas(64) CUtensorMap mx;
    cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, 1};
    cuuint64_t strides[2] = {(cuuint64_t)(ldx * 4), (cuuint64_t)(ldx * 4 * n)};
    cuuint32_t box[3] = {(cuuint32_t)FK, (cuuint32_t)FM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(X), dims, strides, box,
           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return AFMM_ERR_CUDA;
    CUtensorMap mb;
    std::memcpy(&mb, t->tmap_b, sizeof mb);
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    const int tiles = (int)(((n + FM - 1) / FM) * ((n + FN - 1) / FN));
    const int grid = tiles < dp.sm_count ? tiles : dp.sm_count;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(tc_fused_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM));
    const int64_t ldz = d.ldz ? d.ldz : n;
    const int vec = (ldz % 4 == 0) && ((reinterpret_cast<uintptr_t>(Z) & 15u) == 0);
    main_kernel_begin(st);
    tc_fused_kernel<<<grid, F_THREADS, F_SMEM, st>>>(mx, mb, static_cast<float*>(Z), ldz,
                                                     (int)n, (int)n, (int)n, vec, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, grid);
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
