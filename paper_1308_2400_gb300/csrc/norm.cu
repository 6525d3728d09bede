// K6: error of a result against a reference, in FP64 on the GPU.
// out[0] = ||Z - R||_F, out[1] = ||R||_F, out[2] = max |Z - R|.
// Two launches: per-block partial sums (fixed order per block, so the
// result does not depend on scheduling), then one block combines them.
#include "afmm_common.cuh"
#include "elem.cuh"

namespace afmm {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;

struct Part {
    double d2, r2, dmax, pad_;
};

__device__ __forceinline__ Part part_merge(Part a, const Part& b) {
    a.d2 += b.d2;
    a.r2 += b.r2;
    a.dmax = fmax(a.dmax, b.dmax);
    return a;
}

__device__ Part block_reduce(Part p) {
    __shared__ Part sh[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        Part o;
        o.d2 = __shfl_down_sync(0xffffffffu, p.d2, off);
        o.r2 = __shfl_down_sync(0xffffffffu, p.r2, off);
        o.dmax = __shfl_down_sync(0xffffffffu, p.dmax, off);
        p = part_merge(p, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = p;
    __syncthreads();
    if (warp == 0) {
        if (lane < kThreads / 32) p = sh[lane];
        else p = Part{0.0, 0.0, 0.0, 0.0};
        for (int off = 16; off > 0; off >>= 1) {
            Part o;
            o.d2 = __shfl_down_sync(0xffffffffu, p.d2, off);
            o.r2 = __shfl_down_sync(0xffffffffu, p.r2, off);
            o.dmax = __shfl_down_sync(0xffffffffu, p.dmax, off);
            p = part_merge(p, o);
        }
    }
    return p;
}

template <int ZD, int RD>
__global__ void __launch_bounds__(kThreads)
err_partial_kernel(const void* __restrict__ Z, int64_t ldz,
                   const void* __restrict__ R, int64_t ldr, int64_t rows,
                   int64_t cols, Part* __restrict__ parts) {
    Part p{0.0, 0.0, 0.0, 0.0};
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
        for (int64_t c = threadIdx.x; c < cols; c += kThreads) {
            const double z = Elem<ZD>::get(Z, r * ldz + c);
            const double ref = Elem<RD>::get(R, r * ldr + c);
            const double d = z - ref;
            p.d2 = fma(d, d, p.d2);
            p.r2 = fma(ref, ref, p.r2);
            p.dmax = fmax(p.dmax, fabs(d));
        }
    p = block_reduce(p);
    if (threadIdx.x == 0) parts[blockIdx.x] = p;
}

__global__ void __launch_bounds__(kThreads)
err_final_kernel(const Part* __restrict__ parts, int nb, double* out) {
    Part p{0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += kThreads) p = part_merge(p, parts[b]);
    p = block_reduce(p);
    if (threadIdx.x == 0) {
        out[0] = sqrt(p.d2);
        out[1] = sqrt(p.r2);
        out[2] = p.dmax;
    }
}

int blocks_for(int64_t rows) {
    DeviceProps dp;
    int cap = kMaxBlocks;
    if (device_props(&dp) == AFMM_OK && dp.sm_count * 4 < cap)
        cap = dp.sm_count * 4;
    int64_t nb = rows < 1 ? 1 : rows;
    return (int)(nb < cap ? nb : cap);
}

}  // namespace

size_t error_norm_ws_bytes(int64_t rows, int64_t cols) {
    (void)rows;
    (void)cols;
    return sizeof(Part) * kMaxBlocks + 256;
}

afmm_status launch_error_norm(const void* Z, int zdt, int64_t ldz,
                              const void* R, int rdt, int64_t ldr,
                              int64_t rows, int64_t cols, void* ws,
                              double* out_dev, cudaStream_t st) {
    auto ok_dt = [](int d) {
        return d == AFMM_F64 || d == AFMM_F32 || d == AFMM_I32;
    };
    if (!ok_dt(zdt) || !ok_dt(rdt)) return AFMM_ERR_INVALID_ARG;
    const int nb = blocks_for(rows);
    Part* parts = static_cast<Part*>(ws);
    afmm_status rc = dispatch_dtype(zdt, [&]<int ZD>() -> afmm_status {
        return dispatch_dtype(rdt, [&]<int RD>() -> afmm_status {
            if constexpr ((ZD == AFMM_F64 || ZD == AFMM_F32 || ZD == AFMM_I32) &&
                          (RD == AFMM_F64 || RD == AFMM_F32 || RD == AFMM_I32)) {
                err_partial_kernel<ZD, RD><<<nb, kThreads, 0, st>>>(
                    Z, ldz, R, ldr, rows, cols, parts);
                return AFMM_OK;
            } else {
                return AFMM_ERR_INVALID_ARG;
            }
        });
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    err_final_kernel<<<1, kThreads, 0, st>>>(parts, nb, out_dev);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFMM_OK;
}

}  // namespace afmm
