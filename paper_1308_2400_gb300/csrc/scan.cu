// K0: one pass over a matrix gathering what the AFMM planner and the
// validation need (Sec. 2.2 parameters): non-zero count (density d),
// sum and maximum (mean Rep-factor mu, mu'), and the Rep-factor checks of
// Sec. 2 (non-negative integers).  HBM-bound; one read of the matrix.
#include <cfloat>

#include "afmm_common.cuh"
#include "elem.cuh"

namespace afmm {

namespace {

constexpr int kScanThreads = 256;

__device__ __forceinline__ void stats_init(ScanStats& s) {
    s.nnz = s.negative = s.nonint = s.over127 = 0;
    s.sum = 0.0;
    s.maxv = -DBL_MAX;
    s.max_abs = 0.0;
    s.pad_ = 0.0;
}

__device__ __forceinline__ void stats_merge(ScanStats& a, const ScanStats& b) {
    a.nnz += b.nnz;
    a.negative += b.negative;
    a.nonint += b.nonint;
    a.over127 += b.over127;
    a.sum += b.sum;
    a.maxv = fmax(a.maxv, b.maxv);
    a.max_abs = fmax(a.max_abs, b.max_abs);
}

__device__ __forceinline__ void stats_shfl_merge(ScanStats& s, int off) {
    ScanStats o;
    o.nnz = __shfl_down_sync(0xffffffffu, s.nnz, off);
    o.negative = __shfl_down_sync(0xffffffffu, s.negative, off);
    o.nonint = __shfl_down_sync(0xffffffffu, s.nonint, off);
    o.over127 = __shfl_down_sync(0xffffffffu, s.over127, off);
    o.sum = __shfl_down_sync(0xffffffffu, s.sum, off);
    o.maxv = __shfl_down_sync(0xffffffffu, s.maxv, off);
    o.max_abs = __shfl_down_sync(0xffffffffu, s.max_abs, off);
    stats_merge(s, o);
}

// Block-wide reduction; thread 0 returns the total.
__device__ ScanStats block_reduce(ScanStats s) {
    __shared__ ScanStats warp_part[kScanThreads / 32];
    for (int off = 16; off > 0; off >>= 1) stats_shfl_merge(s, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = s;
    __syncthreads();
    if (warp == 0) {
        if (lane < kScanThreads / 32) s = warp_part[lane];
        else stats_init(s);
        for (int off = 16; off > 0; off >>= 1) stats_shfl_merge(s, off);
    }
    return s;
}

template <int DT>
__global__ void __launch_bounds__(kScanThreads)
scan_kernel(const void* __restrict__ M, int64_t n, int64_t ld,
            ScanStats* __restrict__ partials) {
    ScanStats s;
    stats_init(s);
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        for (int64_t c = threadIdx.x; c < n; c += kScanThreads) {
            const double v = Elem<DT>::get(M, r * ld + c);
            if (v != 0.0) {
                s.nnz += 1;
                s.sum += v;
                s.maxv = fmax(s.maxv, v);
                s.max_abs = fmax(s.max_abs, fabs(v));
                s.negative += (v < 0.0);
                s.nonint += (trunc(v) != v);
                s.over127 += (v > 127.0);
            } else {
                s.maxv = fmax(s.maxv, 0.0);
            }
        }
    }
    s = block_reduce(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads)
scan_finalize(const ScanStats* __restrict__ partials, int nb,
              ScanStats* __restrict__ out, int is_rep, int* status) {
    ScanStats s;
    stats_init(s);
    for (int b = threadIdx.x; b < nb; b += kScanThreads)
        stats_merge(s, partials[b]);
    s = block_reduce(s);
    if (threadIdx.x == 0) {
        *out = s;
        if (is_rep && status != nullptr) {
            if (s.negative) atomicCAS(status, 0, (int)AFMM_ERR_NEGATIVE_REP);
            else if (s.nonint) atomicCAS(status, 0, (int)AFMM_ERR_NONINTEGER_REP);
        }
    }
}

// Rep-factor check only (Sec. 2 types: non-negative integers): one read of
// the matrix with 16-byte loads where rows allow, flags reduced per warp,
// one atomic per warp that saw a bad entry.  A negative entry records
// AFMM_ERR_NEGATIVE_REP; otherwise a non-integer (NaN and infinities
// included) records AFMM_ERR_NONINTEGER_REP.
template <int DT>
__device__ __forceinline__ uint32_t rep_flags(typename Elem<DT>::T e) {
    if constexpr (DT == AFMM_U8) {
        return 0u;
    } else if constexpr (DT == AFMM_I8 || DT == AFMM_I32) {
        return e < 0 ? 1u : 0u;
    } else {
        const double v = Elem<DT>::get(&e, 0);
        return (v < 0.0 ? 1u : 0u) | ((!isfinite(v) || trunc(v) != v) ? 2u : 0u);
    }
}

template <int DT>
__global__ void __launch_bounds__(kScanThreads)
rep_check_kernel(const void* __restrict__ M, int64_t n, int64_t ld, int vec, int* status) {
    using T = typename Elem<DT>::T;
    constexpr int V = 16 / (int)sizeof(T);
    const T* m = static_cast<const T*>(M);
    uint32_t bits = 0;
    const int64_t chunks = vec ? n / V : 0;          // whole 16-byte pieces per row
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const T* row = m + r * ld;
        for (int64_t c = threadIdx.x; c < chunks; c += kScanThreads) {
            const uint4 q = reinterpret_cast<const uint4*>(row)[c];
            const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int t = 0; t < V; ++t) bits |= rep_flags<DT>(e[t]);
        }
        for (int64_t c = chunks * V + threadIdx.x; c < n; c += kScanThreads)
            bits |= rep_flags<DT>(row[c]);
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits)
        atomicCAS(status, 0, (int)((bits & 1u) ? AFMM_ERR_NEGATIVE_REP : AFMM_ERR_NONINTEGER_REP));
}

}  // namespace

afmm_status launch_rep_check(const void* M, int dtype, int64_t n, int64_t ld, int* status,
                             cudaStream_t st) {
    if (n <= 0 || dtype == AFMM_U8) return AFMM_OK;      // u8 holds only valid values
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    const int64_t es = (int64_t)dtype_size(dtype);
    const int vec = (reinterpret_cast<uintptr_t>(M) & 15u) == 0 && (ld * es) % 16 == 0;
    const int nb = (int)(n < dp.sm_count * 4 ? n : dp.sm_count * 4);
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        rep_check_kernel<DT><<<nb, kScanThreads, 0, st>>>(M, n, ld, vec, status);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_scan(const void* M, int dtype, int64_t n, int64_t ld,
                        bool is_rep, ScanStats* partials, ScanStats* out,
                        int* status, cudaStream_t st) {
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    int nb = (int)((n < 1) ? 1 : n);
    const int cap = dp.sm_count * 4 < kScanMaxBlocks ? dp.sm_count * 4
                                                     : kScanMaxBlocks;
    if (nb > cap) nb = cap;
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        scan_kernel<DT><<<nb, kScanThreads, 0, st>>>(M, n, ld, partials);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    scan_finalize<<<1, kScanThreads, 0, st>>>(partials, nb, out,
                                              is_rep ? 1 : 0, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return AFMM_OK;
}

}  // namespace afmm
