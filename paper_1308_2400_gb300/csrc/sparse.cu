// Sparse x sparse AFMM product for the quadratic regime of Sec. 2.2: when
// d1 d2 ~ 1/n the paper's addition count mu' d1 d2 n^3 is O(n^2), and the
// work is dominated by reading X and Y and writing Z.
//
// The zero-skip of Sec. 2 is applied to both factors: every row of X and
// of Y is compacted to (column, value) lists in column order (one warp per
// row: ballot + prefix popcount, so the order is deterministic), then one
// warp per output row i walks the non-zero X[i,k] in k order and adds
// X[i,k] * Y[k,j] for the non-zero Y[k,j] into a shared-memory row of Z,
// lanes taking distinct j (no atomics, fixed summation order); the row is
// written to Z once, coalesced.  Rows wider than the shared-memory row are
// done in column chunks.
#include <cuda_runtime.h>

#include "afmm_common.cuh"
#include "bf16_split.cuh"

namespace afmm {
namespace {

constexpr int SP_WARPS = 8;                 // rows per block in the product
constexpr int SP_MAX_CHUNK = 6144;          // floats per warp row buffer

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// cnt[r] = non-zero entries of row r (warp per row).
__global__ void __launch_bounds__(256)
sp_count_kernel(const void* __restrict__ M, int dt, int64_t n, int64_t ld,
                int* __restrict__ cnt) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    int c = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        const int64_t j = j0 + lane;
        const bool nz = j < n && load_any_f(M, r * ld + j, dt) != 0.f;
        c += __popc(__ballot_sync(0xffffffffu, nz));
    }
    if (lane == 0) cnt[r] = c;
}

// ptr[0] = 0, ptr[r+1] = ptr[r] + cnt[r]; one block, sequential chunks.
__global__ void __launch_bounds__(1024)
sp_scan_kernel(const int* __restrict__ cnt, int64_t n, int64_t* __restrict__ ptr) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) {
        carry = 0;
        ptr[0] = 0;
    }
    __syncthreads();
    for (int64_t b = 0; b < n; b += 1024) {
        const int64_t i = b + threadIdx.x;
        part[threadIdx.x] = i < n ? cnt[i] : 0;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {          // inclusive scan
            const int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < n) ptr[i + 1] = carry + part[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
}

// Row r's non-zeros, in column order, at ptr[r] ..: col and value (FP32).
// A row that would run past `cap` entries records AFMM_ERR_OVERFLOW_RISK.
__global__ void __launch_bounds__(256)
sp_fill_kernel(const void* __restrict__ M, int dt, int64_t n, int64_t ld,
               const int64_t* __restrict__ ptr, int64_t cap, int* __restrict__ col,
               float* __restrict__ val, int* status) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    int64_t o = ptr[r];
    if (ptr[r + 1] > cap) {
        if (lane == 0) atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
        return;
    }
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        const int64_t j = j0 + lane;
        const float v = j < n ? load_any_f(M, r * ld + j, dt) : 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, v != 0.f);
        if (v != 0.f) {
            const int64_t p = o + __popc(m & lanemask_lt());
            col[p] = (int)j;
            val[p] = v;
        }
        o += __popc(m);
    }
}

// Z row i (warp per row), columns [c0, c0 + chunk) per pass.
__global__ void __launch_bounds__(SP_WARPS * 32)
sp_mul_kernel(const int64_t* __restrict__ px, const int* __restrict__ cx,
              const float* __restrict__ vx, const int64_t* __restrict__ py,
              const int* __restrict__ cy, const float* __restrict__ vy, int64_t n,
              int chunk, float* __restrict__ Z, int64_t ldz, const int* status) {
    extern __shared__ float srow[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * SP_WARPS + w;
    if (i >= n || *status != 0) return;
    float* acc = srow + (int64_t)w * chunk;
    const int64_t xb = px[i], xe = px[i + 1];
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t c1 = c0 + chunk < n ? c0 + chunk : n;
        for (int64_t j = c0 + lane; j < c1; j += 32) acc[j - c0] = 0.f;
        __syncwarp();
        for (int64_t e = xb; e < xe; ++e) {           // k in increasing order
            const int k = cx[e];
            const float x = vx[e];
            int64_t yb = py[k], ye = py[k + 1];
            if (c0 > 0 || c1 < n) {                    // narrow to [c0, c1)
                int64_t lo = yb, hi = ye;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (cy[mid] < c0) lo = mid + 1; else hi = mid;
                }
                yb = lo;
                hi = ye;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (cy[mid] < c1) lo = mid + 1; else hi = mid;
                }
                ye = lo;
            }
            for (int64_t f = yb + lane; f < ye; f += 32)
                acc[cy[f] - c0] = fmaf(x, vy[f], acc[cy[f] - c0]);
            __syncwarp();
        }
        float* zr = Z + i * ldz;
        for (int64_t j = c0 + lane; j < c1; j += 32) zr[j] = acc[j - c0];
        __syncwarp();
    }
}

}  // namespace

size_t sparse_ws_bytes(int64_t n, int64_t cap_x, int64_t cap_y) {
    const size_t a = 256;
    auto up = [&](size_t b) { return (b + a - 1) / a * a; };
    return up(n * 4) * 2 + up((n + 1) * 8) * 2 + up(cap_x * 8) + up(cap_y * 8);
}

afmm_status launch_sparse(const void* X, int xdt, int64_t ldx, const void* Y, int ydt,
                          int64_t ldy, float* Z, int64_t ldz, int64_t n, int64_t cap_x,
                          int64_t cap_y, void* ws, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    const size_t a = 256;
    auto up = [&](size_t b) { return (b + a - 1) / a * a; };
    char* p = static_cast<char*>(ws);
    int* cnt_x = reinterpret_cast<int*>(p); p += up(n * 4);
    int* cnt_y = reinterpret_cast<int*>(p); p += up(n * 4);
    int64_t* ptr_x = reinterpret_cast<int64_t*>(p); p += up((n + 1) * 8);
    int64_t* ptr_y = reinterpret_cast<int64_t*>(p); p += up((n + 1) * 8);
    // Per factor: column indices (cap * 4 bytes), then values (cap * 4).
    int* col_x = reinterpret_cast<int*>(p);
    float* val_x = reinterpret_cast<float*>(p + cap_x * 4);
    p += up(cap_x * 8);
    int* col_y = reinterpret_cast<int*>(p);
    float* val_y = reinterpret_cast<float*>(p + cap_y * 4);
    const unsigned rb = (unsigned)((n + 7) / 8);
    sp_count_kernel<<<rb, 256, 0, st>>>(X, xdt, n, ldx, cnt_x);
    sp_count_kernel<<<rb, 256, 0, st>>>(Y, ydt, n, ldy, cnt_y);
    sp_scan_kernel<<<1, 1024, 0, st>>>(cnt_x, n, ptr_x);
    sp_scan_kernel<<<1, 1024, 0, st>>>(cnt_y, n, ptr_y);
    sp_fill_kernel<<<rb, 256, 0, st>>>(X, xdt, n, ldx, ptr_x, cap_x, col_x, val_x, status);
    sp_fill_kernel<<<rb, 256, 0, st>>>(Y, ydt, n, ldy, ptr_y, cap_y, col_y, val_y, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    const int chunk = (int)(n < SP_MAX_CHUNK ? (n + 31) / 32 * 32 : SP_MAX_CHUNK);
    const size_t smem = (size_t)SP_WARPS * chunk * sizeof(float);
    AFMM_CUDA_TRY(cudaFuncSetAttribute(sp_mul_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    main_kernel_begin(st);
    sp_mul_kernel<<<(unsigned)((n + SP_WARPS - 1) / SP_WARPS), SP_WARPS * 32, smem, st>>>(
        ptr_x, col_x, val_x, ptr_y, col_y, val_y, n, chunk, Z, ldz, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, (int)((n + SP_WARPS - 1) / SP_WARPS));
    count_launches(7);
    return AFMM_OK;
}

}  // namespace afmm
