// Sparse x sparse AFMM product for the quadratic regime of Sec. 2.2: when
// d1 d2 ~ 1/n the paper's addition count mu' d1 d2 n^3 is O(n^2), and the
// work is dominated by reading X and Y and writing Z.
//
// The zero-skip of Sec. 2 is applied to both factors.  Every row of X and of
// Y is compacted to (column, value) pairs in column order:
//   count  one read of the dense factor with 16-byte loads: per row the
//          non-zero count and a bit mask (one bit per entry, n^2/8 bytes),
//          per block of rows the block's total;
//   fill   per row: its offset (the sum of the totals of the blocks before
//          it, then of the rows before it in its block -- a deterministic
//          layout with no separate scan pass), then the mask words are
//          expanded and only the non-zero values are read again.
// The product takes one warp per row i of Z: it walks the non-zero X[i,k]
// in k order, G entries at a time (their Y-row pairs loaded together, so
// that many loads are in flight), and adds X[i,k] * Y[k,j] into a
// shared-memory row of Z, lanes taking distinct j of one Y row (no atomics;
// each Z[i,j] sums its terms in increasing k).  The row is written to Z
// once with 16-byte stores.  Rows wider than the shared-memory row are done
// in column chunks.
#include <cuda_runtime.h>

#include "afmm_common.cuh"
#include "elem.cuh"

namespace afmm {
namespace {

constexpr int SP_ROWS = 8;                  // rows (warps) per count/fill block
constexpr int SP_MAX_CHUNK = 6144;          // floats per warp row buffer
constexpr int SP_G = 8;                     // X entries whose Y rows load together
constexpr int SP_PRE = 3;                   // 32-entry pieces of a Y row loaded ahead
constexpr int SP_MUL_WARPS = 7;             // most warps (rows) per product block
constexpr int SP_UNROLL = 8;                // 16-byte loads in flight per lane (count)

// Non-zero test of one stored element, in the precision the product uses
// (FP64 values are rounded to FP32 first, as the fill does).
template <int DT>
__device__ __forceinline__ bool nz_elem(const typename Elem<DT>::T* v, int e) {
    return (float)Elem<DT>::get(v, e) != 0.f;
}

// Per row r: cnt[r] = non-zeros, mask[r * W + w] bit b = (entry 32 w + b is
// non-zero); bsum[block] = the block's total.  Warp per row.  `vec`: rows
// are 16-byte aligned and n is a multiple of the 16-byte element count.
template <int DT>
__global__ void __launch_bounds__(SP_ROWS * 32)
sp_count_kernel(const void* __restrict__ M, int64_t n, int64_t ld, bool vec,
                uint32_t* __restrict__ mask, int64_t W, int* __restrict__ cnt,
                int64_t* __restrict__ bsum) {
    using T = typename Elem<DT>::T;
    constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte unit
    constexpr int G = 32 / V;               // lanes per 32-bit mask word
    __shared__ int s_cnt[SP_ROWS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * SP_ROWS + w;
    int c = 0;
    if (r < n) {
        uint32_t* mrow = mask + r * W;
        if (vec) {
            const uint4* row = reinterpret_cast<const uint4*>(
                static_cast<const T*>(M) + r * ld);
            const int64_t units = n / V;
            for (int64_t u0 = 0; u0 < units; u0 += 32 * SP_UNROLL) {
                uint4 q[SP_UNROLL];
#pragma unroll
                for (int s = 0; s < SP_UNROLL; ++s) {
                    const int64_t u = u0 + 32 * s + lane;
                    q[s] = u < units ? row[u] : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int s = 0; s < SP_UNROLL; ++s) {
                    const T* e = reinterpret_cast<const T*>(&q[s]);
                    uint32_t nib = 0;
#pragma unroll
                    for (int t = 0; t < V; ++t) nib |= (uint32_t)nz_elem<DT>(e, t) << t;
                    c += __popc(nib);
                    // Mask word: the V-bit groups of G neighbouring lanes.
                    uint32_t word = V == 32 ? nib : nib << ((lane % G) * V);
#pragma unroll
                    for (int o = 1; o < G; o <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
                    const int64_t widx = ((u0 + 32 * s) * V) / 32 + lane / G;
                    if (lane % G == 0 && widx < W) mrow[widx] = word;
                }
            }
            for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        } else {
            const T* row = static_cast<const T*>(M) + r * ld;
            for (int64_t j0 = 0; j0 < n; j0 += 32) {
                const int64_t j = j0 + lane;
                const bool nz = j < n && (float)Elem<DT>::get(row, j) != 0.f;
                const uint32_t word = __ballot_sync(0xffffffffu, nz);
                c += __popc(word);
                if (lane == 0) mrow[j0 / 32] = word;
            }
        }
    }
    if (lane == 0) s_cnt[w] = c;
    if (lane == 0 && r < n) cnt[r] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int i = 0; i < SP_ROWS; ++i) s += s_cnt[i];
        bsum[blockIdx.x] = s;
    }
}

// Row r's non-zeros as (column, FP32 value bits) pairs at ptr[r] .. in
// column order; ptr[n] = the total.  Rows past `cap` entries record
// AFMM_ERR_OVERFLOW_RISK.  Same row-to-block map as the count.
template <int DT>
__global__ void __launch_bounds__(SP_ROWS * 32)
sp_fill_kernel(const void* __restrict__ M, int64_t n, int64_t ld,
               const uint32_t* __restrict__ mask, int64_t W, const int* __restrict__ cnt,
               const int64_t* __restrict__ bsum, int64_t* __restrict__ ptr, int64_t cap,
               uint2* __restrict__ ent, int* status) {
    using T = typename Elem<DT>::T;
    __shared__ int64_t s_red[SP_ROWS * 32];
    __shared__ int s_cnt[SP_ROWS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * SP_ROWS, r = r0 + w;
    // Offset of this block: the totals of all blocks before it.
    int64_t part = 0;
    for (int64_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) part += bsum[b];
    s_red[threadIdx.x] = part;
    if (lane == 0) s_cnt[w] = r < n ? cnt[r] : 0;
    __syncthreads();
    for (int s = SP_ROWS * 16; s; s >>= 1) {
        if (threadIdx.x < s) s_red[threadIdx.x] += s_red[threadIdx.x + s];
        __syncthreads();
    }
    if (r >= n) return;
    int64_t off = s_red[0];
    for (int i = 0; i < w; ++i) off += s_cnt[i];
    const int c = s_cnt[w];
    if (lane == 0) {
        ptr[r] = off;
        if (r == n - 1) ptr[n] = off + c;
    }
    if (off + c > cap) {
        if (lane == 0) atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
        return;
    }
    const T* row = static_cast<const T*>(M) + r * ld;
    const uint32_t* mrow = mask + r * W;
    for (int64_t w0 = 0; w0 < W; w0 += 32) {
        uint32_t word = w0 + lane < W ? mrow[w0 + lane] : 0u;
        const int pc = __popc(word);
        int incl = pc;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int64_t o = off + incl - pc;
        const int64_t jb = (w0 + lane) * 32;
        // Up to four set bits per lane per round: their loads issue together.
        while (__any_sync(0xffffffffu, word != 0)) {
            int64_t j[4];
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                j[q] = -1;
                if (word) {
                    j[q] = jb + __ffs(word) - 1;
                    word &= word - 1;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[q] = j[q] >= 0 ? (float)Elem<DT>::get(row, j[q]) : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j[q] >= 0) ent[o++] = make_uint2((uint32_t)j[q], __float_as_uint(v[q]));
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// First index in [lo, hi) whose column is >= c (columns increase).
__device__ __forceinline__ int64_t lower_col(const uint2* __restrict__ e, int64_t lo,
                                             int64_t hi, int64_t c) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)e[mid].x < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Z row i (warp per row), columns [c0, c0 + chunk) per pass.  At most
// SP_MUL_WARPS warps per block and two blocks per SM (register cap).
__global__ void __launch_bounds__(SP_MUL_WARPS * 32, 2)
sp_mul_kernel(const int64_t* __restrict__ px, const uint2* __restrict__ ex,
              const int64_t* __restrict__ py, const uint2* __restrict__ ey, int64_t n,
              int chunk, int warps, float* __restrict__ Z, int64_t ldz, bool zvec,
              const int* status) {
    extern __shared__ __align__(16) float srow[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * warps + w;
    if (i >= n || *status != 0) return;
    float* acc = srow + (int64_t)w * chunk;
    float4* acc4 = reinterpret_cast<float4*>(acc);
    const int64_t xb = px[i], xe = px[i + 1];
    float* zr = Z + i * ldz;
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t c1 = c0 + chunk < n ? c0 + chunk : n;
        const bool narrow = c0 > 0 || c1 < n;
        for (int j = lane; j < chunk / 4; j += 32) acc4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        for (int64_t e0 = xb; e0 < xe; e0 += 64) {
            const int m = xe - e0 < 64 ? (int)(xe - e0) : 64;
            // Lane t holds entries e0 + t and e0 + 32 + t: x, and the span
            // [yb, yb + yl) of Y row k inside [c0, c1).
            float xv[2] = {0.f, 0.f};
            int64_t yb[2] = {0, 0};
            int yl[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (lane + 32 * h < m) {
                    const uint2 e = ex[e0 + lane + 32 * h];
                    xv[h] = __uint_as_float(e.y);
                    int64_t b = py[e.x], en = py[e.x + 1];
                    if (narrow) {
                        b = lower_col(ey, b, en, c0);
                        en = lower_col(ey, b, en, c1);
                    }
                    yb[h] = b;
                    yl[h] = (int)(en - b);
                }
            }
            for (int t = 0; t < m; t += SP_G) {
                // Entries t .. t+G-1 (all in one half: G divides 32).
                const int h = t >> 5;
                const float xh = h ? xv[1] : xv[0];
                const int64_t bh = h ? yb[1] : yb[0];
                const int lh = h ? yl[1] : yl[0];
                uint2 a[SP_G][SP_PRE];
                float xs[SP_G];
                const uint2* yp[SP_G];
                int len[SP_G];
#pragma unroll
                for (int u = 0; u < SP_G; ++u) {
                    const int src = (t + u) & 31;
                    xs[u] = __shfl_sync(0xffffffffu, xh, src);
                    yp[u] = ey + __shfl_sync(0xffffffffu, bh, src);
                    len[u] = t + u < m ? __shfl_sync(0xffffffffu, lh, src) : 0;
#pragma unroll
                    for (int c = 0; c < SP_PRE; ++c)
                        a[u][c] = lane + 32 * c < len[u] ? __ldg(yp[u] + lane + 32 * c)
                                                         : make_uint2(0, 0);
                }
#pragma unroll
                for (int u = 0; u < SP_G; ++u) {
#pragma unroll
                    for (int c = 0; c < SP_PRE; ++c) {
                        if (lane + 32 * c < len[u]) {
                            float* d = acc + ((int64_t)a[u][c].x - c0);
                            *d = fmaf(xs[u], __uint_as_float(a[u][c].y), *d);
                        }
                    }
#pragma unroll 4
                    for (int f = lane + 32 * SP_PRE; f < len[u]; f += 32) {
                        const uint2 y = __ldg(yp[u] + f);
                        float* d = acc + ((int64_t)y.x - c0);
                        *d = fmaf(xs[u], __uint_as_float(y.y), *d);
                    }
                    __syncwarp();          // entry u's terms land before entry u+1's
                }
            }
        }
        const int64_t cw = c1 - c0;
        if (zvec) {
            float4* z4 = reinterpret_cast<float4*>(zr + c0);
            for (int64_t j = lane; j < cw / 4; j += 32) __stcs(z4 + j, acc4[j]);
            for (int64_t j = (cw & ~3LL) + lane; j < cw; j += 32) zr[c0 + j] = acc[j];
        } else {
            for (int64_t j = lane; j < cw; j += 32) zr[c0 + j] = acc[j];
        }
        __syncwarp();
    }
}

struct SparseWs {
    uint32_t* mask[2];
    int* cnt[2];
    int64_t* bsum[2];
    int64_t* ptr[2];
    uint2* ent[2];
};

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

size_t sparse_layout(int64_t n, int64_t cap_x, int64_t cap_y, char* base, SparseWs* o) {
    const int64_t W = (n + 31) / 32, nb = (n + SP_ROWS - 1) / SP_ROWS;
    size_t top = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + top : nullptr;
        top += up256(bytes);
        return p;
    };
    for (int m = 0; m < 2; ++m) {
        const int64_t cap = m == 0 ? cap_x : cap_y;
        SparseWs t;
        t.mask[m] = reinterpret_cast<uint32_t*>(take((size_t)n * W * 4));
        t.cnt[m] = reinterpret_cast<int*>(take((size_t)n * 4));
        t.bsum[m] = reinterpret_cast<int64_t*>(take((size_t)nb * 8));
        t.ptr[m] = reinterpret_cast<int64_t*>(take((size_t)(n + 1) * 8));
        t.ent[m] = reinterpret_cast<uint2*>(take((size_t)cap * 8));
        if (o) {
            o->mask[m] = t.mask[m];
            o->cnt[m] = t.cnt[m];
            o->bsum[m] = t.bsum[m];
            o->ptr[m] = t.ptr[m];
            o->ent[m] = t.ent[m];
        }
    }
    return top;
}

// Count + fill of one factor into CSR pairs.
afmm_status compact(const void* M, int dt, int64_t ld, int64_t n, int64_t cap,
                    const SparseWs& ws, int m, int* status, cudaStream_t st) {
    const int64_t W = (n + 31) / 32;
    const unsigned nb = (unsigned)((n + SP_ROWS - 1) / SP_ROWS);
    const size_t es = dtype_size(dt);
    const int64_t V = 16 / (int64_t)es;
    const bool vec = (reinterpret_cast<uintptr_t>(M) % 16 == 0) && ((ld * es) % 16 == 0) &&
                     (n % V == 0);
    return dispatch_dtype(dt, [&]<int DT>() -> afmm_status {
        sp_count_kernel<DT><<<nb, SP_ROWS * 32, 0, st>>>(M, n, ld, vec, ws.mask[m], W,
                                                         ws.cnt[m], ws.bsum[m]);
        sp_fill_kernel<DT><<<nb, SP_ROWS * 32, 0, st>>>(M, n, ld, ws.mask[m], W, ws.cnt[m],
                                                        ws.bsum[m], ws.ptr[m], cap,
                                                        ws.ent[m], status);
        AFMM_CUDA_TRY(cudaGetLastError());
        return AFMM_OK;
    });
}

}  // namespace

size_t sparse_ws_bytes(int64_t n, int64_t cap_x, int64_t cap_y) {
    return sparse_layout(n, cap_x, cap_y, nullptr, nullptr);
}

afmm_status launch_sparse(const void* X, int xdt, int64_t ldx, const void* Y, int ydt,
                          int64_t ldy, float* Z, int64_t ldz, int64_t n, int64_t cap_x,
                          int64_t cap_y, void* ws, int* status, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    SparseWs L;
    sparse_layout(n, cap_x, cap_y, static_cast<char*>(ws), &L);
    AFMM_TRY(compact(X, xdt, ldx, n, cap_x, L, 0, status, st));
    AFMM_TRY(compact(Y, ydt, ldy, n, cap_y, L, 1, status, st));
    const int chunk = (int)(n < SP_MAX_CHUNK ? (n + 31) / 32 * 32 : SP_MAX_CHUNK);
    // Warps per block: two blocks fit in one SM's shared memory.
    int warps = (int)((113 * 1024) / ((size_t)chunk * sizeof(float)));
    warps = warps < 1 ? 1 : (warps > SP_MUL_WARPS ? SP_MUL_WARPS : warps);
    const size_t smem = (size_t)warps * chunk * sizeof(float);
    AFMM_CUDA_TRY(cudaFuncSetAttribute(sp_mul_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    const bool zvec = reinterpret_cast<uintptr_t>(Z) % 16 == 0 && ldz % 4 == 0;
    const unsigned blocks = (unsigned)((n + warps - 1) / warps);
    main_kernel_begin(st);
    sp_mul_kernel<<<blocks, warps * 32, smem, st>>>(L.ptr[0], L.ent[0], L.ptr[1], L.ent[1], n,
                                                    chunk, warps, Z, ldz, zvec, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, (int)blocks);
    count_launches(5);
    return AFMM_OK;
}

}  // namespace afmm
