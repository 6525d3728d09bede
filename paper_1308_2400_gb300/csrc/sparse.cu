// Sparse x sparse AFMM product for the quadratic regime of Sec. 2.2: when
// d1 d2 ~ 1/n the paper's addition count mu' d1 d2 n^3 is O(n^2), and the
// work is dominated by reading X and Y and writing Z.
//
// The zero-skip of Sec. 2 is applied to both factors.  Every row of X and of
// Y is compacted to (column, FP32 value) pairs in column order, in one read
// of the dense factor: one warp per row, 16-byte loads, the non-zeros of
// each 16-byte piece placed by a warp prefix sum of their counts, and
// written straight from registers into the row's slot of R pairs (R from
// the density hint: the expected row count plus six standard deviations).
// A row with more than R non-zeros -- possible when the density is uneven
// -- is compacted again by its warp, whole, into an overflow region.  The
// compaction also records, per row, how many pairs fall before each
// column-chunk boundary.  X and Y are compacted by one launch.
//
// The product takes one warp per (row i, column chunk) of Z: it walks the
// non-zero X[i,k] in k order, G entries at a time (the chunk's pairs of
// their Y rows loaded together, so that many loads are in flight), and
// adds X[i,k] * Y[k,j] into a shared-memory row piece of Z, lanes taking
// distinct j of one Y row (no atomics; each Z[i,j] sums its terms in
// increasing k).  The piece is written to Z once with 16-byte stores.
#include <cuda_runtime.h>

#include <cmath>

#include "afmm_common.cuh"
#include "elem.cuh"

namespace afmm {
namespace {

constexpr int SP_ROWS = 8;                  // warps (rows) per compaction block
constexpr int SP_CW = 6144;                 // widest Z row piece a product warp holds
constexpr int SP_G = 8;                     // X entries whose Y pairs load together
constexpr int SP_PRE = 2;                   // 16-byte loads (2 pairs) per lane loaded ahead
constexpr int SP_MUL_WARPS = 7;             // most warps per product block
constexpr int SP_UNROLL = 4;                // 16-byte loads per lane and round (two rounds in flight)

// One factor's compaction.  Row r's pairs start at ptr[r] (r * R, or in the
// overflow region after the n * R slots) and number cnt[r]; spl[r * (C-1) +
// b - 1] = pairs of row r with column < b * SP_CW (b = 1 .. C-1).
struct SpMat {
    const void* M;
    int64_t ld;
    int vec;              // rows 16-byte aligned and n a multiple of 16 bytes
    int rep;              // the factor holds Rep-factors: check them (Sec. 2 types)
    int R;                // slot size (pairs per row)
    uint2* ent;           // n * R slots, then ovf_cap overflow pairs
    int64_t ovf_cap;
    int* cnt;
    int64_t* ptr;
    int* spl;
};
struct SpArgs {
    SpMat m[2];           // X, Y
    int64_t n;
    int C;                // column chunks of the product
    unsigned long long* ovf_used;   // two counters, zero before a compaction
    int* status;
};

// Non-zero test of one stored element, in the precision the product uses
// (FP64 values are rounded to FP32 first, like the stored value).
template <int DT>
__device__ __forceinline__ bool nz_elem(const typename Elem<DT>::T* v, int e) {
    return (float)Elem<DT>::get(v, e) != 0.f;
}

// Rep-factor check bits of one stored element: 1 negative, 2 not an
// integer (NaN and infinities included).
template <int DT>
__device__ __forceinline__ uint32_t rep_check_bits(const typename Elem<DT>::T* v, int e) {
    if constexpr (DT == AFMM_U8) {
        return 0u;
    } else if constexpr (DT == AFMM_I8 || DT == AFMM_I32) {
        return v[e] < 0 ? 1u : 0u;
    } else {
        const double x = Elem<DT>::get(v, e);
        return (x < 0.0 ? 1u : 0u) | ((!isfinite(x) || trunc(x) != x) ? 2u : 0u);
    }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Row r of one factor: the first R pairs into its slot, the count, the
// chunk split counts; a longer row, whole, into the overflow region.
template <int DT>
__device__ __forceinline__ void compact_row(const SpArgs& a, const SpMat& A, int mi, int64_t r,
                                            int lane) {
    using T = typename Elem<DT>::T;
    constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte piece
    const int64_t n = a.n;
    uint2* out = A.ent + r * A.R;
    const int R = A.R;
    int* spl = A.spl + r * (a.C - 1);
    const T* row = static_cast<const T*>(A.M) + r * A.ld;
    int c = 0;
    uint32_t bad = 0;
    if (A.vec) {
        const uint4* row4 = reinterpret_cast<const uint4*>(row);
        const int64_t units = n / V;
        // The next round of 16-byte pieces is loaded while this one is
        // placed, so the row streams in without gaps.
        uint4 q[SP_UNROLL], qn[SP_UNROLL];
#pragma unroll
        for (int s = 0; s < SP_UNROLL; ++s) {
            const int64_t u = 32 * s + lane;
            q[s] = u < units ? row4[u] : make_uint4(0, 0, 0, 0);
        }
        for (int64_t u0 = 0; u0 < units; u0 += 32 * SP_UNROLL) {
            const int64_t un = u0 + 32 * SP_UNROLL;
            if (un < units) {
#pragma unroll
                for (int s = 0; s < SP_UNROLL; ++s) {
                    const int64_t u = un + 32 * s + lane;
                    qn[s] = u < units ? row4[u] : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int s = 0; s < SP_UNROLL; ++s) {
                const int64_t col0 = (u0 + 32 * s) * V;      // first column of the 32 pieces
                if (col0 > 0 && col0 < n && col0 % SP_CW == 0 && lane == 0)
                    spl[col0 / SP_CW - 1] = c;
                const T* e = reinterpret_cast<const T*>(&q[s]);
                uint32_t nib = 0;
#pragma unroll
                for (int t = 0; t < V; ++t) nib |= (uint32_t)nz_elem<DT>(e, t) << t;
                if (A.rep) {
#pragma unroll
                    for (int t = 0; t < V; ++t) bad |= rep_check_bits<DT>(e, t);
                }
                const unsigned any = __ballot_sync(0xffffffffu, nib != 0);
                if (any == 0) continue;
                const int pc = __popc(nib);
                int excl, tot;
                if (__ballot_sync(0xffffffffu, pc > 1) == 0) {   // at most one per piece
                    excl = __popc(any & lanemask_lt());
                    tot = __popc(any);
                } else {
                    int incl = pc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += t;
                    }
                    excl = incl - pc;
                    tot = __shfl_sync(0xffffffffu, incl, 31);
                }
                if (nib) {
                    int pos = c + excl;
                    const int64_t j0 = col0 + (int64_t)lane * V;
#pragma unroll
                    for (int t = 0; t < V; ++t) {
                        if ((nib >> t) & 1u) {
                            if (pos < R)
                                out[pos] = make_uint2((uint32_t)(j0 + t),
                                                      __float_as_uint((float)Elem<DT>::get(e, t)));
                            ++pos;
                        }
                    }
                }
                c += tot;
            }
#pragma unroll
            for (int s = 0; s < SP_UNROLL; ++s) q[s] = qn[s];
        }
    } else {
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            if (j0 > 0 && j0 % SP_CW == 0 && lane == 0) spl[j0 / SP_CW - 1] = c;
            const int64_t j = j0 + lane;
            if (A.rep && j < n) bad |= rep_check_bits<DT>(row, (int)j);
            const float v = j < n ? (float)Elem<DT>::get(row, j) : 0.f;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0.f);
            if (v != 0.f) {
                const int pos = c + __popc(m & lanemask_lt());
                if (pos < R) out[pos] = make_uint2((uint32_t)j, __float_as_uint(v));
            }
            c += __popc(m);
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && lane == 0)
        atomicCAS(a.status, 0, (int)((bad & 1u) ? AFMM_ERR_NEGATIVE_REP : AFMM_ERR_NONINTEGER_REP));
    int64_t start = r * (int64_t)R;
    if (c > R) {
        // Longer than the slot: the whole row into the overflow region.
        // Even counts keep every row start 16-byte aligned.
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.ovf_used + mi, (unsigned long long)((c + 1) & ~1));
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)(base + c) > A.ovf_cap) {
            if (lane == 0) atomicCAS(a.status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
            return;
        }
        start = n * (int64_t)R + (int64_t)base;
        uint2* o = A.ent + start;
        int pos = 0;
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            const int64_t j = j0 + lane;
            const float v = j < n ? (float)Elem<DT>::get(row, j) : 0.f;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0.f);
            if (v != 0.f) {
                const int p = pos + __popc(m & lanemask_lt());
                if (p < c) o[p] = make_uint2((uint32_t)j, __float_as_uint(v));
            }
            pos += __popc(m);
        }
    }
    if (lane == 0) {
        A.cnt[r] = c;
        A.ptr[r] = start;
    }
}

// blockIdx.y = 0: rows of X, 1: rows of Y; one warp per row.
template <int DTX, int DTY>
__global__ void __launch_bounds__(SP_ROWS * 32) sp_compact_kernel(SpArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * SP_ROWS + (threadIdx.x >> 5);
    if (r >= a.n) return;
    if (blockIdx.y == 0) compact_row<DTX>(a, a.m[0], 0, r, lane);
    else compact_row<DTY>(a, a.m[1], 1, r, lane);
}

struct SpMul {
    const int64_t* px;
    const int* nx;
    const uint2* ex;
    const int64_t* py;
    const int* ny;
    const uint2* ey;
    const int* sy;        // Y split counts, C - 1 per row
    int64_t n;
    int C, warps, row_floats;
    float* Z;
    int64_t ldz;
    int zvec;
    const int* status;
    unsigned long long* ovf_used;
};

// Z[i, c0 : c0 + SP_CW) for one warp (the whole row when n <= SP_CW),
// accumulated in shared memory.  IT indexes the pairs (int when they
// number fewer than 2^31).  Pairs are read two at a time with 16-byte loads
// from the even index at or below a span's start; pairs outside the span
// are masked (every slot and overflow row starts at an even index).
template <typename IT>
__global__ void __launch_bounds__(SP_MUL_WARPS * 32, 2)
sp_mul_kernel(SpMul a) {
    extern __shared__ __align__(16) float srow[];
    // The compaction is complete (stream order): its counters are reset here
    // for the next call, before anything can return.
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ovf_used[0] = 0;
        a.ovf_used[1] = 0;
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * a.warps + w;
    const int64_t i = item / a.C;
    const int cc = (int)(item % a.C);
    if (i >= a.n || *a.status != 0) return;
    const int64_t c0 = (int64_t)cc * SP_CW;
    const int64_t c1 = c0 + SP_CW < a.n ? c0 + SP_CW : a.n;
    const int cw = (int)(c1 - c0), cw4 = (cw + 3) / 4;
    float* acc = srow + w * a.row_floats;
    float4* acc4 = reinterpret_cast<float4*>(acc);
    for (int j = lane; j < cw4; j += 32) acc4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    const uint4* ey4 = reinterpret_cast<const uint4*>(a.ey);
    const int64_t xb = a.px[i], xe = xb + a.nx[i];
    const int S = a.C - 1;
    for (int64_t e0 = xb; e0 < xe; e0 += 32) {
        const int m = xe - e0 < 32 ? (int)(xe - e0) : 32;
        // Lane t holds entry e0 + t: x and the span [ys, ye) of Y row k's
        // pairs inside the column piece.
        float xv = 0.f;
        IT ys = 0, ye = 0;
        if (lane < m) {
            const uint2 e = a.ex[e0 + lane];
            xv = __uint_as_float(e.y);
            const int64_t k = e.x;
            const IT b = (IT)a.py[k];
            int lo = 0, hi = a.ny[k];
            if (S > 0) {
                if (cc > 0) lo = a.sy[k * S + cc - 1];
                if (cc < S) hi = a.sy[k * S + cc];
            }
            ys = b + lo;
            ye = b + hi;
        }
        for (int t = 0; t < m; t += SP_G) {
            uint4 p[SP_G][SP_PRE];
            float xs[SP_G];
            IT s0[SP_G], s1[SP_G];
#pragma unroll
            for (int u = 0; u < SP_G; ++u) {
                const int src = (t + u) & 31;
                xs[u] = __shfl_sync(0xffffffffu, xv, src);
                s0[u] = __shfl_sync(0xffffffffu, ys, src);
                s1[u] = __shfl_sync(0xffffffffu, ye, src);
                if (t + u >= m) s1[u] = s0[u];
                const IT al = s0[u] & ~(IT)1;
#pragma unroll
                for (int q = 0; q < SP_PRE; ++q) {
                    const IT f = al + 2 * (lane + 32 * q);
                    p[u][q] = f < s1[u] ? __ldg(ey4 + (f >> 1)) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < SP_G; ++u) {
                const IT al = s0[u] & ~(IT)1;
                // This lane's pairs of entry u have distinct columns: read
                // all the Z values first, then write them.
                float v[SP_PRE][2];
                bool ok[SP_PRE][2];
#pragma unroll
                for (int q = 0; q < SP_PRE; ++q) {
                    const IT f = al + 2 * (lane + 32 * q);
                    ok[q][0] = f >= s0[u] && f < s1[u];
                    ok[q][1] = f + 1 < s1[u];
                    v[q][0] = ok[q][0] ? acc[(int)p[u][q].x - (int)c0] : 0.f;
                    v[q][1] = ok[q][1] ? acc[(int)p[u][q].z - (int)c0] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < SP_PRE; ++q) {
                    if (ok[q][0])
                        acc[(int)p[u][q].x - (int)c0] =
                            fmaf(xs[u], __uint_as_float(p[u][q].y), v[q][0]);
                    if (ok[q][1])
                        acc[(int)p[u][q].z - (int)c0] =
                            fmaf(xs[u], __uint_as_float(p[u][q].w), v[q][1]);
                }
                for (IT f = al + 2 * (lane + 32 * SP_PRE); f < s1[u]; f += 64) {
                    const uint4 y = __ldg(ey4 + (f >> 1));
                    const bool ok1 = f + 1 < s1[u];
                    const float z0 = acc[(int)y.x - (int)c0];
                    const float z1 = ok1 ? acc[(int)y.z - (int)c0] : 0.f;
                    acc[(int)y.x - (int)c0] = fmaf(xs[u], __uint_as_float(y.y), z0);
                    if (ok1) acc[(int)y.z - (int)c0] = fmaf(xs[u], __uint_as_float(y.w), z1);
                }
                __syncwarp();          // entry u's terms land before entry u+1's
            }
        }
    }
    float* zr = a.Z + i * a.ldz + c0;
    if (a.zvec) {
        float4* z4 = reinterpret_cast<float4*>(zr);
        for (int j = lane; j < cw / 4; j += 32) __stcs(z4 + j, acc4[j]);
        for (int j = (cw & ~3) + lane; j < cw; j += 32) zr[j] = acc[j];
    } else {
        for (int j = lane; j < cw; j += 32) zr[j] = acc[j];
    }
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

int chunks_of(int64_t n) { return (int)((n + SP_CW - 1) / SP_CW); }

// Slot size R and overflow capacity of a factor with density hint d (< 0:
// unknown, R = n and no overflow).
void sparse_shape(int64_t n, double d, int* R, int64_t* ovf) {
    *R = (int)n;
    *ovf = 0;
    if (!(d >= 0.0)) return;
    const double mu = d * (double)n;
    const double want = std::ceil((mu + 6.0 * std::sqrt(mu) + 16.0) / 32.0) * 32.0;
    if (want >= (double)n) return;
    *R = (int)want;
    const double n2 = (double)n * (double)n;
    const double c = 2.0 * d * n2 + 32.0 * (double)n + 1024.0;
    *ovf = (int64_t)(c < n2 ? c : n2);
}

// Workspace: the two overflow counters; per factor the slots and overflow
// pairs, counts, row starts and chunk split counts.
size_t sparse_layout(int64_t n, double d1, double d2, char* base, SpArgs* o) {
    size_t top = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + top : nullptr;
        top += up256(bytes);
        return p;
    };
    unsigned long long* used = reinterpret_cast<unsigned long long*>(take(16));
    if (o) o->ovf_used = used;
    const int C = chunks_of(n);
    for (int m = 0; m < 2; ++m) {
        int R;
        int64_t ovf;
        sparse_shape(n, m == 0 ? d1 : d2, &R, &ovf);
        SpMat t{};
        t.R = R;
        t.ovf_cap = ovf;
        // Two spare pairs: a 16-byte load at a span's last odd index stays inside.
        t.ent = reinterpret_cast<uint2*>(take(((size_t)n * R + ovf + 2) * 8));
        t.cnt = reinterpret_cast<int*>(take((size_t)n * 4));
        t.ptr = reinterpret_cast<int64_t*>(take((size_t)n * 8));
        t.spl = reinterpret_cast<int*>(take((size_t)n * (C - 1) * 4 + 4));
        if (o) o->m[m] = t;
    }
    return top;
}

bool rows_vec(const void* M, int dt, int64_t ld, int64_t n) {
    const size_t es = dtype_size(dt);
    return reinterpret_cast<uintptr_t>(M) % 16 == 0 && (ld * es) % 16 == 0 &&
           n % (int64_t)(16 / es) == 0;
}

}  // namespace

size_t sparse_ws_bytes(int64_t n, double d1, double d2) {
    return sparse_layout(n, d1, d2, nullptr, nullptr);
}

afmm_status sparse_reset(void* ws, cudaStream_t st) {
    // The overflow counters sit at the start of the workspace.
    AFMM_CUDA_TRY(cudaMemsetAsync(ws, 0, 16, st));
    return AFMM_OK;
}

afmm_status launch_sparse(const void* X, int xdt, int64_t ldx, const void* Y, int ydt,
                          int64_t ldy, float* Z, int64_t ldz, int64_t n, double d1,
                          double d2, void* ws, int* status, cudaStream_t st, int rep_which) {
    if (n <= 0) return AFMM_OK;
    SpArgs a{};
    sparse_layout(n, d1, d2, static_cast<char*>(ws), &a);
    a.n = n;
    a.C = chunks_of(n);
    a.status = status;
    a.m[0].M = X;
    a.m[0].ld = ldx;
    a.m[0].vec = rows_vec(X, xdt, ldx, n);
    a.m[1].M = Y;
    a.m[1].ld = ldy;
    a.m[1].vec = rows_vec(Y, ydt, ldy, n);
    a.m[0].rep = rep_which == 0;
    a.m[1].rep = rep_which == 1;
    // Compaction: one warp per row of X (grid.y = 0) and of Y (grid.y = 1).
    const dim3 grid((unsigned)((n + SP_ROWS - 1) / SP_ROWS), 2);
    AFMM_TRY(dispatch_dtype(xdt, [&]<int DTX>() -> afmm_status {
        return dispatch_dtype(ydt, [&]<int DTY>() -> afmm_status {
            sp_compact_kernel<DTX, DTY><<<grid, SP_ROWS * 32, 0, st>>>(a);
            return AFMM_OK;
        });
    }));
    AFMM_CUDA_TRY(cudaGetLastError());
    SpMul mp{};
    mp.px = a.m[0].ptr;
    mp.nx = a.m[0].cnt;
    mp.ex = a.m[0].ent;
    mp.py = a.m[1].ptr;
    mp.ny = a.m[1].cnt;
    mp.ey = a.m[1].ent;
    mp.sy = a.m[1].spl;
    mp.n = n;
    mp.C = a.C;
    mp.Z = Z;
    mp.ldz = ldz;
    mp.zvec = reinterpret_cast<uintptr_t>(Z) % 16 == 0 && ldz % 4 == 0;
    mp.status = status;
    mp.ovf_used = a.ovf_used;
    const int row_floats = a.C > 1 ? SP_CW : (int)((n + 31) / 32 * 32);
    // Warps per block: two blocks fit in one SM's shared memory.
    int warps = (int)((113 * 1024) / ((size_t)row_floats * sizeof(float)));
    mp.warps = warps < 1 ? 1 : (warps > SP_MUL_WARPS ? SP_MUL_WARPS : warps);
    mp.row_floats = row_floats;
    const size_t smem = (size_t)mp.warps * row_floats * sizeof(float);
    const int64_t pairs_y = n * (int64_t)a.m[1].R + a.m[1].ovf_cap;
    auto kern = pairs_y < (int64_t)1 << 31 ? sp_mul_kernel<int> : sp_mul_kernel<int64_t>;
    AFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    AFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       100));
    const int64_t items = n * a.C;
    const unsigned blocks = (unsigned)((items + mp.warps - 1) / mp.warps);
    main_kernel_begin(st);
    kern<<<blocks, mp.warps * 32, smem, st>>>(mp);
    AFMM_CUDA_TRY(cudaGetLastError());
    main_kernel_end(st, (int)blocks);
    count_launches(2);
    return AFMM_OK;
}

}  // namespace afmm
