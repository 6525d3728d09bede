// K2 (CUDA-core side): operand conversions that feed the GEMM kernels.
// All are single HBM passes.  They change storage, never values, except
// the row-scaled slicing of the FP64 target, whose truncation is below
// 2^-55 of the row maximum.
#include "afmm_common.cuh"
#include "elem.cuh"

namespace afmm {

namespace {

constexpr int kThreads = 256;

inline dim3 grid2d(int64_t cols, int64_t rows) {
    int64_t gx = (cols + kThreads - 1) / kThreads;
    int64_t gy = rows < 65535 ? rows : 65535;
    if (gx < 1) gx = 1;
    if (gy < 1) gy = 1;
    return dim3((unsigned)gx, (unsigned)gy);
}

template <int DT>
__global__ void to_f32_kernel(const void* __restrict__ src, int64_t n,
                              int64_t lds, float* __restrict__ dst,
                              int64_t ldd) {
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= n) return;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y)
        dst[r * ldd + c] = (float)Elem<DT>::get(src, r * lds + c);
}

// int8 value of an integer-valued entry.  A value that int8 cannot hold
// exactly records an error and packs as 0: a non-integer (NaN included) as
// AFMM_ERR_NONINTEGER_REP for a Rep-factor (`rep`), else
// AFMM_ERR_OVERFLOW_RISK; a negative Rep-factor (Sec. 2 types) as
// AFMM_ERR_NEGATIVE_REP; a value outside [-128, 127] as
// AFMM_ERR_OVERFLOW_RISK.
__device__ __forceinline__ int to_i8_checked(double v, int* status, int rep) {
    if (!(trunc(v) == v)) {
        atomicCAS(status, 0, rep ? (int)AFMM_ERR_NONINTEGER_REP : (int)AFMM_ERR_OVERFLOW_RISK);
        return 0;
    }
    if (rep && v < 0.0) {
        atomicCAS(status, 0, (int)AFMM_ERR_NEGATIVE_REP);
        return 0;
    }
    if (v < -128.0 || v > 127.0) {
        atomicCAS(status, 0, (int)AFMM_ERR_OVERFLOW_RISK);
        return 0;
    }
    return (int)v;
}

template <int DT>
__global__ void pack_b_i8_kernel(const void* __restrict__ B, int64_t n,
                                 int64_t ldb, int32_t* __restrict__ W,
                                 int64_t ldw, int64_t kwords, int* status, int rep) {
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= ldw) return;
    for (int64_t kw = blockIdx.y; kw < kwords; kw += gridDim.y) {
        uint32_t w = 0;
        if (c < n) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int64_t k = kw * 4 + t;
                if (k < n) {
                    const int q = to_i8_checked(Elem<DT>::get(B, k * ldb + c),
                                                status, rep);
                    w |= (uint32_t)(q & 0xff) << (8 * t);
                }
            }
        }
        W[kw * ldw + c] = (int32_t)w;
    }
}

template <int DT>
__global__ void pack_a_i8_kernel(const void* __restrict__ A, int64_t n,
                                 int64_t lda, int8_t* __restrict__ D,
                                 int64_t ldd, int* status, int rep) {
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= ldd) return;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        int q = 0;
        if (c < n) q = to_i8_checked(Elem<DT>::get(A, r * lda + c), status, rep);
        D[r * ldd + c] = (int8_t)q;
    }
}

// Exponent e with |v| < 2^e for a non-zero finite double, from its bits:
// a normal number with biased exponent b lies in [2^(b-1023), 2^(b-1022)).
__device__ __forceinline__ int exp_bound(double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int b = (int)((bits >> 52) & 0x7ff);
    return (b == 0 ? 1 : b) - 1022;
}

constexpr int kEmptyRowExp = -1100;

template <int DT>
__global__ void __launch_bounds__(kThreads)
row_exponent_kernel(const void* __restrict__ A, int64_t n, int64_t lda,
                    int32_t* __restrict__ E) {
    __shared__ int red[kThreads / 32];
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        int e = kEmptyRowExp;
        for (int64_t c = threadIdx.x; c < n; c += kThreads) {
            const double v = Elem<DT>::get(A, r * lda + c);
            if (v != 0.0) e = max(e, exp_bound(v));
        }
        for (int off = 16; off > 0; off >>= 1)
            e = max(e, __shfl_down_sync(0xffffffffu, e, off));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            int m = red[0];
            for (int w = 1; w < kThreads / 32; ++w) m = max(m, red[w]);
            E[r] = m;
        }
        __syncthreads();
    }
}

// Digits of |v| * 2^(W - e) (W = bits * slices <= 63), most significant
// first, each in [0, 2^bits), with the sign of v.  Pure integer work on the
// IEEE-754 fields: |v| = m * 2^(b - 1075) with m the 53-bit significand.
template <int DT>
__global__ void slice_rows_kernel(const void* __restrict__ A, int64_t n,
                                  int64_t lda, const int32_t* __restrict__ E,
                                  int slices, int bits,
                                  int8_t* __restrict__ Q, int64_t ldq) {
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= ldq) return;
    const int W = bits * slices;
    const unsigned long long dmask = (1ull << bits) - 1ull;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        unsigned long long T = 0;
        bool neg = false;
        if (c < n) {
            const double v = Elem<DT>::get(A, r * lda + c);
            if (v != 0.0) {
                const unsigned long long b =
                    (unsigned long long)__double_as_longlong(v);
                neg = (b >> 63) != 0;
                const int be = (int)((b >> 52) & 0x7ff);
                unsigned long long m = b & ((1ull << 52) - 1ull);
                if (be != 0) m |= (1ull << 52);
                const int shift = (be == 0 ? 1 : be) - 1075 + W - E[r];
                if (shift >= 0) T = m << shift;
                else T = (-shift >= 64) ? 0ull : (m >> (-shift));
            }
        }
        for (int s = 0; s < slices; ++s) {
            const int d = (int)((T >> (W - bits * (s + 1))) & dmask);
            Q[((int64_t)s * n + r) * ldq + c] = (int8_t)(neg ? -d : d);
        }
    }
}

// 2^k as a double: built from its exponent field when normal, else ldexp.
__device__ __forceinline__ double pow2(int k) {
    if (k >= -1022 && k <= 1023)
        return __longlong_as_double((long long)(k + 1023) << 52);
    return ldexp(1.0, k);
}

// Row exponent and slicing in one pass for rows of at most 256 * PER
// elements: block r keeps row r in registers, reduces its exponent bound
// E[r] (as row_exponent_kernel) and writes the digit slices (as
// slice_rows_kernel).
template <int DT, int PER>
__global__ void __launch_bounds__(kThreads)
exp_slice_rows_kernel(const void* __restrict__ A, int64_t n, int64_t lda,
                      int32_t* __restrict__ E, int slices, int bits,
                      int8_t* __restrict__ Q, int64_t ldq) {
    __shared__ int red[kThreads / 32];
    const int W = bits * slices;
    const unsigned long long dmask = (1ull << bits) - 1ull;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        double v[PER];
        int e = kEmptyRowExp;
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int64_t c = threadIdx.x + (int64_t)kThreads * p;
            v[p] = c < n ? (double)Elem<DT>::get(A, r * lda + c) : 0.0;
            if (v[p] != 0.0) e = max(e, exp_bound(v[p]));
        }
        for (int off = 16; off > 0; off >>= 1)
            e = max(e, __shfl_down_sync(0xffffffffu, e, off));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
        __syncthreads();
        int er = red[0];
        for (int w = 1; w < kThreads / 32; ++w) er = max(er, red[w]);
        if (threadIdx.x == 0) E[r] = er;
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int64_t c = threadIdx.x + (int64_t)kThreads * p;
            if (c >= ldq) break;
            unsigned long long T = 0;
            bool neg = false;
            if (v[p] != 0.0) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(v[p]);
                neg = (b >> 63) != 0;
                const int be = (int)((b >> 52) & 0x7ff);
                unsigned long long m = b & ((1ull << 52) - 1ull);
                if (be != 0) m |= (1ull << 52);
                const int shift = (be == 0 ? 1 : be) - 1075 + W - er;
                if (shift >= 0) T = m << shift;
                else T = (-shift >= 64) ? 0ull : (m >> (-shift));
            }
            for (int s = 0; s < slices; ++s) {
                const int d = (int)((T >> (W - bits * (s + 1))) & dmask);
                Q[((int64_t)s * n + r) * ldq + c] = (int8_t)(neg ? -d : d);
            }
        }
        __syncthreads();                   // red[] is reused by the next row
    }
}

__global__ void recombine_f64_kernel(const int32_t* __restrict__ P,
                                     int64_t ldp, const int32_t* __restrict__ E,
                                     int slices, int bits, int64_t n,
                                     double* __restrict__ Z, int64_t ldz) {
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= n) return;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        const int e = E[r];
        double z = 0.0;
        // Smallest slice first; each term is exact (|P| < 2^31, scale a
        // power of two), only the additions round.
        for (int s = slices - 1; s >= 0; --s) {
            const int32_t p = P[((int64_t)s * n + r) * ldp + c];
            z += (double)p * pow2(e - bits * (s + 1));
        }
        Z[r * ldz + c] = z;
    }
}

// dst[c][r] = src[r][c] for an rows x cols matrix of ES-byte elements,
// through a 32 x 32 shared-memory tile (coalesced on both sides).
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ src, int64_t rows,
                                 int64_t cols, int64_t lds, T* __restrict__ dst,
                                 int64_t ldd) {
    __shared__ T tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = src[r * lds + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[c * ldd + r] = tile[threadIdx.x][i];
    }
}

}  // namespace

afmm_status launch_transpose(const void* src, size_t esize, int64_t rows,
                             int64_t cols, int64_t lds, void* dst, int64_t ldd,
                             cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return AFMM_OK;
    const int64_t gx = (cols + 31) / 32, gy = (rows + 31) / 32;
    if (gy > 65535) return AFMM_ERR_UNSUPPORTED;
    const dim3 grid((unsigned)gx, (unsigned)gy), block(32, 8);
    switch (esize) {
        case 1: transpose_kernel<uint8_t><<<grid, block, 0, st>>>(
                    (const uint8_t*)src, rows, cols, lds, (uint8_t*)dst, ldd); break;
        case 2: transpose_kernel<uint16_t><<<grid, block, 0, st>>>(
                    (const uint16_t*)src, rows, cols, lds, (uint16_t*)dst, ldd); break;
        case 4: transpose_kernel<uint32_t><<<grid, block, 0, st>>>(
                    (const uint32_t*)src, rows, cols, lds, (uint32_t*)dst, ldd); break;
        case 8: transpose_kernel<unsigned long long><<<grid, block, 0, st>>>(
                    (const unsigned long long*)src, rows, cols, lds,
                    (unsigned long long*)dst, ldd); break;
        default: return AFMM_ERR_INVALID_ARG;
    }
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_to_f32(const void* src, int dtype, int64_t n, int64_t lds,
                          float* dst, int64_t ldd, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        to_f32_kernel<DT><<<grid2d(n, n), kThreads, 0, st>>>(src, n, lds, dst,
                                                             ldd);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_pack_b_i8(const void* B, int dtype, int64_t n, int64_t ldb,
                             int32_t* W, int64_t ldw, int* status,
                             cudaStream_t st, bool rep) {
    if (n <= 0) return AFMM_OK;
    const int64_t kwords = (n + 3) / 4;
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        pack_b_i8_kernel<DT><<<grid2d(ldw, kwords), kThreads, 0, st>>>(
            B, n, ldb, W, ldw, kwords, status, rep ? 1 : 0);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_pack_a_i8(const void* A, int dtype, int64_t n, int64_t lda,
                             int8_t* D, int64_t ldd, int* status,
                             cudaStream_t st, bool rep) {
    if (n <= 0) return AFMM_OK;
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        pack_a_i8_kernel<DT><<<grid2d(ldd, n), kThreads, 0, st>>>(
            A, n, lda, D, ldd, status, rep ? 1 : 0);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_row_exponents(const void* A, int dtype, int64_t n,
                                 int64_t lda, int32_t* E, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    const unsigned nb = (unsigned)(n < 65535 ? n : 65535);
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        row_exponent_kernel<DT><<<nb, kThreads, 0, st>>>(A, n, lda, E);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_slice_rows_i8(const void* A, int dtype, int64_t n,
                                 int64_t lda, const int32_t* E, int slices,
                                 int bits, int8_t* Q, int64_t ldq,
                                 cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (bits < 1 || bits > 7 || slices < 1 || bits * slices > 63)
        return AFMM_ERR_INVALID_ARG;
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        slice_rows_kernel<DT><<<grid2d(ldq, n), kThreads, 0, st>>>(
            A, n, lda, E, slices, bits, Q, ldq);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_exp_slice_rows_i8(const void* A, int dtype, int64_t n,
                                     int64_t lda, int32_t* E, int slices, int bits,
                                     int8_t* Q, int64_t ldq, cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    if (bits < 1 || bits > 7 || slices < 1 || bits * slices > 63)
        return AFMM_ERR_INVALID_ARG;
    if (ldq > 4 * kThreads) {
        AFMM_TRY(launch_row_exponents(A, dtype, n, lda, E, st));
        return launch_slice_rows_i8(A, dtype, n, lda, E, slices, bits, Q, ldq, st);
    }
    const unsigned nb = (unsigned)(n < 65535 ? n : 65535);
    afmm_status rc = dispatch_dtype(dtype, [&]<int DT>() -> afmm_status {
        if (ldq <= kThreads)
            exp_slice_rows_kernel<DT, 1><<<nb, kThreads, 0, st>>>(A, n, lda, E, slices, bits, Q,
                                                                  ldq);
        else
            exp_slice_rows_kernel<DT, 4><<<nb, kThreads, 0, st>>>(A, n, lda, E, slices, bits, Q,
                                                                  ldq);
        return AFMM_OK;
    });
    AFMM_TRY(rc);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

afmm_status launch_recombine_f64(const int32_t* P, int64_t ldp,
                                 const int32_t* E, int slices, int bits,
                                 int64_t n, double* Z, int64_t ldz,
                                 cudaStream_t st) {
    if (n <= 0) return AFMM_OK;
    recombine_f64_kernel<<<grid2d(n, n), kThreads, 0, st>>>(P, ldp, E, slices,
                                                           bits, n, Z, ldz);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
