// Internal declarations shared by the translation units of libafmm.
// Nothing here is part of the C ABI (include/afmm.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "afmm.h"

namespace afmm {

// ------------------------------------------------------------------ errors
#define AFMM_CUDA_TRY(expr)                                                  \
    do {                                                                     \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) {                                             \
            afmm::set_last_cuda_error(e_, #expr, __FILE__, __LINE__);        \
            return (e_ == cudaErrorMemoryAllocation) ? AFMM_ERR_OOM          \
                                                     : AFMM_ERR_CUDA;        \
        }                                                                    \
    } while (0)

#define AFMM_TRY(expr)                                                       \
    do {                                                                     \
        afmm_status s_ = (expr);                                             \
        if (s_ != AFMM_OK) return s_;                                        \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file,
                         int line);
// Set the text afmm_last_error_detail returns for this thread.
void set_last_error_text(const char* text);

// Kernel-launch counter of the calling thread (every launcher adds the
// kernels it launched) and the main-kernel timing hook of a call.
void count_launches(int k);
int64_t launch_counter();
struct MainTimer {
    cudaEvent_t start = nullptr, stop = nullptr;  // null: timing off
    int ctas = 0;
    bool started = false;     // start recorded by this call's first main launch
};
MainTimer* current_main_timer();   // set by the plan around a call
// Record around the main kernel launch (no-ops without a current timer); a
// call with several main launches is timed from the first start to the last
// end.
void main_kernel_begin(cudaStream_t st);
void main_kernel_end(cudaStream_t st, int ctas);

// ------------------------------------------------------------------ dtypes
inline size_t dtype_size(int dt) {
    switch (dt) {
        case AFMM_F64: return 8;
        case AFMM_F32: case AFMM_I32: return 4;
        case AFMM_BF16: return 2;
        case AFMM_E4M3: case AFMM_I8: case AFMM_U8: return 1;
        default: return 0;
    }
}
inline bool dtype_is_integer(int dt) {
    return dt == AFMM_I32 || dt == AFMM_I8 || dt == AFMM_U8;
}

// Device-side statistics of one matrix (K0 scan), reduced over the matrix.
struct ScanStats {
    unsigned long long nnz;        // non-zero entries
    unsigned long long negative;   // entries < 0
    unsigned long long nonint;     // entries that are not integers
    unsigned long long over127;    // entries > 127 (int8 packing limit)
    double sum;                    // sum of entries
    double maxv;                   // largest entry (-inf when empty)
    double max_abs;                // largest |entry|
    double pad_;
};
constexpr int kScanMaxBlocks = 1024;

// Per-device facts read once.
struct DeviceProps {
    int device = -1;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
};
afmm_status device_props(DeviceProps* out);

// ------------------------------------------------------------------ kernels
// K0: statistics of an n x n matrix; `partials` holds kScanMaxBlocks
// entries.  When `status` is non-null and `is_rep` is set, a negative or
// non-integer entry records an error code there.
afmm_status launch_scan(const void* M, int dtype, int64_t n, int64_t ld,
                        bool is_rep, ScanStats* partials, ScanStats* out,
                        int* status, cudaStream_t st);

// Rep-factor check alone (no statistics): a negative entry records
// AFMM_ERR_NEGATIVE_REP in `status`, else a non-integer one (NaN, infinity)
// AFMM_ERR_NONINTEGER_REP.  Launches nothing for u8 (always valid).
afmm_status launch_rep_check(const void* M, int dtype, int64_t n, int64_t ld, int* status,
                             cudaStream_t st);

// K2: conversions.
// dst[r*ldd + c] = (float) src[r*lds + c]
afmm_status launch_to_f32(const void* src, int dtype, int64_t n, int64_t lds,
                          float* dst, int64_t ldd, cudaStream_t st);
// dst[c*ldd + r] = src[r*lds + c] for esize-byte elements.
afmm_status launch_transpose(const void* src, size_t esize, int64_t rows,
                             int64_t cols, int64_t lds, void* dst, int64_t ldd,
                             cudaStream_t st);
// Pack an integer-valued n x n matrix B (row-major) into int8 words
// W[kw*ldw + c] = bytes B[4kw..4kw+3][c] (k-word-major, zero padded to a
// multiple of 4 rows).  Values outside [-128, 127] or not integers record
// AFMM_ERR_OVERFLOW_RISK in `status`; with `rep` (the matrix holds
// Rep-factors) a negative value records AFMM_ERR_NEGATIVE_REP and a
// non-integer AFMM_ERR_NONINTEGER_REP.
afmm_status launch_pack_b_i8(const void* B, int dtype, int64_t n, int64_t ldb,
                             int32_t* W, int64_t ldw, int* status,
                             cudaStream_t st, bool rep);
// Copy an integer-valued n x n matrix A (row-major) into int8 rows
// D[r*ldd + c] (ldd a multiple of 4, padding zeroed).  Same checks.
afmm_status launch_pack_a_i8(const void* A, int dtype, int64_t n, int64_t lda,
                             int8_t* D, int64_t ldd, int* status,
                             cudaStream_t st, bool rep);
// Row-scaled integer slicing of a real matrix for the FP64 target:
// E[r] = smallest e with max_c |A[r][c]| < 2^e; digit slices
// Q[s*n + r][c] (int8, ldq) with A[r][c] ~= sum_s Q * 2^(E[r]-w(s+1)).
afmm_status launch_row_exponents(const void* A, int dtype, int64_t n,
                                 int64_t lda, int32_t* E, cudaStream_t st);
afmm_status launch_slice_rows_i8(const void* A, int dtype, int64_t n,
                                 int64_t lda, const int32_t* E, int slices,
                                 int bits, int8_t* Q, int64_t ldq,
                                 cudaStream_t st);
// Both of the above in one pass (one launch) when ldq <= 1024.
afmm_status launch_exp_slice_rows_i8(const void* A, int dtype, int64_t n,
                                     int64_t lda, int32_t* E, int slices, int bits,
                                     int8_t* Q, int64_t ldq, cudaStream_t st);
// Z[r][c] = sum_s P[s*n + r][c] * 2^(E[r] - bits*(s+1)), in FP64.
afmm_status launch_recombine_f64(const int32_t* P, int64_t ldp,
                                 const int32_t* E, int slices, int bits,
                                 int64_t n, double* Z, int64_t ldz,
                                 cudaStream_t st);

// K1: CUDA-core GEMMs, C (M x N) = A (M x K) * B (K x N), row-major.
// FP32 FMA with zero-skip of A over 4-row groups and K-blocked sums.  With
// the K0 tile masks xm, ym (launch_tile_masks) a CTA loads and multiplies
// only the 32-wide k tiles whose A and B tiles both hold a non-zero, and
// adds their number to *ktiles (when given).
afmm_status launch_simt_f32(const float* A, int64_t lda, const float* B,
                            int64_t ldb, float* C, int64_t ldc, int64_t M,
                            int64_t N, int64_t K, cudaStream_t st,
                            const uint8_t* xm = nullptr, const uint8_t* ym = nullptr,
                            unsigned long long* ktiles = nullptr);
// K0 tile masks for launch_simt_f32: one byte per 64 x 32 tile of A
// ([ceil(M/64)][ceil(K/32)]) and per 32 x 256 tile of B ([ceil(K/32)]
// [ceil(N/256)]), 1 when the tile holds a non-zero.  simt_mask_bytes gives
// the bytes of both (B's at *ym_offset, 16-byte aligned).
size_t simt_mask_bytes(int64_t M, int64_t N, int64_t K, size_t* ym_offset);
afmm_status launch_tile_masks(const float* A, int64_t lda, const float* B, int64_t ldb,
                              int64_t M, int64_t N, int64_t K, uint8_t* xm, uint8_t* ym,
                              cudaStream_t st);
// FP32 FMA without zero-skip (simt_dense.cu), for dense Base factors: A
// given transposed (AT, K x M, ldat a multiple of 4, 16-byte aligned, else
// AFMM_ERR_INVALID_ARG), sums K-blocked over 128 k.
afmm_status launch_simt_f32_dense(const float* AT, int64_t ldat, const float* B,
                                  int64_t ldb, float* C, int64_t ldc, int64_t M,
                                  int64_t N, int64_t K, cudaStream_t st);
// dst = src^T as FP32 (n x n, src of afmm_dtype `dtype`, row strides lds
// and ldd elements).
afmm_status launch_to_f32_transposed(const void* src, int dtype, int64_t n, int64_t lds,
                                     float* dst, int64_t ldd, cudaStream_t st);
// int8 dot products: A int8 rows (lda bytes, multiple of 4), B packed
// k-word-major int32 words (ldw words), C int32.
afmm_status launch_simt_dp4a(const int8_t* A, int64_t lda, const int32_t* W,
                             int64_t ldw, int32_t* C, int64_t ldc, int64_t M,
                             int64_t N, int64_t K, cudaStream_t st);

// Grouped K1 (FP32): one launch over the tiles of many independent
// products.  jobs[] and tile_prefix[] (exclusive prefix of each job's tile
// count, simt_tiles) are device arrays.
struct SimtJob {
    const float* A;
    const float* B;
    float* C;
    int64_t lda, ldb, ldc, M, N, K;
    int vec, tiles_n;
};
int simt_tiles(int64_t M, int64_t N);
int simt_tiles_n(int64_t N);
afmm_status launch_simt_f32_grouped(const SimtJob* jobs, const int* tile_prefix,
                                    int njobs, int total_tiles, cudaStream_t st);

// Dispatch MLP (mlp.cu).
int64_t mlp_param_count(const afmm_mlp_shape& s);
int64_t mlp_work_floats(const afmm_mlp_shape& s, int rows);
afmm_status mlp_forward(const afmm_mlp_shape& s, const float* params, const float* X,
                        int rows, float* P, float* work, cudaStream_t st);
afmm_status mlp_loss_grad(const afmm_mlp_shape& s, const float* params, const float* X,
                          const float* T, const float* M, int rows, float count,
                          float* grads, float* work, float* loss, cudaStream_t st);
afmm_status mlp_adam(int64_t n, float* params, const float* grads, float* m, float* v,
                     float lr, float b1, float b2, float eps, int step, cudaStream_t st);

// Sparse x sparse product (sparse.cu): workspace for density hints d1, d2
// (< 0: unknown) and the launch sequence (compaction of X and Y, rows past
// their slot into an overflow region; product).  rep_which: the factor
// holding Rep-factors (0 X, 1 Y, -1 none), checked by the compaction.
size_t sparse_ws_bytes(int64_t n, double d1, double d2);
// Zero the compaction's overflow counters (a fresh or re-bound workspace;
// after an error).  Each product leaves them at zero for the next call.
afmm_status sparse_reset(void* ws, cudaStream_t st);
afmm_status launch_sparse(const void* X, int xdt, int64_t ldx, const void* Y, int ydt,
                          int64_t ldy, float* Z, int64_t ldz, int64_t n, double d1,
                          double d2, void* ws, int* status, cudaStream_t st,
                          int rep_which);

// K6: error norms, partial sums in `ws` (error_norm_ws_bytes bytes).
size_t error_norm_ws_bytes(int64_t rows, int64_t cols);
afmm_status launch_error_norm(const void* Z, int zdt, int64_t ldz,
                              const void* R, int rdt, int64_t ldr,
                              int64_t rows, int64_t cols, void* ws,
                              double* out_dev, cudaStream_t st);

}  // namespace afmm
