// Tensor-core (tcgen05 / TMEM / TMA) path of libafmm: internal interface.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "afmm.h"

namespace afmm {

// Per-plan state of the tensor-core variants: operand buffers in the
// workspace and the TMA descriptors that read them.
struct TcPlan {
    int64_t n = 0;
    int slices = 3;
    int64_t ld_a = 0, ld_b = 0;     // leading dims (elements) of A / B operands
    int64_t rows_a = 0, rows_b = 0; // rows of the stacked A / B buffers
    size_t a_bytes = 0, b_bytes = 0;
    void* a = nullptr;              // A operand(s), K-major (BF16 or E4M3)
    void* b = nullptr;              // B operand(s), K-major (B^T rows)
    bool sliced_a = true;           // real factor on the A side (case A)
    bool both = false;              // both factors sliced (real x real)
    int kb_per_chunk = 0;           // exact form: K chunk in 32-wide k-blocks
    float lim_a = 256.f, lim_b = 256.f;  // exact form: largest |value| allowed
    // Case A split form with rows of Z not 16-byte aligned (ldz % 4 != 0):
    // the product goes to this buffer (ld_z = n rounded up to 4, so its
    // epilogue stores stay 16-byte wide) and is copied into Z.
    size_t z_bytes = 0;
    int64_t ld_z = 0;
    void* z = nullptr;
    // FP8 form (E4M3 operands, one byte per element, ld_a / ld_b multiples
    // of 16): amax[m] = FP32 bits of the largest |value| of A row m, which
    // sets the power of two the row's slices were scaled by.
    bool f8 = false;
    size_t s_bytes = 0;
    uint32_t* amax = nullptr;
    // FP8 and real x real forms: k-blocks after which the hi sum is added
    // into FP32 registers (0: once per tile); AFMM_TC_CHUNK_KB in the
    // environment overrides.
    int chunk_kb = 0;
    alignas(64) unsigned char tmap_a[128];
    alignas(64) unsigned char tmap_b[128];
    // Case B split form computed as Z^T = Y^T X^T: A side = the b buffer.
    alignas(64) unsigned char tmap_at[128];
    alignas(64) unsigned char tmap_bt[128];
    // B side with 128-row boxes (half a B tile per CTA of a two-SM pair)
    // and with 64-row boxes (half of a 128-column part of a last-round tile).
    alignas(64) unsigned char tmap_b2[128];
    alignas(64) unsigned char tmap_bt2[128];
    alignas(64) unsigned char tmap_b3[128];
    alignas(64) unsigned char tmap_bt3[128];
    // The pair kernel's maps with 128-byte operand rows (128-byte swizzle):
    // A (128-row boxes), the two B halves, and Case B's transposed roles.
    alignas(64) unsigned char tmap_aw[128];
    alignas(64) unsigned char tmap_atw[128];
    alignas(64) unsigned char tmap_b2w[128];
    alignas(64) unsigned char tmap_bt2w[128];
    alignas(64) unsigned char tmap_b3w[128];
    alignas(64) unsigned char tmap_bt3w[128];
    bool maps_ready = false;
    // Split form: run the two-SM (cta_group::2) product kernel.
    bool pair = false;
    // FP16 two-slice form (fp16_split.cuh): FP16 operands, amax[m] sets
    // the power of two row m of the real factor was scaled by.
    bool h16 = false;
    // Exact form on E4M3 digits (Case A, two-SM kernel): A = two digit
    // slices of X, B = Rep-factors, one byte each; Z int32.
    bool x8 = false;
};

// TMA descriptor (written to `out`, 128 bytes, 64-byte aligned) of a stack
// of `slices` matrices of es-byte elements (2: BF16, 1: E4M3), `rows` x
// `cols` with leading dimension `ld` elements; boxes of row_bytes (64 or
// 128) of columns x box_rows rows x 1 slice, swizzle of the same width.
afmm_status tc_encode_map(void* out, void* base, int64_t cols, int64_t rows,
                          int64_t ld, int slices, int box_rows, int es = 2,
                          int row_bytes = 64);

// Operand conversions (tc_operands.cu): dst BF16 [slices][n][ldk].  Rows
// kept (K-major A) or transposed (K-major B, dst row = source column).
// exact: one slice that must equal the source and stay within |lim|
// (AFMM_ERR_OVERFLOW_RISK in *status otherwise); else 2 or 3 RN slices.
// rep: the source holds Rep-factors, checked to be non-negative integers
// (AFMM_ERR_NEGATIVE_REP / AFMM_ERR_NONINTEGER_REP in *status otherwise).
// (tc_widen_rows converts rows [r0, r1) only; r1 < 0 means n.)
afmm_status tc_widen_rows(int slices, bool exact, const void* src, int dt, int64_t n,
                          int64_t lds, void* dst, int64_t ldk, float lim, int* status,
                          cudaStream_t st, int64_t r0 = 0, int64_t r1 = -1,
                          bool rep = false);
afmm_status tc_widen_transpose(int slices, bool exact, const void* src, int dt, int64_t n,
                               int64_t lds, void* dst, int64_t ldk, float lim, int* status,
                               cudaStream_t st, bool rep = false);
// The same transposition, exact, to FP16 (the FP16 two-slice form's
// Rep-factor operand; |value| <= lim and exact in FP16).
afmm_status tc_widen_transpose_h16(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                                   int64_t ldk, float lim, int* status, cudaStream_t st,
                                   bool rep);
// FP16 two-slice form (tc_f16.cu): rows [r0, r1) of the real factor
// (row-major n x n) as two FP16 slices dst[(s * n + r) * ldk + c] (ldk a
// multiple of 8, zero for n <= c < ldk), row r scaled by 2^h16_row_shift
// (amax[r]), amax[r] = FP32 bits of the row's largest |value|.  A
// non-finite value records AFMM_ERR_OVERFLOW_RISK.
afmm_status tc_h16_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                        int64_t ldk, uint32_t* amax, int* status, cudaStream_t st,
                        int64_t r0 = 0, int64_t r1 = -1);
// Case B: the columns of the real factor as the K-major rows of two FP16
// slices, column c scaled by 2^h16_row_shift(amax[c]) (amax written here).
afmm_status tc_h16_transpose(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                             int64_t ldk, uint32_t* amax, int* status, cudaStream_t st);
// Exact form on E4M3 digits (tc_x8.cu): the rows of X (integers, |x| <=
// 255) as two digit slices dst[(s * n + r) * ldk + c], h = floor(x / 16)
// and l = x - 16 h; the Rep-factors of Y (0 .. 16) transposed to K-major
// E4M3.  ldk a multiple of 16; range errors record AFMM_ERR_OVERFLOW_RISK.
afmm_status tc_x8_digit_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                             int64_t ldk, int* status, cudaStream_t st);
afmm_status tc_x8_rep_transpose(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                                int64_t ldk, int* status, cudaStream_t st);
// Case B: the columns of Y (integer Base values) as two transposed digit
// slices; the Rep-factors of X kept as E4M3 rows.
afmm_status tc_x8_digit_transpose(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                                  int64_t ldk, int* status, cudaStream_t st);
afmm_status tc_x8_rep_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                           int64_t ldk, int* status, cudaStream_t st);
// The exact form on E4M3 digits (n >= 512): conversions and the two-SM
// product into Z (int32); Case B as Z^T = Y^T X^T.
afmm_status tc_run_exact_x8(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                            void* Z, int* status, cudaStream_t st);
// Case B: the Rep-factors' rows kept as exact FP16 (|value| <= lim).
afmm_status tc_h16_rep_rows(const void* src, int dt, int64_t n, int64_t lds, void* dst,
                            int64_t ldk, float lim, int* status, cudaStream_t st);

// FP8 form conversions (tc_fp8.cu): dst E4M3 [slices][n][ldk], ldk a
// multiple of 16.  rep: one slice that must equal the source (Rep-factors;
// AFMM_ERR_OVERFLOW_RISK in *status otherwise).  Else four slices of each
// row (tc_f8_rows) or column (tc_f8_transpose) scaled by a power of two
// from its largest |value|, whose FP32 bits go to amax[row or column]
// (a non-finite value: AFMM_ERR_OVERFLOW_RISK).  tc_f8_rows converts rows
// [r0, r1) only; r1 < 0 means n.
afmm_status tc_f8_rows(bool rep, const void* src, int dt, int64_t n, int64_t lds, void* dst,
                       int64_t ldk, uint32_t* amax, int* status, cudaStream_t st,
                       int64_t r0 = 0, int64_t r1 = -1);
afmm_status tc_f8_transpose(bool rep, const void* src, int dt, int64_t n, int64_t lds,
                            void* dst, int64_t ldk, uint32_t* amax, int* status,
                            cudaStream_t st);

// True when this device can run the tensor-core kernels (sm_103).
bool tc_available();
// slices = 0 selects the exact-integer form (one BF16 operand each side);
// f8 the FP8 form (four E4M3 slices).
// h16 the FP16 two-slice form (slices = 2); x8 the exact form on E4M3
// digits (Case A, slices = 2).
void tc_layout(TcPlan* t, const afmm_desc& d, int slices, bool f8 = false, bool h16 = false,
               bool x8 = false);
// Largest K chunk (multiple of 32) with chunk * amax * bmax < 2^24, or 0
// when even one 32-wide block could overflow.
int tc_exact_chunk_k(double amax, double bmax);
afmm_status tc_bind_workspace(TcPlan* t, void* a, void* b, void* z, void* s);
// Split / widen the operands and run the tcgen05 product into Z (F32).
afmm_status tc_run_split(TcPlan* t, const afmm_desc& d, const void* X,
                         const void* Y, void* Z, int* status, cudaStream_t st);
// Real x real (AFMM_CASE_REAL): three BF16 slices of X and of Y^T, six
// slice products into Z (F32).
afmm_status tc_run_real(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                        void* Z, int* status, cudaStream_t st);
// The FP8 form: E4M3 slices and Rep-factors, the tcgen05 product into Z.
afmm_status tc_run_fp8(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                       void* Z, int* status, cudaStream_t st);
// The FP16 two-slice form (Case A): X as two row-scaled FP16 slices, Y as
// FP16 Rep-factors, the tcgen05 product into Z.
afmm_status tc_run_h16(TcPlan* t, const afmm_desc& d, const void* X, const void* Y,
                       void* Z, int* status, cudaStream_t st);
// The same product in pieces for transfer pipelining: tc_split_prepare_b
// converts the B operand (all of the factor that is not split by rows);
// tc_split_rows converts rows [r0, r1) of the A operand and computes rows
// [r0, r1) of Z.  Case A or B, 2 or 3 BF16 slices (the separate-split
// path) or the FP8 form.
afmm_status tc_split_prepare_b(TcPlan* t, const afmm_desc& d, const void* Y, int* status,
                               cudaStream_t st);
afmm_status tc_split_rows(TcPlan* t, const afmm_desc& d, const void* X, void* Z,
                          int64_t r0, int64_t r1, int* status, cudaStream_t st);
// tc_split_rows in its two steps: convert rows [r0, r1) of the A operand
// (X may be a device-mapped pointer to pinned host memory), then multiply
// them.
afmm_status tc_split_convert_rows(TcPlan* t, const afmm_desc& d, const void* X, int64_t r0,
                                  int64_t r1, int* status, cudaStream_t st);
afmm_status tc_split_product_rows(TcPlan* t, const afmm_desc& d, void* Z, int64_t r0,
                                  int64_t r1, int* status, cudaStream_t st);
// Row blocks of Z for pipelining an n x n product: boundaries multiples of
// the tile extent along Z's rows (128 in Case A, 256 in Case B, whose
// product is Z^T; 256 for the two-SM kernel, `pair`), chosen so each
// block's tile count fills whole waves of `sms` CTAs (sms / 2 pairs).
int tc_row_blocks(int64_t n, int sms, int64_t* bounds, int max_blocks, bool caseb,
                  bool pair = false);
// The schedule of the host-buffer pipeline: first and last blocks of about
// one wave of tiles, whole-wave blocks between (tc_row_blocks when n is too
// small for that).  Returns the number of blocks; bounds[0..k] are Z rows.
int tc_pipe_blocks(int64_t n, int sms, int64_t* bounds, int max_blocks, bool caseb,
                   bool pair = false);
// Case A, three slices, X FP32 with 16-byte aligned rows: the fused kernel
// (tc_fused.cu) reads X directly and splits it in shared memory.
bool tc_fused_usable(const afmm_desc& d, const void* X);
afmm_status tc_run_fused_caseA(const TcPlan* t, const afmm_desc& d, const void* X,
                               void* Z, int* status, cudaStream_t st);

// Exact integer product into Z (I32).
afmm_status tc_run_exact(TcPlan* t, const afmm_desc& d, const void* X,
                         const void* Y, void* Z, int* status, cudaStream_t st);

// Launch a kernel whose only wait can never complete; returns the status
// it recorded (AFMM_ERR_TIMEOUT expected).
afmm_status tc_selftest_bounded_wait(uint64_t limit_ns, cudaStream_t st);

}  // namespace afmm
