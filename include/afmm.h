/*
 * afmm.h -- C ABI of the GB300 (sm_103a) AFMM library.
 *
 * The library computes the AFMM product of Singh, Chakraborty and Mallick,
 * "An Adaptable Fast Matrix Multiplication (AFMM) Algorithm" (arXiv
 * 1308.2400), Sec. 2: Z = X * Y for two dense n x n matrices where one
 * factor holds non-negative integer "Rep-factors" and the other real "Base"
 * values, zero Base values skipped.
 *   Case A: X real (Base), Y integer Rep-factors  (Sec. 2, Case-A listing).
 *   Case B: X integer Rep-factors, Y real (Base)  (Sec. 2, Case-B listing).
 * The paper forms each term Rep * Base by adding Base Rep times; the result
 * is the ordinary product (Sec. 2.1 Point 1), which the GPU forms with
 * exact multiply-add or tensor-core products (see each variant below).
 *
 * Conventions for every entry point
 *  - Matrices are dense and row-major (Sec. 2 recommends the "adjacency
 *    matrix", i.e. dense, storage).  Leading dimensions count elements.
 *  - Z is overwritten (the paper starts Z at zero, Sec. 2).
 *  - X, Y, Z may be device pointers or host pointers (pageable or pinned);
 *    the library asks the CUDA runtime which.  Host buffers are staged
 *    through device buffers the plan owns: the call copies X and Y in,
 *    computes, copies Z out and synchronises the stream before returning
 *    (the split tensor-core forms at n >= 1024 overlap the copies of row
 *    blocks with the products on two extra streams).  With device pointers
 *    the call is asynchronous on `stream`; from the third call in a row on
 *    the same device buffers, problems with n <= 2048 are replayed from a
 *    CUDA graph captured by the plan.
 *  - The caller owns X, Y, Z.  A plan owns its workspace unless the caller
 *    lends one (afmm_plan_set_workspace).  A plan holds per-call state
 *    (workspace, staging buffers, replay graph): calls on one plan must be
 *    made from one thread at a time; separate plans are independent.
 *  - Errors are returned as afmm_status, never thrown.  Errors found by a
 *    kernel (a negative or non-integer Rep-factor, a bounded wait that ran
 *    out) are written to the plan's device status word and returned by the
 *    next afmm_plan_sync on that plan.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.
 */
#ifndef AFMM_H
#define AFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AFMM_OK = 0,
    AFMM_ERR_INVALID_ARG = 1,     /* bad pointer, size, dtype or enum value */
    AFMM_ERR_UNSUPPORTED = 2,     /* valid request this library cannot serve */
    AFMM_ERR_NEGATIVE_REP = 3,    /* a Rep-factor is negative (Sec. 2 types) */
    AFMM_ERR_OVERFLOW_RISK = 4,   /* exact target could leave the int32 range */
    AFMM_ERR_OOM = 5,             /* device or host allocation failed */
    AFMM_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    AFMM_ERR_TIMEOUT = 7,         /* a bounded device-side wait ran out */
    AFMM_ERR_NO_DEVICE = 8,       /* no usable CUDA device */
    AFMM_ERR_NONINTEGER_REP = 9   /* a Rep-factor is not an integer */
} afmm_status;

/* Which factor holds the Rep-factors (Sec. 2).  AFMM_CASE_REAL: neither --
 * both factors real, the generalisation the paper's conclusion (Sec. 4)
 * leaves open; such plans multiply with afmm_mul_real, FP32 target. */
typedef enum { AFMM_CASE_A = 0, AFMM_CASE_B = 1, AFMM_CASE_REAL = 2 } afmm_case;

/* Element types.  AFMM_E4M3 is FP8 e4m3 (OCP, "fn"); it holds the integers
 * 0..16 exactly.  Rep-factor matrices may be I32, I8, U8, E4M3, BF16 or F32
 * (integral values); real matrices F64, F32 or BF16; an exact product also
 * accepts an I8 or I32 Base matrix. */
typedef enum {
    AFMM_F64 = 0, AFMM_F32 = 1, AFMM_BF16 = 2, AFMM_E4M3 = 3,
    AFMM_I32 = 4, AFMM_I8 = 5, AFMM_U8 = 6
} afmm_dtype;

/* Accuracy the product must reach against the exact product:
 *   FP32  relative Frobenius error <= 1e-6, Z F32;
 *   FP64  relative Frobenius error <= 1e-12, Z F64;
 *   EXACT bit-exact integers, Z I32 (both factors integer). */
typedef enum {
    AFMM_TARGET_FP32 = 0, AFMM_TARGET_FP64 = 1, AFMM_TARGET_EXACT = 2
} afmm_target;

/* Kernel variants a plan can run (AFMM_VARIANT_AUTO lets the planner pick). */
typedef enum {
    AFMM_VARIANT_AUTO = -1,
    /* CUDA cores, FP32 FMA, skips k where the Base is zero for a group of
     * rows, K-blocked accumulation.  FP32 target. */
    AFMM_VARIANT_SIMT_F32 = 0,
    /* Tensor cores (tcgen05, TMEM accumulators): the real factor split
     * into three BF16 slices (hi+mid+lo represent FP32 exactly), the
     * Rep-factors widened to BF16 (exact up to 256), FP32 accumulation
     * with the hi slice's products kept apart from the smaller slices'.
     * Case B is computed as Z^T = Y^T X^T.  FP32 target. */
    AFMM_VARIANT_TC_BF16X3 = 1,
    /* As above with two slices: does not reach the FP32 target in general;
     * offered for error studies only (never chosen automatically). */
    AFMM_VARIANT_TC_BF16X2 = 2,
    /* CUDA cores, FP64 target: the real factor cut into row-scaled integer
     * slices, exact int32 products, FP64 recombination. */
    AFMM_VARIANT_SIMT_F64SLICE = 3,
    /* CUDA cores, exact integers: int8 dot products (dp4a), int32 sums. */
    AFMM_VARIANT_SIMT_EXACT = 4,
    /* Tensor cores, exact integers: operands exact in BF16 (|v| <= 256),
     * K cut into chunks whose FP32 partial sums stay below 2^24 (so every
     * partial sum is an exact integer), chunks added in int32; 256 x 256
     * output tiles. */
    AFMM_VARIANT_TC_EXACT = 5,
    /* CUDA cores, both factors compacted to per-row (column, value) lists
     * -- the zero-skip of Sec. 2 on both sides -- for the quadratic regime
     * of Sec. 2.2 (d1 d2 n small): HBM-bound, FP32 target.  Its workspace
     * holds, per row, a slot sized from the d1, d2 hints (expected count
     * plus six standard deviations; all n without hints) and an overflow
     * region for longer rows (2 d n^2 + 32 n + 1024 entries); more
     * non-zeros than that is reported as AFMM_ERR_OVERFLOW_RISK by
     * afmm_plan_sync and Z is not written. */
    AFMM_VARIANT_SPARSE = 6,
    /* Tensor cores with 8-bit floats (tcgen05 kind::f8f6f4, FP32 TMEM
     * accumulators): each row of the real factor scaled by a power of two
     * (its largest |value| into [128, 256)) and split into four E4M3
     * slices -- three round-to-nearest slices and one of the third
     * residual times 2^12 -- so the slices hold about 20 significant bits;
     * Rep-factors held as E4M3, exact for 0..16 and every integral E4M3
     * value up to 448 (others, and non-finite real values: the call
     * records AFMM_ERR_OVERFLOW_RISK, reported by afmm_plan_sync).  Four
     * E4M3 MMAs per K step in place of three BF16 ones at twice the
     * rate.  The hi sum is closed every 16 K blocks of 64 and the chunks
     * added in FP32 (AFMM_TC_CHUNK_KB in the environment, read at plan
     * creation, overrides the count; 0 = never).  FP32 target; never
     * chosen automatically. */
    AFMM_VARIANT_TC_FP8X4 = 7,
    /* Tensor cores for two real factors (AFMM_CASE_REAL): both split into
     * three BF16 slices (hi+mid+lo = the FP32 value), and the six slice
     * products down to 2^-16 of the hi product -- (hi,hi), (hi,mid),
     * (mid,hi), (hi,lo), (mid,mid), (lo,hi) -- with the (hi,hi) products
     * kept in their own FP32 accumulator, closed every 12 K blocks of 32
     * and the chunks added in FP32 (AFMM_TC_CHUNK_KB overrides, as above)
     * (an Ozaki-style split; Ozaki, Ogita, Oishi and Rump, Numer.
     * Algorithms 59, 2012; Ootomo and Yokota, IJHPCA 36, 2022).  FP32
     * target. */
    AFMM_VARIANT_TC_BF16X3X3 = 8,
    /* The split BF16 form of AFMM_VARIANT_TC_BF16X3 with 128 x 128 output
     * tiles in place of 128 x 256: less padding for sizes just above a
     * multiple of 128, more staged bytes per flop.  A route of
     * afmm_mul_batched only (a plan refuses it with AFMM_ERR_UNSUPPORTED). */
    AFMM_VARIANT_TC_BF16X3_N128 = 9,
    /* Tensor cores, two FP16 slices of the real factor: each row of X
     * (Case A; each column of Y in Case B) scaled by a power of two so that
     * its largest |value| lies in
     * [2^14, 2^15), then split as hi + lo 2^-8, hi the value rounded to 8
     * significant bits and lo the remainder times 2^8 rounded to FP16
     * (split half precision; Ootomo and Yokota, IJHPCA 36, 2022).  The
     * Rep-factors (integers up to 2048, exact in FP16) are the other FP16
     * operand; the hi and lo products go to two FP32 accumulators, summed
     * once and scaled back exactly in the epilogue.  Two MMAs per K step
     * where AFMM_VARIANT_TC_BF16X3 takes three, at the same tensor rate;
     * its representation error, below 2^-20 of each value, keeps the FP32
     * target.  A Rep-factor above 2048 (or not exact in FP16) or a
     * non-finite real factor records AFMM_ERR_OVERFLOW_RISK (reported by
     * afmm_plan_sync).  Never chosen automatically. */
    AFMM_VARIANT_TC_F16X2 = 10,
    /* Exact target, n >= 512, on E4M3 digits: each integer Base value x
     * (of X in Case A, of Y in Case B; |x| <= 255) as x = 16 h + l with
     * h = floor(x / 16) and
     * l in [0, 15], the Rep-factors (0 .. 16) and both digits exact in
     * E4M3; two kind::f8f6f4 MMAs per K step (twice the BF16 rate) on CTA
     * pairs, the h and l products in two FP32 accumulators whose sums stay
     * exact integers (n 16 16 < 2^24 for n < 65536), Z = 16 acc_h + acc_l
     * in int32.  A value outside those ranges records
     * AFMM_ERR_OVERFLOW_RISK (a negative or non-integer Rep-factor
     * AFMM_ERR_NEGATIVE_REP / _NONINTEGER_REP), reported by
     * afmm_plan_sync.  Chosen automatically for exact plans whose
     * magnitude hints (rep_max <= 16, base_max <= 255) allow it. */
    AFMM_VARIANT_TC_EXACT_F8 = 11,
    AFMM_VARIANT_COUNT_ = 12
} afmm_variant;

/* Flags for afmm_desc.flags. */
#define AFMM_FLAG_VALIDATE 0x1u  /* also scan both factors on every call
                                    for the paper's parameters (realised
                                    d1, d2, mu', read by afmm_get_info) */
#define AFMM_FLAG_FUSED_SPLIT 0x2u  /* Case A, FP32 X with 16-byte aligned
                                    rows: split X into BF16 slices inside
                                    the product kernel instead of in a
                                    separate pass (measured slower on
                                    GB300: 2.50 ms vs 1.73 ms at n=8192) */

/* One problem (Sec. 2): sizes, layout, element types and the paper's
 * parameters.  d1, d2 are the densities (fraction of non-zero entries) of X
 * and Y, mu_prime the mean of the non-zero Rep-factors (Sec. 2.2: "known to
 * the experimenter in advance").  A negative hint means "unknown". */
typedef struct {
    int64_t n;          /* X, Y, Z are n x n, n >= 0 */
    int64_t ldx, ldy, ldz; /* leading dimensions (elements); 0 means n */
    int32_t kase;       /* afmm_case */
    int32_t x_dtype, y_dtype, z_dtype;  /* afmm_dtype */
    int32_t target;     /* afmm_target */
    int32_t variant;    /* afmm_variant; AFMM_VARIANT_AUTO to let the plan pick */
    uint32_t flags;     /* AFMM_FLAG_* */
    int32_t reserved_;  /* must be 0 */
    double d1, d2, mu_prime;  /* hints, < 0 when unknown */
    /* Magnitude hints for the exact tensor-core form (< 0 when unknown):
     * the largest Rep-factor and the largest |Base| value.  They size the
     * K chunks whose FP32 partial sums must stay exact; every call checks
     * the data against them on the device (AFMM_ERR_OVERFLOW_RISK at
     * afmm_plan_sync when a value exceeds its hint). */
    double rep_max, base_max;
} afmm_desc;

/* What a plan decided and, after a validating call, what it measured. */
typedef struct {
    int32_t variant;        /* afmm_variant the plan runs */
    int32_t slices;         /* slices of the real factor (1 when unsliced) */
    int32_t slice_bits;     /* bits per slice for the integer-slice forms */
    int32_t k_split;        /* K chunks kept apart for exactness (>= 1) */
    uint64_t workspace_bytes;
    /* Measured by the last validating call (-1 before one ran): */
    double d1, d2;          /* realised densities of X and Y */
    double mu_prime, mu;    /* mean of non-zero / of all Rep-factors */
    double rep_max;         /* largest Rep-factor */
    double expected_additions;  /* mu' d1 d2 n^3 (Sec. 2.2) */
} afmm_info;

typedef struct afmm_plan_s* afmm_plan;

/* Human-readable name of a status code (static storage, never NULL). */
const char* afmm_status_string(afmm_status s);

/* Text of the last CUDA failure seen by this thread (empty if none). */
const char* afmm_last_error_detail(void);

/* Library version as major*10000 + minor*100 + patch. */
int afmm_version(void);

/* Create a plan for one problem (Sec. 2 problem statement).  Validates the
 * descriptor, picks the variant (a forced variant is honoured or refused
 * with AFMM_ERR_UNSUPPORTED), sizes the workspace.  Allocates nothing on
 * the device.  *out receives the plan (NULL on error). */
afmm_status afmm_plan_create(afmm_plan* out, const afmm_desc* desc);

/* Destroy a plan and free what it owns (not a lent workspace).  NULL is
 * accepted and ignored.  The caller must not use the plan afterwards. */
afmm_status afmm_plan_destroy(afmm_plan plan);

/* Device workspace the plan needs, in bytes (may be 0). */
afmm_status afmm_plan_workspace_size(afmm_plan plan, size_t* bytes);

/* Lend the plan a device workspace of at least afmm_plan_workspace_size
 * bytes, 256-byte aligned.  Without one the plan allocates its own on first
 * use.  The caller keeps ownership and must keep it alive while the plan
 * runs on it. */
afmm_status afmm_plan_set_workspace(afmm_plan plan, void* workspace,
                                    size_t bytes);

/* Case A product (Sec. 2, Case-A): X real Base values, Y Rep-factors.
 * Z = X * Y, overwritten.  The plan must have been created with
 * kase == AFMM_CASE_A.
 * Every call of either case checks the Rep-factors (Sec. 2 types them as
 * non-negative integers; no flag needed): a negative one is reported as
 * AFMM_ERR_NEGATIVE_REP, a non-integer one (NaN and infinities included)
 * as AFMM_ERR_NONINTEGER_REP, by afmm_plan_sync (or the next call's
 * status); Z is then unspecified.  Most forms check in the conversion or
 * compaction that reads the Rep-factors anyway; the FP32 CUDA-core form
 * reads them in place and runs one check pass first (none for u8
 * Rep-factors, which cannot be invalid).  Negative Base values are valid. */
afmm_status afmm_mul_caseA(afmm_plan plan, const void* X, const void* Y,
                           void* Z, void* stream);

/* Case B product (Sec. 2, Case-B): X Rep-factors, Y real Base values.
 * The plan must have been created with kase == AFMM_CASE_B. */
afmm_status afmm_mul_caseB(afmm_plan plan, const void* X, const void* Y,
                           void* Z, void* stream);

/* Product of two real matrices, Z = X * Y (no Rep-factor: the Sec. 4
 * generalisation).  X and Y F32, F64, BF16 or integer typed, Z F32, FP32
 * target.  The plan must have been created with kase == AFMM_CASE_REAL;
 * its variant is AFMM_VARIANT_TC_BF16X3X3 (tensor cores) or
 * AFMM_VARIANT_SIMT_F32 (CUDA cores, skipping zero entries of X). */
afmm_status afmm_mul_real(afmm_plan plan, const void* X, const void* Y, void* Z,
                          void* stream);

/* Rows [r0, r1) of Z = X * Y from rows [r0, r1) of X and all of Y (Sec.
 * 2.1: row I of Z is final once the K loop of row I is done, and it needs
 * row I of X only), for splitting one product into row blocks, e.g. one
 * block per GPU with Y copied to each.  Xrows points at row r0 of X (the
 * plan's ldx), Zrows at row r0 of Z (ldz); both hold r1 - r0 rows; Y is the
 * whole n x n factor.  Device pointers only (AFMM_ERR_INVALID_ARG for host
 * memory).  Case A or B plans running AFMM_VARIANT_TC_BF16X3, _TC_BF16X2 or
 * _TC_FP8X4 (others: AFMM_ERR_UNSUPPORTED); 0 <= r0 <= r1 <= n.  Each row
 * block equals the same rows of a whole-product call bit for bit.
 * Rep-factors are checked as in afmm_mul_caseA; asynchronous on `stream`. */
afmm_status afmm_mul_rows(afmm_plan plan, int64_t r0, int64_t r1, const void* Xrows,
                          const void* Y, void* Zrows, void* stream);

/* Wait for the plan's work on `stream` and return the first error a kernel
 * recorded since the previous sync (clearing it), else AFMM_OK. */
afmm_status afmm_plan_sync(afmm_plan plan, void* stream);

/* The plan's decisions and, after a validating call and a sync, the
 * measured parameters of the last instance. */
afmm_status afmm_get_info(afmm_plan plan, afmm_info* out);

/* Counters of a plan, for measurement.  When kernel timing is enabled the
 * plan records a CUDA event pair around its main product kernel on the
 * call's stream (the events are timed on that stream, so they measure that
 * kernel's launches only).  afmm_plan_counters synchronises those events. */
typedef struct {
    int64_t calls;             /* afmm_mul_* calls on this plan */
    int64_t kernel_launches;   /* kernels those calls launched */
    int64_t timed_launches;    /* main-kernel launches timed by events */
    double timed_ms;           /* their summed duration, milliseconds */
    int32_t main_kernel_ctas;  /* grid size of the last main-kernel launch */
    int32_t reserved_;
    /* Plain FP32 variant on its zero-skip kernel (Base density hint below
     * 0.16): the 32-wide k tiles its CTAs multiplied since the workspace
     * was bound, summed over calls.  A CTA skips a k tile whose 64 x 32 tile
     * of the first factor or 32 x 256 tile of the second is all zero (the
     * K0 tile masks, Sec. 2's zero-skip at tile granularity).  Read with a
     * device synchronisation; -1 for every other variant. */
    int64_t simt_k_tiles;
} afmm_counters;

/* Enable (1) or disable (0) event timing of the main kernel; enabling
 * resets the timed totals. */
afmm_status afmm_plan_enable_kernel_timing(afmm_plan plan, int enable);
afmm_status afmm_plan_counters(afmm_plan plan, afmm_counters* out);

/* Self-test of the bounded waits every tensor-core kernel uses: launches
 * one CTA that waits on an mbarrier nothing will complete, for at most
 * `limit_ns` nanoseconds (capped at 2 s), and returns the status the
 * kernel recorded: AFMM_ERR_TIMEOUT when the wait ran out as designed.
 * The CUDA context stays usable.  Synchronises `stream`. */
afmm_status afmm_selftest_bounded_wait(uint64_t limit_ns, void* stream);

/* Batched product: `count` independent instances (Sec. 2 problems of
 * different n, Case A or B), each described by descs[t], FP32 target
 * (z_dtype F32).  Each instance takes one of three routes: the tcgen05
 * split-BF16 form with 128 x 256 output tiles (AFMM_VARIANT_TC_BF16X3) or
 * with 128 x 128 tiles (AFMM_VARIANT_TC_BF16X3_N128), or the CUDA-core
 * zero-skip form (AFMM_VARIANT_SIMT_F32).  descs[t].variant forces the
 * route; AFMM_VARIANT_AUTO asks the installed dispatch model
 * (afmm_set_dispatch_model) or, without one, applies the built-in rule
 * (128 x 256 tensor-core tiles unless the Base density hint is below 0.02
 * or n < 32).  All tensor-core instances, of both tile widths, run in one
 * persistent grouped launch, all CUDA-core instances in another; the first call with a given
 * descriptor array builds the plan (workspace, TMA descriptors, tile lists)
 * and a CUDA graph of the launches, later calls with an identical array
 * only refresh the pointer table and launch the graph (a few plans are
 * cached).  X[t], Y[t], Z[t] are device pointers; Z[t] depends only on X[t]
 * and Y[t].  Asynchronous on `stream`; calls with the same descriptor array
 * must not overlap on different streams.  Rep-factors are checked on
 * every call: a negative one, a non-integer one or one above 256 is
 * reported by afmm_batched_sync (AFMM_ERR_NEGATIVE_REP,
 * AFMM_ERR_NONINTEGER_REP, AFMM_ERR_OVERFLOW_RISK) and turns a
 * tensor-core instance's Z into NaN (a CUDA-core instance's Z is then
 * unspecified); a bounded wait that runs out is reported the same way. */
afmm_status afmm_mul_batched(int count, const afmm_desc* descs,
                             const void* const* X, const void* const* Y,
                             void* const* Z, void* stream);

/* Synchronise `stream` and return the status recorded by the kernels of the
 * cached batch with this descriptor array (AFMM_OK, a Rep-factor error, or
 * AFMM_ERR_TIMEOUT), clearing it; AFMM_ERR_INVALID_ARG when no such batch
 * ran. */
afmm_status afmm_batched_sync(int count, const afmm_desc* descs, void* stream);

/* Relative error of a result against a reference, in FP64 on the GPU:
 * out[0] = ||Z - R||_F, out[1] = ||R||_F, out[2] = max |Z - R| over the
 * rows x cols matrices (row-major, leading dimensions ldz, ldr; dtypes F64,
 * F32 or I32).  Device pointers; `out` is host memory, filled before
 * return (the call synchronises `stream`).  `workspace` is a device buffer
 * of afmm_error_norm_workspace_size() bytes, or NULL to let the call
 * allocate and free one. */
size_t afmm_error_norm_workspace_size(int64_t rows, int64_t cols);
afmm_status afmm_error_norm(const void* Z, int32_t z_dtype, int64_t ldz,
                            const void* R, int32_t r_dtype, int64_t ldr,
                            int64_t rows, int64_t cols, void* workspace,
                            double out[3], void* stream);

/* ------------------------------------------------------------------
 * Learned dispatch of batched instances (the paper has no counterpart:
 * Sec. 2.2's addition count mu' d1 d2 n^3 is one of the model's inputs).
 * A small MLP maps AFMM_DISPATCH_FEATURES features of an instance to one
 * predicted log2-time per kernel variant; the batch planner picks the
 * variant with the smallest prediction.  Parameters are FP32, flat,
 * row-major: [W1 (F x H), b1 (H), W2 (H x H), b2 (H), W3 (H x V), b3 (V)];
 * H1 = relu(x W1 + b1), H2 = relu(H1 W2 + b2), p = H2 W3 + b3.
 * ------------------------------------------------------------------ */
#define AFMM_DISPATCH_FEATURES 10
typedef struct {
    int32_t features, hidden, outputs, reserved_;
} afmm_mlp_shape;

/* Features of one instance, from its descriptor (hints used as given):
 * log2 n, Base density, Rep density, log2(1 + mu'), case (0 A, 1 B),
 * log2(1 + mu' d1 d2 n^3), log2 n^3, (1 - Base density)^8, and the padded
 * area of 256-wide and of 128-wide output tiles relative to n
 * (ceil(n / 256) * 256 / n, ceil(n / 128) * 128 / n).  out holds
 * AFMM_DISPATCH_FEATURES floats (host memory). */
afmm_status afmm_dispatch_features(const afmm_desc* desc, float* out);

int64_t afmm_mlp_param_count(const afmm_mlp_shape* shape);
/* Device scratch (floats) the forward / training calls need for `rows`. */
int64_t afmm_mlp_work_floats(const afmm_mlp_shape* shape, int rows);

/* P (rows x outputs) = MLP(X) (rows x features), device pointers. */
afmm_status afmm_mlp_forward(const afmm_mlp_shape* shape, const float* params,
                             const float* X, int rows, float* P, float* work,
                             void* stream);

/* Mean-squared error over the observed targets (mask M = 1) and its
 * gradient with respect to every parameter: loss (device float) =
 * sum M (P - T)^2 / count, grads laid out like params.  Device pointers. */
afmm_status afmm_mlp_loss_grad(const afmm_mlp_shape* shape, const float* params,
                               const float* X, const float* T, const float* M,
                               int rows, float count, float* grads, float* work,
                               float* loss, void* stream);

/* One Adam step (bias-corrected, step >= 1) on n parameters, in place. */
afmm_status afmm_mlp_adam(int64_t n, float* params, const float* grads, float* m,
                          float* v, float lr, float beta1, float beta2, float eps,
                          int step, void* stream);

/* Install the dispatch model used for batched instances whose variant is
 * AFMM_VARIANT_AUTO (host copies are kept; NULL params removes it):
 * features are normalised as (x - mean) / scale, and output o predicts the
 * time of variant variant_of_output[o]. */
afmm_status afmm_set_dispatch_model(const afmm_mlp_shape* shape, const float* params,
                                    const float* feat_mean, const float* feat_scale,
                                    const int32_t* variant_of_output);

/* The variant the batch planner would give this instance (host call). */
int32_t afmm_dispatch_variant(const afmm_desc* desc);

/* FP64-target product that allocates nothing (the paper has no counterpart:
 * this entry point exists for callers of this library, not for the method).
 *
 * Who needs it: callers that cannot call cudaMalloc -- for example code
 * running while another allocator holds all of the device's memory, loops
 * that cannot afford the device synchronisation cudaMalloc and cudaFree
 * imply, or hosts that forbid allocation from the context they call in.
 *
 * What it computes: the same product as a plan with target
 * AFMM_TARGET_FP64 (row-scaled 7-bit digits of the real factor, exact int32
 * digit products, FP64 recombination), Case A or B as desc->kase says.
 * X, Y, Z are DEVICE pointers laid out as desc describes (dtypes, leading
 * dimensions; z_dtype must be AFMM_F64); the caller owns them.  Hints and
 * desc->variant are ignored.
 *
 * Scratch: one fixed device array of about 3.8 MiB inside this library,
 * enough for n <= 256; n > 256 returns AFMM_ERR_UNSUPPORTED (and
 * afmm_last_error_detail says so).  Under CUDA's default lazy module
 * loading the array and this library's device code take their device
 * memory on the first use on each device (a call of this or any other
 * entry point), unless CUDA_MODULE_LOADING=EAGER is set; a device then
 * holds them until the process exits.  So a caller whose memory will later
 * be taken over by another allocator makes one small warm-up call per
 * device first, and that first call should also come before any stream
 * capture.  Each call looks up the array's device address
 * (cudaGetSymbolAddress with the device current), which allocates nothing
 * once the code is loaded and stays right after a cudaDeviceReset.
 *
 * Calls share the array and keep its last contents (the call clears what
 * must start at zero).  Calls that overlap on the GPU -- issued on several
 * streams or from several threads without ordering -- race on it.
 *
 * Asynchronous on `stream`.  A negative or non-integer Rep-factor (NaN
 * included) or one above 127 cannot be reported through a status word
 * without allocating one per call, so it turns every element of Z into NaN
 * instead.  Returns AFMM_ERR_INVALID_ARG for a bad descriptor, a host
 * pointer, or a device pointer of another device than the current one. */
afmm_status afmm_mul_noalloc(const afmm_desc* desc, const void* X,
                             const void* Y, void* Z, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AFMM_H */
