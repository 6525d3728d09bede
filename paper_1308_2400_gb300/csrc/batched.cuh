// Batched products: shared records of the planner (batched.cpp) and the
// grouped kernels (batched_kernels.cu).  Plain host/device structs.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "afmm.h"

namespace afmm {

// Tile shape of the grouped tensor-core kernel.
constexpr int GB_BM = 128, GB_BN = 256, GB_BK = 32;

// Rows per block of the B-operand transposition for Case A instances whose
// Rep-factors are one-byte elements (byte tiles; every other instance is
// transposed in 64 x 64 tiles).  Columns per block: 64.
constexpr int GB_U8_ROWS = 128;

// Blocks of the B-operand transposition of an instance of size n.
inline int64_t g_transpose_blocks(int64_t n, bool byte_tiles) {
    const int64_t cols = (n + 63) / 64;
    return byte_tiles ? (n + GB_U8_ROWS - 1) / GB_U8_ROWS * cols : cols * cols;
}

// Device record of one tensor-core instance.
struct GInst {
    const void* X;
    const void* Y;
    float* Z;
    void* A;               // BF16, K-major A operand(s): [S][n][ldk]
    void* B;               // BF16, K-major B operand(s): [S][n][ldk]
    int64_t n, ldx, ldy, ldz, ldk;
    int kind;              // 0: X real, sliced on A; 1: Y real, sliced on B
    int x_dtype, y_dtype;
    int flag;              // index into the per-instance error flags
    int bn;                // output tile width: 256, or 128 (route 2)
    int pad_;
};

// Device record of one operand widened to FP32 for the CUDA-core form
// (dst null: an FP32 Rep-factor operand that is only checked).
struct WJob {
    const void* src;
    float* dst;
    int64_t n, lds;
    int dtype;
    int rep;               // the operand holds Rep-factors: check them
};

// One tensor-core tile: instance, tile row, tile column.
struct TileRec {
    int inst, tm, tn, pad;
};

// Grouped launches (device arrays throughout).
afmm_status launch_batch_convert(const GInst* inst, const int* row_prefix,
                                 const int* row_job, const int* tt_prefix,
                                 const int* tt_job, int ninst, int rows_total,
                                 int tt_total, int* flags, int* status, cudaStream_t st);
afmm_status launch_batch_tc(const GInst* inst, const void* maps, const int* cta_off,
                            const int* tiles, int grid, const int* flags, int* status,
                            cudaStream_t st);
afmm_status launch_batch_widen(const WJob* jobs, const int* prefix, int njobs,
                               int rows_total, int* status, cudaStream_t st);

// Routes of a batched instance: 0 CUDA cores, 1 tensor cores with 128 x 256
// tiles, 2 tensor cores with 128 x 128 tiles.
// Route of an instance under the built-in rule (0 or 1).
int batch_rule_route(const afmm_desc& d);
// Enqueue `count` independent products on `stream`; `kernels_out` receives
// the number of kernels one call launches.
afmm_status batched_run(int count, const afmm_desc* descs, const void* const* X,
                        const void* const* Y, void* const* Z, void* stream,
                        int* kernels_out);
// Status word of the cached batch with these descriptors (after a sync).
afmm_status batched_status(int count, const afmm_desc* descs, int* out);
void batched_clear_cache();
// Learned dispatch (batched.cpp).
afmm_status dispatch_features(const afmm_desc& d, float* out);
afmm_status set_dispatch_model(const afmm_mlp_shape* s, const float* params,
                               const float* mean, const float* scale,
                               const int32_t* variants);
int dispatch_route(const afmm_desc& d);   // route 0, 1 or 2 (see above)

}  // namespace afmm
