// C ABI of libafmm (include/afmm.h): plans, the planner that picks a
// kernel variant for a problem of Sec. 2, workspace layout, host-buffer
// staging and the device status word.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "afmm_common.cuh"
#include "batched.cuh"
#include "tc_gemm.cuh"

namespace afmm {

namespace {
thread_local char g_last_err[512] = {0};
}

void set_last_cuda_error(cudaError_t e, const char* what, const char* file,
                         int line) {
    snprintf(g_last_err, sizeof(g_last_err), "%s (%d) in %s at %s:%d",
             cudaGetErrorString(e), (int)e, what, file, line);
}

namespace {
thread_local int64_t g_launches = 0;
thread_local MainTimer* g_timer = nullptr;
}
void count_launches(int k) { g_launches += k; }
int64_t launch_counter() { return g_launches; }
MainTimer* current_main_timer() { return g_timer; }
void set_main_timer(MainTimer* t) { g_timer = t; }
void main_kernel_begin(cudaStream_t st) {
    // A call that splits its product into several launches is timed from
    // the first one's start to the last one's end.
    if (g_timer && g_timer->start && !g_timer->started) {
        cudaEventRecord(g_timer->start, st);
        g_timer->started = true;
    }
}
void main_kernel_end(cudaStream_t st, int ctas) {
    if (g_timer && g_timer->stop) {
        cudaEventRecord(g_timer->stop, st);
        g_timer->ctas = ctas;
    }
}

void set_last_error_text(const char* text) {
    snprintf(g_last_err, sizeof(g_last_err), "%s", text);
}

afmm_status device_props(DeviceProps* out) {
    static std::mutex mu;
    static DeviceProps cache[64];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return AFMM_ERR_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lk(mu);
    DeviceProps& p = cache[dev];
    if (p.device != dev) {
        int v = 0;
        AFMM_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        p.sm_count = v;
        AFMM_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, dev));
        p.cc_major = v;
        AFMM_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMinor, dev));
        p.cc_minor = v;
        AFMM_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        p.smem_optin = (size_t)v;
        p.device = dev;
    }
    *out = p;
    return AFMM_OK;
}

}  // namespace afmm

using namespace afmm;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Plain FP32 variant: the dense CUDA-core kernel unless the Base density
// hint is low.  Zero-skip gains on whole 4-row groups of zero Base values,
// (1 - d1)^4 of them.  Measured at n = 8192: zero-skip 18.7 ms at d1 = 0.15
// and 21.5 ms at 0.2, the dense kernel 19.1 ms at any density.  No hint:
// dense.
constexpr double kSimtDenseMinD1 = 0.16;
inline bool simt_dense(const afmm_desc& d) {
    return d.d1 < 0.0 || d.d1 >= kSimtDenseMinD1;
}

// FP64-target slicing: 8 digits of 7 bits (56 bits of each row-scaled
// value), each an int8, so products run on int8 dot products.
constexpr int kF64Bits = 7;
constexpr int kF64Slices = 8;

}  // namespace

struct afmm_plan_s {
    afmm_desc d;
    int variant = 0;
    int slices = 1, bits = 0, ksplit = 1;
    // Workspace layout (byte offsets; 0 size means unused).
    size_t ws_bytes = 0;
    size_t off_status = 0, off_sx = 0, off_sy = 0, off_part = 0;
    size_t off_a = 0, off_b = 0, off_c = 0, off_e = 0;
    size_t off_t1 = 0, off_t2 = 0, off_t3 = 0;
    int64_t lda = 0, ldb = 0;           // leading dims of converted operands
    char* ws = nullptr;
    bool ws_owned = false;
    bool ws_ready = false;              // status word zeroed
    bool validated = false;
    // Staging buffers for host pointers (owned).
    void* stage[3] = {nullptr, nullptr, nullptr};
    size_t stage_bytes[3] = {0, 0, 0};
    TcPlan tc;                          // tensor-core state (tensor maps)
    // Measurement counters.
    int64_t calls = 0, launches = 0, timed = 0;
    double timed_ms = 0.0;
    int last_ctas = 0;
    bool timing = false;
    std::vector<MainTimer> pending, spare;
    // Transfer pipelining of host buffers (created on first use).
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev[2 * 16 + 2] = {};
    // Replay of repeated calls on the same device buffers (small problems,
    // where the gaps between launches are a large part of a call): the
    // third call in a row with the same X, Y, Z is captured into a CUDA
    // graph on a private stream; later ones launch it.
    const void* g_x = nullptr;
    const void* g_y = nullptr;
    void* g_z = nullptr;
    int g_seen = 0;
    bool g_off = false;                 // capture failed once: stay eager
    cudaGraphExec_t g_exec = nullptr;
    cudaStream_t g_cap = nullptr;
    int64_t g_launches = 0;
};

namespace {

bool rep_dtype_ok(int dt) {
    return dt == AFMM_I32 || dt == AFMM_I8 || dt == AFMM_U8 ||
           dt == AFMM_E4M3 || dt == AFMM_BF16 || dt == AFMM_F32;
}
bool real_dtype_ok(int dt) {
    return dt == AFMM_F64 || dt == AFMM_F32 || dt == AFMM_BF16;
}

// Byte span of an n x n row-major matrix with leading dimension ld.
size_t span_bytes(int64_t n, int64_t ld, int dt) {
    if (n <= 0) return 0;
    return (size_t)((n - 1) * ld + n) * dtype_size(dt);
}

afmm_status check_desc(const afmm_desc* d) {
    if (!d) return AFMM_ERR_INVALID_ARG;
    if (d->n < 0 || d->reserved_ != 0) return AFMM_ERR_INVALID_ARG;
    if (d->kase != AFMM_CASE_A && d->kase != AFMM_CASE_B && d->kase != AFMM_CASE_REAL)
        return AFMM_ERR_INVALID_ARG;
    if (d->target < AFMM_TARGET_FP32 || d->target > AFMM_TARGET_EXACT)
        return AFMM_ERR_INVALID_ARG;
    if (d->variant < AFMM_VARIANT_AUTO || d->variant >= AFMM_VARIANT_COUNT_)
        return AFMM_ERR_INVALID_ARG;
    for (int dt : {d->x_dtype, d->y_dtype, d->z_dtype})
        if (dtype_size(dt) == 0) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d->n;
    const int64_t ldx = d->ldx ? d->ldx : n, ldy = d->ldy ? d->ldy : n,
                  ldz = d->ldz ? d->ldz : n;
    if (ldx < n || ldy < n || ldz < n) return AFMM_ERR_INVALID_ARG;
    if (d->kase == AFMM_CASE_REAL) {
        // Two real factors: FP32 target only.
        for (int dt : {d->x_dtype, d->y_dtype})
            if (!real_dtype_ok(dt) && !dtype_is_integer(dt)) return AFMM_ERR_INVALID_ARG;
        if (d->target != AFMM_TARGET_FP32 || d->z_dtype != AFMM_F32)
            return AFMM_ERR_INVALID_ARG;
        return AFMM_OK;
    }
    const int rep_dt = d->kase == AFMM_CASE_A ? d->y_dtype : d->x_dtype;
    const int base_dt = d->kase == AFMM_CASE_A ? d->x_dtype : d->y_dtype;
    if (!rep_dtype_ok(rep_dt)) return AFMM_ERR_INVALID_ARG;
    if (d->target == AFMM_TARGET_EXACT) {
        if (!dtype_is_integer(base_dt) || !dtype_is_integer(rep_dt) ||
            d->z_dtype != AFMM_I32)
            return AFMM_ERR_INVALID_ARG;
    } else {
        if (!real_dtype_ok(base_dt) && !dtype_is_integer(base_dt))
            return AFMM_ERR_INVALID_ARG;
        if (d->target == AFMM_TARGET_FP32 && d->z_dtype != AFMM_F32)
            return AFMM_ERR_INVALID_ARG;
        if (d->target == AFMM_TARGET_FP64 && d->z_dtype != AFMM_F64)
            return AFMM_ERR_INVALID_ARG;
    }
    return AFMM_OK;
}

bool variant_serves(int v, const afmm_desc* d) {
    if (d->kase == AFMM_CASE_REAL)
        return v == AFMM_VARIANT_SIMT_F32 ||
               (v == AFMM_VARIANT_TC_BF16X3X3 && tc_available());
    switch (v) {
        case AFMM_VARIANT_SIMT_F32:
            return d->target == AFMM_TARGET_FP32;
        case AFMM_VARIANT_TC_BF16X3:
        case AFMM_VARIANT_TC_BF16X2:
        case AFMM_VARIANT_TC_FP8X4:
            return d->target == AFMM_TARGET_FP32 && tc_available();
        case AFMM_VARIANT_TC_F16X2:
            return d->target == AFMM_TARGET_FP32 && tc_available();
        case AFMM_VARIANT_SIMT_F64SLICE:
            return d->target == AFMM_TARGET_FP64;
        case AFMM_VARIANT_SIMT_EXACT:
            return d->target == AFMM_TARGET_EXACT;
        case AFMM_VARIANT_TC_EXACT:
            return d->target == AFMM_TARGET_EXACT && tc_available();
        case AFMM_VARIANT_TC_EXACT_F8:
            return d->target == AFMM_TARGET_EXACT && d->n >= 512 && tc_available();
        case AFMM_VARIANT_SPARSE:
            return d->target == AFMM_TARGET_FP32;
        default:
            return false;
    }
}

int auto_variant(const afmm_desc* d) {
    if (d->kase == AFMM_CASE_REAL)
        return (tc_available() && d->n >= 128) ? AFMM_VARIANT_TC_BF16X3X3
                                               : AFMM_VARIANT_SIMT_F32;
    if (d->target == AFMM_TARGET_EXACT) {
        // E4M3 digits when the magnitude hints fit them (twice the BF16
        // rate and a quarter fewer staged bytes per MMA).
        if (tc_available() && d->n >= 512 && d->n < 65536 &&
            d->rep_max >= 0.0 && d->rep_max <= 16.0 && d->base_max >= 0.0 &&
            d->base_max <= 255.0)
            return AFMM_VARIANT_TC_EXACT_F8;
        return (tc_available() && d->n >= 128) ? AFMM_VARIANT_TC_EXACT
                                               : AFMM_VARIANT_SIMT_EXACT;
    }
    if (d->target == AFMM_TARGET_FP64) return AFMM_VARIANT_SIMT_F64SLICE;
    // FP32 target.  Quadratic regime of Sec. 2.2 (on average at most a few
    // non-zero terms per element of Z): both factors compacted.
    if (d->d1 >= 0.0 && d->d2 >= 0.0 && d->d1 * d->d2 * (double)d->n <= 4.0 &&
        d->n >= 64)
        return AFMM_VARIANT_SPARSE;
    // Tensor cores for the dense regime; the zero-skipping CUDA-core kernel
    // when the Base factor is very sparse (the useful work mu' d1 d2 n^3 is
    // then far below the dense n^3).
    const double dbase = d->kase == AFMM_CASE_A ? d->d1 : d->d2;
    if (tc_available() && d->n >= 128 && !(dbase >= 0.0 && dbase < 0.05))
        return AFMM_VARIANT_TC_BF16X3;
    return AFMM_VARIANT_SIMT_F32;
}

// Bump allocator for the workspace layout.
struct Layout {
    size_t top = 0;
    size_t take(size_t bytes) {
        if (bytes == 0) return 0;
        size_t off = align_up(top, kAlign);
        top = off + align_up(bytes, kAlign);
        return off;
    }
};

void plan_layout(afmm_plan_s* p) {
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    Layout L;
    L.top = 0;
    p->off_status = L.take(kAlign);
    p->off_sx = L.take(sizeof(ScanStats));
    p->off_sy = L.take(sizeof(ScanStats));
    p->off_part = L.take(sizeof(ScanStats) * kScanMaxBlocks);
    const size_t nn = (size_t)n * (size_t)n;
    switch (p->variant) {
        case AFMM_VARIANT_SIMT_F32: {
            if (simt_dense(d)) {
                p->lda = round_up(n, 4);
                p->off_a = L.take((size_t)n * p->lda * 4);      // X^T
            } else {
                if (d.x_dtype != AFMM_F32) p->off_a = L.take(nn * 4);
                p->off_c = L.take(simt_mask_bytes(n, n, n, nullptr));   // K0 tile masks
            }
            if (d.y_dtype != AFMM_F32) p->off_b = L.take(nn * 4);
            break;
        }
        case AFMM_VARIANT_SIMT_EXACT: {
            p->lda = round_up(n, 4);
            p->ldb = round_up(n, 4);
            p->off_a = L.take((size_t)n * p->lda);
            p->off_b = L.take((size_t)((n + 3) / 4) * p->ldb * 4);
            break;
        }
        case AFMM_VARIANT_SIMT_F64SLICE: {
            p->lda = round_up(n, 4);
            p->ldb = round_up(n, 4);
            p->off_e = L.take((size_t)n * 4);
            p->off_a = L.take((size_t)p->slices * n * p->lda);
            p->off_b = L.take((size_t)((n + 3) / 4) * p->ldb * 4);
            p->off_c = L.take((size_t)p->slices * nn * 4);
            if (d.kase == AFMM_CASE_B) {
                p->off_t1 = L.take(nn * dtype_size(d.y_dtype));
                p->off_t2 = L.take(nn * dtype_size(d.x_dtype));
                p->off_t3 = L.take(nn * 8);
            }
            break;
        }
        case AFMM_VARIANT_SPARSE: {
            p->off_a = L.take(sparse_ws_bytes(n, d.d1, d.d2));
            break;
        }
        case AFMM_VARIANT_TC_EXACT:
        case AFMM_VARIANT_TC_BF16X3:
        case AFMM_VARIANT_TC_BF16X2: {
            tc_layout(&p->tc, d, p->variant == AFMM_VARIANT_TC_EXACT ? 0 : p->slices);
            p->ksplit = p->variant == AFMM_VARIANT_TC_EXACT
                            ? (int)((d.n + 32LL * p->tc.kb_per_chunk - 1) /
                                    (32LL * (p->tc.kb_per_chunk > 0 ? p->tc.kb_per_chunk : 1)))
                            : 1;
            p->off_a = L.take(p->tc.a_bytes);
            p->off_b = L.take(p->tc.b_bytes);
            p->off_c = L.take(p->tc.z_bytes);
            break;
        }
        case AFMM_VARIANT_TC_BF16X3X3: {
            tc_layout(&p->tc, d, p->slices);
            p->off_a = L.take(p->tc.a_bytes);
            p->off_b = L.take(p->tc.b_bytes);
            p->off_c = L.take(p->tc.z_bytes);
            break;
        }
        case AFMM_VARIANT_TC_FP8X4:
        case AFMM_VARIANT_TC_F16X2:
        case AFMM_VARIANT_TC_EXACT_F8: {
            tc_layout(&p->tc, d, p->slices, p->variant == AFMM_VARIANT_TC_FP8X4,
                      p->variant == AFMM_VARIANT_TC_F16X2,
                      p->variant == AFMM_VARIANT_TC_EXACT_F8);
            p->off_a = L.take(p->tc.a_bytes);
            p->off_b = L.take(p->tc.b_bytes);
            p->off_c = L.take(p->tc.z_bytes);
            p->off_e = L.take(p->tc.s_bytes);
            break;
        }
        default:
            break;
    }
    p->ws_bytes = L.top;
}

bool is_host_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

afmm_status ensure_workspace(afmm_plan_s* p, cudaStream_t st) {
    if (!p->ws && p->ws_bytes) {
        void* w = nullptr;
        AFMM_CUDA_TRY(cudaMalloc(&w, p->ws_bytes));
        p->ws = static_cast<char*>(w);
        p->ws_owned = true;
        p->ws_ready = false;
    }
    if (!p->ws_ready) {
        AFMM_CUDA_TRY(cudaMemsetAsync(p->ws + p->off_status, 0, kAlign, st));
        if (p->variant == AFMM_VARIANT_TC_BF16X3 ||
            p->variant == AFMM_VARIANT_TC_BF16X2 ||
            p->variant == AFMM_VARIANT_TC_EXACT || p->variant == AFMM_VARIANT_TC_FP8X4 ||
            p->variant == AFMM_VARIANT_TC_BF16X3X3 || p->variant == AFMM_VARIANT_TC_F16X2 ||
            p->variant == AFMM_VARIANT_TC_EXACT_F8)
            AFMM_TRY(tc_bind_workspace(&p->tc, p->ws + p->off_a, p->ws + p->off_b,
                                       p->ws + p->off_c, p->ws + p->off_e));
        if (p->variant == AFMM_VARIANT_SPARSE) AFMM_TRY(sparse_reset(p->ws + p->off_a, st));
        p->ws_ready = true;
    }
    return AFMM_OK;
}

template <typename T>
T* wsp(afmm_plan_s* p, size_t off) {
    return reinterpret_cast<T*>(p->ws + off);
}

// The zero-skip kernel's count of multiplied k tiles: a 64-bit word after
// the status word (zeroed with it when the workspace is bound).
unsigned long long* simt_ktiles(afmm_plan_s* p) {
    return reinterpret_cast<unsigned long long*>(p->ws + p->off_status + 8);
}

afmm_status run_simt_f32(afmm_plan_s* p, const void* X, const void* Y, void* Z,
                         cudaStream_t st) {
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    const float* A = static_cast<const float*>(X);
    const float* B = static_cast<const float*>(Y);
    int64_t lda = d.ldx ? d.ldx : n, ldb = d.ldy ? d.ldy : n;
    if (simt_dense(d)) {
        float* AT = wsp<float>(p, p->off_a);
        AFMM_TRY(launch_to_f32_transposed(X, d.x_dtype, n, lda, AT, p->lda, st));
        if (d.y_dtype != AFMM_F32) {
            AFMM_TRY(launch_to_f32(Y, d.y_dtype, n, ldb, wsp<float>(p, p->off_b), n, st));
            B = wsp<float>(p, p->off_b);
            ldb = n;
        }
        return launch_simt_f32_dense(AT, p->lda, B, ldb, static_cast<float*>(Z),
                                     d.ldz ? d.ldz : n, n, n, n, st);
    }
    if (d.x_dtype != AFMM_F32) {
        AFMM_TRY(launch_to_f32(X, d.x_dtype, n, lda, wsp<float>(p, p->off_a), n, st));
        A = wsp<float>(p, p->off_a);
        lda = n;
    }
    if (d.y_dtype != AFMM_F32) {
        AFMM_TRY(launch_to_f32(Y, d.y_dtype, n, ldb, wsp<float>(p, p->off_b), n, st));
        B = wsp<float>(p, p->off_b);
        ldb = n;
    }
    // K0 tile masks: k tiles whose A or B tile is all zero are not loaded.
    size_t ym_off = 0;
    simt_mask_bytes(n, n, n, &ym_off);
    uint8_t* xm = wsp<uint8_t>(p, p->off_c);
    AFMM_TRY(launch_tile_masks(A, lda, B, ldb, n, n, n, xm, xm + ym_off, st));
    return launch_simt_f32(A, lda, B, ldb, static_cast<float*>(Z),
                           d.ldz ? d.ldz : n, n, n, n, st, xm, xm + ym_off, simt_ktiles(p));
}

afmm_status run_simt_exact(afmm_plan_s* p, const void* X, const void* Y,
                           void* Z, cudaStream_t st) {
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    int* status = wsp<int>(p, p->off_status);
    AFMM_TRY(launch_pack_a_i8(X, d.x_dtype, n, d.ldx ? d.ldx : n,
                              wsp<int8_t>(p, p->off_a), p->lda, status, st,
                              d.kase == AFMM_CASE_B));
    AFMM_TRY(launch_pack_b_i8(Y, d.y_dtype, n, d.ldy ? d.ldy : n,
                              wsp<int32_t>(p, p->off_b), p->ldb, status, st,
                              d.kase == AFMM_CASE_A));
    return launch_simt_dp4a(wsp<int8_t>(p, p->off_a), p->lda,
                            wsp<int32_t>(p, p->off_b), p->ldb,
                            static_cast<int32_t*>(Z), d.ldz ? d.ldz : n, n, n,
                            n, st);
}

// Case A form: X real, Y Rep-factors.  Z F64.
afmm_status run_f64slice_a(afmm_plan_s* p, const void* X, int xdt, int64_t ldx,
                           const void* Y, int ydt, int64_t ldy, double* Z,
                           int64_t ldz, cudaStream_t st) {
    const int64_t n = p->d.n;
    int* status = wsp<int>(p, p->off_status);
    int32_t* E = wsp<int32_t>(p, p->off_e);
    int8_t* Q = wsp<int8_t>(p, p->off_a);
    int32_t* W = wsp<int32_t>(p, p->off_b);
    int32_t* P = wsp<int32_t>(p, p->off_c);
    AFMM_TRY(launch_exp_slice_rows_i8(X, xdt, n, ldx, E, p->slices, p->bits, Q, p->lda,
                                      st));
    AFMM_TRY(launch_pack_b_i8(Y, ydt, n, ldy, W, p->ldb, status, st, true));
    AFMM_TRY(launch_simt_dp4a(Q, p->lda, W, p->ldb, P, n,
                              (int64_t)p->slices * n, n, n, st));
    return launch_recombine_f64(P, n, E, p->slices, p->bits, n, Z, ldz, st);
}

afmm_status run_simt_f64slice(afmm_plan_s* p, const void* X, const void* Y,
                              void* Z, cudaStream_t st) {
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    const int64_t ldx = d.ldx ? d.ldx : n, ldy = d.ldy ? d.ldy : n,
                  ldz = d.ldz ? d.ldz : n;
    if (d.kase == AFMM_CASE_A)
        return run_f64slice_a(p, X, d.x_dtype, ldx, Y, d.y_dtype, ldy,
                              static_cast<double*>(Z), ldz, st);
    // Case B: Z^T = Y^T X^T, a case-A product of the transposes.
    void* YT = p->ws + p->off_t1;
    void* XT = p->ws + p->off_t2;
    double* ZT = wsp<double>(p, p->off_t3);
    AFMM_TRY(launch_transpose(Y, dtype_size(d.y_dtype), n, n, ldy, YT, n, st));
    AFMM_TRY(launch_transpose(X, dtype_size(d.x_dtype), n, n, ldx, XT, n, st));
    AFMM_TRY(run_f64slice_a(p, YT, d.y_dtype, n, XT, d.x_dtype, n, ZT, n, st));
    return launch_transpose(ZT, 8, n, n, n, Z, ldz, st);
}

afmm_status run_variant(afmm_plan_s* p, const void* X, const void* Y, void* Z,
                        cudaStream_t st) {
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    const bool x_rep = d.kase == AFMM_CASE_B, y_rep = d.kase == AFMM_CASE_A;
    if (d.flags & AFMM_FLAG_VALIDATE) {
        // Rep-factors are checked (non-negative integers); real factors of
        // a real x real plan only counted.
        int* status = wsp<int>(p, p->off_status);
        ScanStats* part = wsp<ScanStats>(p, p->off_part);
        AFMM_TRY(launch_scan(X, d.x_dtype, n, d.ldx ? d.ldx : n, x_rep, part,
                             wsp<ScanStats>(p, p->off_sx), status, st));
        AFMM_TRY(launch_scan(Y, d.y_dtype, n, d.ldy ? d.ldy : n, y_rep, part,
                             wsp<ScanStats>(p, p->off_sy), status, st));
        p->validated = true;
    } else if ((x_rep || y_rep) && p->variant == AFMM_VARIANT_SIMT_F32) {
        // Every call checks the Rep-factors (Sec. 2 types: non-negative
        // integers).  The other forms check them in the conversion or
        // compaction that reads them; this one reads them in place, so a
        // check pass runs first (no launch for u8 Rep-factors, which are
        // always valid).
        AFMM_TRY(launch_rep_check(x_rep ? X : Y, x_rep ? d.x_dtype : d.y_dtype, n,
                                  x_rep ? (d.ldx ? d.ldx : n) : (d.ldy ? d.ldy : n),
                                  wsp<int>(p, p->off_status), st));
    }
    if (n == 0) return AFMM_OK;
    switch (p->variant) {
        case AFMM_VARIANT_SIMT_F32: return run_simt_f32(p, X, Y, Z, st);
        case AFMM_VARIANT_SIMT_EXACT: return run_simt_exact(p, X, Y, Z, st);
        case AFMM_VARIANT_SIMT_F64SLICE: return run_simt_f64slice(p, X, Y, Z, st);
        case AFMM_VARIANT_TC_BF16X3:
        case AFMM_VARIANT_TC_BF16X2:
            return tc_run_split(&p->tc, d, X, Y, Z, wsp<int>(p, p->off_status), st);
        case AFMM_VARIANT_TC_EXACT:
            return tc_run_exact(&p->tc, d, X, Y, Z, wsp<int>(p, p->off_status), st);
        case AFMM_VARIANT_TC_FP8X4:
            return tc_run_fp8(&p->tc, d, X, Y, Z, wsp<int>(p, p->off_status), st);
        case AFMM_VARIANT_TC_F16X2:
            return tc_run_h16(&p->tc, d, X, Y, Z, wsp<int>(p, p->off_status), st);
        case AFMM_VARIANT_TC_EXACT_F8:
            return tc_run_exact_x8(&p->tc, d, X, Y, Z, wsp<int>(p, p->off_status), st);
        case AFMM_VARIANT_TC_BF16X3X3:
            return tc_run_real(&p->tc, d, X, Y, Z, wsp<int>(p, p->off_status), st);
        case AFMM_VARIANT_SPARSE:
            return launch_sparse(X, d.x_dtype, d.ldx ? d.ldx : n, Y, d.y_dtype,
                                 d.ldy ? d.ldy : n, static_cast<float*>(Z),
                                 d.ldz ? d.ldz : n, n, d.d1, d.d2,
                                 p->ws + p->off_a, wsp<int>(p, p->off_status), st,
                                 y_rep ? 1 : (x_rep ? 0 : -1));
        default: return AFMM_ERR_UNSUPPORTED;
    }
}

afmm_status stage_buffer(afmm_plan_s* p, int idx, size_t bytes, void** out) {
    if (p->stage_bytes[idx] < bytes) {
        if (p->stage[idx]) cudaFree(p->stage[idx]);
        p->stage[idx] = nullptr;
        p->stage_bytes[idx] = 0;
        AFMM_CUDA_TRY(cudaMalloc(&p->stage[idx], bytes));
        p->stage_bytes[idx] = bytes;
    }
    *out = p->stage[idx];
    return AFMM_OK;
}

// Host X, Y, Z and the split tensor-core form: copy Y in, convert it; then
// for row blocks of X: copy in (stream s_in), convert and multiply (the
// call's stream), copy the rows of Z out (stream s_out), so transfers in
// both directions overlap the products.  Pinned host memory makes the
// copies asynchronous; pageable memory still gives the right result.
afmm_status run_pipelined_host(afmm_plan_s* p, const void* X, const void* Y, void* Z,
                               cudaStream_t st) {
    const afmm_desc& d = p->d;
    const int64_t n = d.n, ldx = d.ldx, ldz = d.ldz;
    const size_t ex = dtype_size(d.x_dtype), ez = dtype_size(d.z_dtype);
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    if (!p->s_in) {
        AFMM_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
        AFMM_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
        for (auto& e : p->ev) AFMM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    void *dX, *dY, *dZ;
    AFMM_TRY(stage_buffer(p, 2, span_bytes(n, ldz, d.z_dtype), &dZ));
    int* status = wsp<int>(p, p->off_status);
    int64_t bounds[17];
    const int nb = tc_pipe_blocks(n, dp.sm_count, bounds, 16, d.kase == AFMM_CASE_B,
                                  p->tc.pair && !p->tc.f8);
    cudaEvent_t ev_y = p->ev[0], ev_done = p->ev[1];
    AFMM_TRY(stage_buffer(p, 0, span_bytes(n, ldx, d.x_dtype), &dX));
    AFMM_TRY(stage_buffer(p, 1, span_bytes(n, d.ldy, d.y_dtype), &dY));
    // The staging buffers may still be read by the previous call's copies.
    AFMM_CUDA_TRY(cudaEventRecord(ev_done, st));
    AFMM_CUDA_TRY(cudaStreamWaitEvent(p->s_in, ev_done, 0));
    AFMM_CUDA_TRY(cudaMemcpyAsync(dY, Y, span_bytes(n, d.ldy, d.y_dtype),
                                  cudaMemcpyHostToDevice, p->s_in));
    AFMM_CUDA_TRY(cudaEventRecord(ev_y, p->s_in));
    AFMM_CUDA_TRY(cudaStreamWaitEvent(st, ev_y, 0));
    AFMM_TRY(tc_split_prepare_b(&p->tc, d, dY, status, st));
    for (int b = 0; b < nb; ++b) {
        const int64_t r0 = bounds[b], r1 = bounds[b + 1];
        cudaEvent_t e_in = p->ev[2 + 2 * b], e_c = p->ev[3 + 2 * b];
        const size_t xoff = (size_t)r0 * ldx * ex;
        const size_t xbytes = (size_t)((r1 - r0 - 1) * ldx + n) * ex;
        AFMM_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(dX) + xoff,
                                      static_cast<const char*>(X) + xoff, xbytes,
                                      cudaMemcpyHostToDevice, p->s_in));
        AFMM_CUDA_TRY(cudaEventRecord(e_in, p->s_in));
        AFMM_CUDA_TRY(cudaStreamWaitEvent(st, e_in, 0));
        AFMM_TRY(tc_split_rows(&p->tc, d, dX, dZ, r0, r1, status, st));
        AFMM_CUDA_TRY(cudaEventRecord(e_c, st));
        AFMM_CUDA_TRY(cudaStreamWaitEvent(p->s_out, e_c, 0));
        const size_t zoff = (size_t)r0 * ldz * ez;
        const size_t zbytes = (size_t)((r1 - r0 - 1) * ldz + n) * ez;
        AFMM_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(Z) + zoff,
                                      static_cast<const char*>(dZ) + zoff, zbytes,
                                      cudaMemcpyDeviceToHost, p->s_out));
    }
    AFMM_CUDA_TRY(cudaEventRecord(ev_done, p->s_out));
    AFMM_CUDA_TRY(cudaStreamWaitEvent(st, ev_done, 0));
    AFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return AFMM_OK;
}

constexpr int64_t kGraphMaxN = 2048;

void graph_drop(afmm_plan_s* p) {
    if (p->g_exec) cudaGraphExecDestroy(p->g_exec);
    p->g_exec = nullptr;
}

// Device-buffer call through the replay graph: *done is true when the
// product was launched here (replayed, or captured and launched).
afmm_status graph_call(afmm_plan_s* p, const void* X, const void* Y, void* Z,
                       cudaStream_t st, bool* done) {
    *done = false;
    if (X != p->g_x || Y != p->g_y || Z != p->g_z) {
        graph_drop(p);
        p->g_x = X;
        p->g_y = Y;
        p->g_z = Z;
        p->g_seen = 1;
        return AFMM_OK;
    }
    if (!p->g_exec) {
        if (++p->g_seen < 3) return AFMM_OK;
        if (!p->g_cap)
            AFMM_CUDA_TRY(cudaStreamCreateWithFlags(&p->g_cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        AFMM_CUDA_TRY(cudaStreamBeginCapture(p->g_cap, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = launch_counter();
        const afmm_status rc = run_variant(p, X, Y, Z, p->g_cap);
        const cudaError_t ec = cudaStreamEndCapture(p->g_cap, &g);
        p->g_launches = launch_counter() - l0;
        count_launches((int)-p->g_launches);      // nothing ran yet
        cudaError_t ei = cudaErrorUnknown;
        if (rc == AFMM_OK && ec == cudaSuccess && g)
            ei = cudaGraphInstantiate(&p->g_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            (void)cudaGetLastError();               // capture errors are not sticky
            p->g_exec = nullptr;
            p->g_off = true;                        // this plan stays eager
            return AFMM_OK;
        }
    }
    AFMM_CUDA_TRY(cudaGraphLaunch(p->g_exec, st));
    count_launches((int)p->g_launches);
    p->launches += p->g_launches;
    p->calls += 1;
    *done = true;
    return AFMM_OK;
}

afmm_status mul_impl(afmm_plan p, const void* X, const void* Y, void* Z,
                     void* stream, int expect_case) {
    if (!p) return AFMM_ERR_INVALID_ARG;
    if (p->d.kase != expect_case) return AFMM_ERR_INVALID_ARG;
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    if (n > 0 && (!X || !Y || !Z)) return AFMM_ERR_INVALID_ARG;
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AFMM_TRY(ensure_workspace(p, st));
    const size_t bx = span_bytes(n, d.ldx ? d.ldx : n, d.x_dtype);
    const size_t by = span_bytes(n, d.ldy ? d.ldy : n, d.y_dtype);
    const size_t bz = span_bytes(n, d.ldz ? d.ldz : n, d.z_dtype);
    const bool hx = is_host_ptr(X), hy = is_host_ptr(Y), hz = is_host_ptr(Z);
    if (hx && hy && hz && n >= 1024 && !(d.flags & (AFMM_FLAG_VALIDATE | AFMM_FLAG_FUSED_SPLIT)) &&
        (p->variant == AFMM_VARIANT_TC_BF16X3 || p->variant == AFMM_VARIANT_TC_BF16X2 ||
         p->variant == AFMM_VARIANT_TC_FP8X4)) {
        const int64_t l0 = launch_counter();
        afmm_status rc = run_pipelined_host(p, X, Y, Z, st);
        p->launches += launch_counter() - l0;
        p->calls += 1;
        return rc;
    }
    const void* dX = X;
    const void* dY = Y;
    void* dZ = Z;
    if (hx) {
        void* b;
        AFMM_TRY(stage_buffer(p, 0, bx, &b));
        AFMM_CUDA_TRY(cudaMemcpyAsync(b, X, bx, cudaMemcpyHostToDevice, st));
        dX = b;
    }
    if (hy) {
        void* b;
        AFMM_TRY(stage_buffer(p, 1, by, &b));
        AFMM_CUDA_TRY(cudaMemcpyAsync(b, Y, by, cudaMemcpyHostToDevice, st));
        dY = b;
    }
    if (hz) {
        void* b;
        AFMM_TRY(stage_buffer(p, 2, bz, &b));
        dZ = b;
    }
    if (!hx && !hy && !hz && !p->timing && !p->g_off && n <= kGraphMaxN) {
        bool replay = false;
        AFMM_TRY(graph_call(p, X, Y, Z, st, &replay));
        if (replay) return AFMM_OK;
    }
    MainTimer tm;
    if (p->timing) {
        if (!p->spare.empty()) {
            tm = p->spare.back();
            p->spare.pop_back();
        } else {
            AFMM_CUDA_TRY(cudaEventCreate(&tm.start));
            AFMM_CUDA_TRY(cudaEventCreate(&tm.stop));
        }
        tm.ctas = -1;
        tm.started = false;
        set_main_timer(&tm);
    }
    const int64_t l0 = launch_counter();
    afmm_status rc = run_variant(p, dX, dY, dZ, st);
    set_main_timer(nullptr);
    p->launches += launch_counter() - l0;
    p->calls += 1;
    if (p->timing) {
        if (tm.ctas >= 0) {
            p->last_ctas = tm.ctas;
            p->pending.push_back(tm);
        } else {
            p->spare.push_back(tm);
        }
    }
    AFMM_TRY(rc);
    if (hz) AFMM_CUDA_TRY(cudaMemcpyAsync(Z, dZ, bz, cudaMemcpyDeviceToHost, st));
    if (hx || hy || hz) AFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return AFMM_OK;
}

}  // namespace

extern "C" {

const char* afmm_status_string(afmm_status s) {
    switch (s) {
        case AFMM_OK: return "AFMM_OK";
        case AFMM_ERR_INVALID_ARG: return "AFMM_ERR_INVALID_ARG";
        case AFMM_ERR_UNSUPPORTED: return "AFMM_ERR_UNSUPPORTED";
        case AFMM_ERR_NEGATIVE_REP: return "AFMM_ERR_NEGATIVE_REP";
        case AFMM_ERR_OVERFLOW_RISK: return "AFMM_ERR_OVERFLOW_RISK";
        case AFMM_ERR_OOM: return "AFMM_ERR_OOM";
        case AFMM_ERR_CUDA: return "AFMM_ERR_CUDA";
        case AFMM_ERR_TIMEOUT: return "AFMM_ERR_TIMEOUT";
        case AFMM_ERR_NO_DEVICE: return "AFMM_ERR_NO_DEVICE";
        case AFMM_ERR_NONINTEGER_REP: return "AFMM_ERR_NONINTEGER_REP";
        default: return "AFMM_ERR_UNKNOWN";
    }
}

const char* afmm_last_error_detail(void) { return afmm::g_last_err; }

int afmm_version(void) { return 100; }

afmm_status afmm_plan_create(afmm_plan* out, const afmm_desc* desc) {
    if (!out) return AFMM_ERR_INVALID_ARG;
    *out = nullptr;
    AFMM_TRY(check_desc(desc));
    afmm_plan_s* p = new (std::nothrow) afmm_plan_s();
    if (!p) return AFMM_ERR_OOM;
    p->d = *desc;
    if (!p->d.ldx) p->d.ldx = desc->n;
    if (!p->d.ldy) p->d.ldy = desc->n;
    if (!p->d.ldz) p->d.ldz = desc->n;
    int v = desc->variant;
    if (v == AFMM_VARIANT_AUTO) v = auto_variant(desc);
    if (!variant_serves(v, desc)) {
        delete p;
        return AFMM_ERR_UNSUPPORTED;
    }
    p->variant = v;
    if (v == AFMM_VARIANT_SIMT_F64SLICE) {
        p->slices = kF64Slices;
        p->bits = kF64Bits;
        // int32 sums of n products of 7-bit digits and int8 Rep-factors.
        if ((double)desc->n * 127.0 * 128.0 >= 2147483647.0) {
            delete p;
            return AFMM_ERR_OVERFLOW_RISK;
        }
    } else if (v == AFMM_VARIANT_SIMT_EXACT) {
        if ((double)desc->n * 128.0 * 128.0 >= 2147483647.0) {
            delete p;
            return AFMM_ERR_OVERFLOW_RISK;
        }
    } else if (v == AFMM_VARIANT_TC_EXACT) {
        // int32 sums of n products of operands exact in BF16 (|v| <= 256,
        // or the magnitude hints when given).
        const double rb = desc->rep_max >= 0.0 ? desc->rep_max : 256.0;
        const double bb = desc->base_max >= 0.0 ? desc->base_max : 256.0;
        if ((double)desc->n * rb * bb >= 2147483647.0 ||
            tc_exact_chunk_k(rb, bb) < 32) {
            delete p;
            return AFMM_ERR_OVERFLOW_RISK;
        }
    } else if (v == AFMM_VARIANT_TC_BF16X3) {
        p->slices = 3;
    } else if (v == AFMM_VARIANT_TC_BF16X2) {
        p->slices = 2;
    } else if (v == AFMM_VARIANT_TC_FP8X4) {
        p->slices = 4;
    } else if (v == AFMM_VARIANT_TC_F16X2) {
        p->slices = 2;
    } else if (v == AFMM_VARIANT_TC_EXACT_F8) {
        // Digit and Rep-factor magnitudes at most 16: FP32 sums of n products
        // stay exact integers below 2^24.
        if ((double)desc->n * 16.0 * 16.0 >= 16777216.0) {
            delete p;
            return AFMM_ERR_OVERFLOW_RISK;
        }
        p->slices = 2;
    } else if (v == AFMM_VARIANT_TC_BF16X3X3) {
        p->slices = 3;
    }
    plan_layout(p);
    *out = p;
    return AFMM_OK;
}

afmm_status afmm_plan_destroy(afmm_plan p) {
    if (!p) return AFMM_OK;
    graph_drop(p);
    if (p->g_cap) {
        cudaStreamSynchronize(p->g_cap);
        cudaStreamDestroy(p->g_cap);
    }
    if (p->s_in) {
        cudaStreamSynchronize(p->s_in);
        cudaStreamSynchronize(p->s_out);
        for (auto& e : p->ev)
            if (e) cudaEventDestroy(e);
        cudaStreamDestroy(p->s_in);
        cudaStreamDestroy(p->s_out);
    }
    for (auto* v : {&p->pending, &p->spare})
        for (auto& t : *v) {
            cudaEventDestroy(t.start);
            cudaEventDestroy(t.stop);
        }
    if (p->ws_owned && p->ws) cudaFree(p->ws);
    for (int i = 0; i < 3; ++i)
        if (p->stage[i]) cudaFree(p->stage[i]);
    delete p;
    return AFMM_OK;
}

afmm_status afmm_plan_workspace_size(afmm_plan p, size_t* bytes) {
    if (!p || !bytes) return AFMM_ERR_INVALID_ARG;
    *bytes = p->ws_bytes;
    return AFMM_OK;
}

afmm_status afmm_plan_set_workspace(afmm_plan p, void* ws, size_t bytes) {
    if (!p) return AFMM_ERR_INVALID_ARG;
    if (bytes < p->ws_bytes || (p->ws_bytes && !ws) ||
        (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
        return AFMM_ERR_INVALID_ARG;
    if (p->ws_owned && p->ws) cudaFree(p->ws);
    p->ws = static_cast<char*>(ws);
    p->ws_owned = false;
    p->ws_ready = false;
    return AFMM_OK;
}

afmm_status afmm_mul_caseA(afmm_plan p, const void* X, const void* Y, void* Z,
                           void* stream) {
    return mul_impl(p, X, Y, Z, stream, AFMM_CASE_A);
}

afmm_status afmm_mul_real(afmm_plan p, const void* X, const void* Y, void* Z,
                          void* stream) {
    return mul_impl(p, X, Y, Z, stream, AFMM_CASE_REAL);
}

afmm_status afmm_mul_caseB(afmm_plan p, const void* X, const void* Y, void* Z,
                           void* stream) {
    return mul_impl(p, X, Y, Z, stream, AFMM_CASE_B);
}

afmm_status afmm_mul_rows(afmm_plan p, int64_t r0, int64_t r1, const void* Xrows,
                          const void* Y, void* Zrows, void* stream) {
    if (!p) return AFMM_ERR_INVALID_ARG;
    const afmm_desc& d = p->d;
    const int64_t n = d.n;
    if (d.kase != AFMM_CASE_A && d.kase != AFMM_CASE_B) return AFMM_ERR_INVALID_ARG;
    if (r0 < 0 || r1 < r0 || r1 > n) return AFMM_ERR_INVALID_ARG;
    if (r1 == r0) return AFMM_OK;
    if (!Xrows || !Y || !Zrows) return AFMM_ERR_INVALID_ARG;
    if (p->variant != AFMM_VARIANT_TC_BF16X3 && p->variant != AFMM_VARIANT_TC_BF16X2 &&
        p->variant != AFMM_VARIANT_TC_FP8X4)
        return AFMM_ERR_UNSUPPORTED;
    for (const void* q : {Xrows, Y, static_cast<const void*>(Zrows)})
        if (is_host_ptr(q)) return AFMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AFMM_TRY(ensure_workspace(p, st));
    const int64_t ldx = d.ldx ? d.ldx : n, ldz = d.ldz ? d.ldz : n;
    // The kernels address row r of X and of Z (r in [r0, r1)) from the
    // start of the matrix; the caller holds rows [r0, r1) only, so the
    // base handed down is r0 rows before its pointers (never dereferenced).
    const uintptr_t xb = reinterpret_cast<uintptr_t>(Xrows) -
                         (uintptr_t)(r0 * ldx * (int64_t)dtype_size(d.x_dtype));
    const uintptr_t zb = reinterpret_cast<uintptr_t>(Zrows) -
                         (uintptr_t)(r0 * ldz * (int64_t)dtype_size(d.z_dtype));
    int* status = wsp<int>(p, p->off_status);
    const int64_t l0 = launch_counter();
    afmm_status rc = tc_split_prepare_b(&p->tc, d, Y, status, st);
    if (rc == AFMM_OK)
        rc = tc_split_rows(&p->tc, d, reinterpret_cast<const void*>(xb),
                           reinterpret_cast<void*>(zb), r0, r1, status, st);
    p->launches += launch_counter() - l0;
    p->calls += 1;
    return rc;
}

afmm_status afmm_plan_sync(afmm_plan p, void* stream) {
    if (!p) return AFMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AFMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!p->ws) return AFMM_OK;
    int code = 0;
    AFMM_CUDA_TRY(cudaMemcpy(&code, p->ws + p->off_status, sizeof(int),
                             cudaMemcpyDeviceToHost));
    if (code != 0) {
        const int zero = 0;
        AFMM_CUDA_TRY(cudaMemcpy(p->ws + p->off_status, &zero, sizeof(int),
                                 cudaMemcpyHostToDevice));
        if (p->variant == AFMM_VARIANT_SPARSE) {
            AFMM_TRY(sparse_reset(p->ws + p->off_a, st));
            AFMM_CUDA_TRY(cudaStreamSynchronize(st));
        }
        return static_cast<afmm_status>(code);
    }
    return AFMM_OK;
}

afmm_status afmm_get_info(afmm_plan p, afmm_info* out) {
    if (!p || !out) return AFMM_ERR_INVALID_ARG;
    afmm_info& o = *out;
    o.variant = p->variant;
    o.slices = p->slices;
    o.slice_bits = p->bits;
    o.k_split = p->ksplit;
    o.workspace_bytes = p->ws_bytes;
    o.d1 = o.d2 = o.mu_prime = o.mu = o.rep_max = o.expected_additions = -1.0;
    if (p->validated && p->ws) {
        AFMM_CUDA_TRY(cudaDeviceSynchronize());
        ScanStats sx, sy;
        AFMM_CUDA_TRY(cudaMemcpy(&sx, p->ws + p->off_sx, sizeof sx,
                                 cudaMemcpyDeviceToHost));
        AFMM_CUDA_TRY(cudaMemcpy(&sy, p->ws + p->off_sy, sizeof sy,
                                 cudaMemcpyDeviceToHost));
        const double n = (double)p->d.n, n2 = n * n;
        const ScanStats& rep = p->d.kase == AFMM_CASE_A ? sy : sx;
        o.d1 = n2 > 0 ? (double)sx.nnz / n2 : 0.0;
        o.d2 = n2 > 0 ? (double)sy.nnz / n2 : 0.0;
        if (p->d.kase != AFMM_CASE_REAL) {       // no Rep-factor otherwise
            o.mu_prime = rep.nnz ? rep.sum / (double)rep.nnz : 0.0;
            o.mu = n2 > 0 ? rep.sum / n2 : 0.0;
            o.rep_max = rep.maxv;
            o.expected_additions = o.mu_prime * o.d1 * o.d2 * n * n2;
        }
    }
    return AFMM_OK;
}

afmm_status afmm_plan_enable_kernel_timing(afmm_plan p, int enable) {
    if (!p) return AFMM_ERR_INVALID_ARG;
    p->timing = enable != 0;
    p->timed = 0;
    p->timed_ms = 0.0;
    for (auto& t : p->pending) p->spare.push_back(t);
    p->pending.clear();
    return AFMM_OK;
}

afmm_status afmm_plan_counters(afmm_plan p, afmm_counters* out) {
    if (!p || !out) return AFMM_ERR_INVALID_ARG;
    for (auto& t : p->pending) {
        AFMM_CUDA_TRY(cudaEventSynchronize(t.stop));
        float ms = 0.f;
        AFMM_CUDA_TRY(cudaEventElapsedTime(&ms, t.start, t.stop));
        p->timed_ms += ms;
        p->timed += 1;
        p->spare.push_back(t);
    }
    p->pending.clear();
    out->calls = p->calls;
    out->kernel_launches = p->launches;
    out->timed_launches = p->timed;
    out->timed_ms = p->timed_ms;
    out->main_kernel_ctas = p->last_ctas;
    out->reserved_ = 0;
    out->simt_k_tiles = -1;
    if (p->variant == AFMM_VARIANT_SIMT_F32 && !simt_dense(p->d) && p->ws_ready) {
        unsigned long long v = 0;
        AFMM_CUDA_TRY(cudaMemcpy(&v, simt_ktiles(p), sizeof(v), cudaMemcpyDeviceToHost));
        out->simt_k_tiles = (int64_t)v;
    }
    return AFMM_OK;
}

int64_t afmm_mlp_param_count(const afmm_mlp_shape* s) {
    if (!s || s->features <= 0 || s->hidden <= 0 || s->outputs <= 0) return -1;
    return mlp_param_count(*s);
}

int64_t afmm_mlp_work_floats(const afmm_mlp_shape* s, int rows) {
    if (!s || rows < 0 || s->features <= 0 || s->hidden <= 0 || s->outputs <= 0) return -1;
    return mlp_work_floats(*s, rows);
}

afmm_status afmm_mlp_forward(const afmm_mlp_shape* s, const float* params, const float* X,
                             int rows, float* P, float* work, void* stream) {
    if (afmm_mlp_param_count(s) < 0 || rows < 0 || (rows > 0 && (!params || !X || !P || !work)))
        return AFMM_ERR_INVALID_ARG;
    if (rows == 0) return AFMM_OK;
    return mlp_forward(*s, params, X, rows, P, work, static_cast<cudaStream_t>(stream));
}

afmm_status afmm_mlp_loss_grad(const afmm_mlp_shape* s, const float* params, const float* X,
                               const float* T, const float* M, int rows, float count,
                               float* grads, float* work, float* loss, void* stream) {
    if (afmm_mlp_param_count(s) < 0 || rows <= 0 || !params || !X || !T || !M || !grads ||
        !work || !loss)
        return AFMM_ERR_INVALID_ARG;
    return mlp_loss_grad(*s, params, X, T, M, rows, count, grads, work, loss,
                         static_cast<cudaStream_t>(stream));
}

afmm_status afmm_mlp_adam(int64_t n, float* params, const float* grads, float* m, float* v,
                          float lr, float beta1, float beta2, float eps, int step,
                          void* stream) {
    if (n < 0 || step < 1 || (n > 0 && (!params || !grads || !m || !v)))
        return AFMM_ERR_INVALID_ARG;
    if (n == 0) return AFMM_OK;
    return mlp_adam(n, params, grads, m, v, lr, beta1, beta2, eps, step,
                    static_cast<cudaStream_t>(stream));
}

afmm_status afmm_dispatch_features(const afmm_desc* d, float* out) {
    if (!d || !out) return AFMM_ERR_INVALID_ARG;
    return dispatch_features(*d, out);
}

afmm_status afmm_set_dispatch_model(const afmm_mlp_shape* s, const float* params,
                                    const float* mean, const float* scale,
                                    const int32_t* variants) {
    afmm_status rc = set_dispatch_model(s, params, mean, scale, variants);
    if (rc == AFMM_OK) batched_clear_cache();   // cached routes may change
    return rc;
}

int32_t afmm_dispatch_variant(const afmm_desc* d) {
    if (!d) return -1;
    const int r = dispatch_route(*d);
    return r == 2 ? AFMM_VARIANT_TC_BF16X3_N128
                  : r == 1 ? AFMM_VARIANT_TC_BF16X3 : AFMM_VARIANT_SIMT_F32;
}

afmm_status afmm_batched_sync(int count, const afmm_desc* descs, void* stream) {
    if (count < 0 || (count > 0 && !descs)) return AFMM_ERR_INVALID_ARG;
    AFMM_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int code = 0;
    AFMM_TRY(batched_status(count, descs, &code));
    return static_cast<afmm_status>(code);
}

afmm_status afmm_selftest_bounded_wait(uint64_t limit_ns, void* stream) {
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    return tc_selftest_bounded_wait(limit_ns, static_cast<cudaStream_t>(stream));
}

afmm_status afmm_mul_batched(int count, const afmm_desc* descs,
                             const void* const* X, const void* const* Y,
                             void* const* Z, void* stream) {
    if (count < 0 || (count > 0 && (!descs || !X || !Y || !Z)))
        return AFMM_ERR_INVALID_ARG;
    return batched_run(count, descs, X, Y, Z, stream, nullptr);
}

size_t afmm_error_norm_workspace_size(int64_t rows, int64_t cols) {
    return error_norm_ws_bytes(rows, cols);
}

afmm_status afmm_error_norm(const void* Z, int32_t z_dtype, int64_t ldz,
                            const void* R, int32_t r_dtype, int64_t ldr,
                            int64_t rows, int64_t cols, void* workspace,
                            double out[3], void* stream) {
    if (!out || rows < 0 || cols < 0 || ldz < cols || ldr < cols)
        return AFMM_ERR_INVALID_ARG;
    if (rows > 0 && cols > 0 && (!Z || !R)) return AFMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t wsb = error_norm_ws_bytes(rows, cols);
    void* ws = workspace;
    bool owned = false;
    if (!ws) {
        AFMM_CUDA_TRY(cudaMalloc(&ws, wsb));
        owned = true;
    }
    double* out_dev = reinterpret_cast<double*>(static_cast<char*>(ws) + wsb - 256);
    afmm_status rc = launch_error_norm(Z, z_dtype, ldz, R, r_dtype, ldr, rows,
                                       cols, ws, out_dev, st);
    if (rc == AFMM_OK) {
        cudaError_t e = cudaMemcpyAsync(out, out_dev, 3 * sizeof(double),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_last_cuda_error(e, "error norm readback", __FILE__, __LINE__);
            rc = AFMM_ERR_CUDA;
        }
    }
    if (owned) cudaFree(ws);
    return rc;
}

}  // extern "C"


