// afmm_mul_noalloc: the FP64-target product for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while another
// allocator has reserved all of the device's memory, real-time loops that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree,
// or hosts whose policy forbids allocating from inside their callbacks.
// The plan API sizes a workspace and allocates it (or borrows one from the
// caller); this entry point instead keeps its scratch in one file-scope
// device array of fixed size, so it allocates nothing at any call.
//
// The array holds the scratch of the FP64-target form for n <= 256: row
// exponents, eight 7-bit digit slices of the real factor, the packed
// Rep-factors, the exact int32 digit products and, for Case B, transposes.
// A device holds the array from the first call on it (CUDA loads this
// library's device code lazily unless CUDA_MODULE_LOADING=EAGER) until the
// process exits.  All calls share it: calls that overlap on the GPU
// (several streams or threads at once) race on it and must not be issued.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "afmm_common.cuh"

namespace afmm {
namespace {

constexpr int64_t kNoAllocMaxN = 256;
constexpr int kNoAllocBits = 7;
constexpr int kNoAllocSlices = 8;

// Byte offsets inside the scratch array (each 256-byte aligned).
constexpr size_t kOffStatus = 0;
constexpr size_t kOffE = 256;
constexpr size_t kOffQ = kOffE + kNoAllocMaxN * 4;                                  // int8 digits
constexpr size_t kOffW = kOffQ + (size_t)kNoAllocSlices * kNoAllocMaxN * kNoAllocMaxN;  // packed Y
constexpr size_t kOffP = kOffW + (size_t)(kNoAllocMaxN / 4) * kNoAllocMaxN * 4;     // int32 products
constexpr size_t kOffT1 = kOffP + (size_t)kNoAllocSlices * kNoAllocMaxN * kNoAllocMaxN * 4;
constexpr size_t kOffT2 = kOffT1 + (size_t)kNoAllocMaxN * kNoAllocMaxN * 8;
constexpr size_t kOffT3 = kOffT2 + (size_t)kNoAllocMaxN * kNoAllocMaxN * 8;
constexpr size_t kNoAllocScratchBytes = kOffT3 + (size_t)kNoAllocMaxN * kNoAllocMaxN * 8;
static_assert(kOffQ % 256 == 0 && kOffW % 256 == 0 && kOffP % 256 == 0 &&
                  kOffT1 % 256 == 0 && kOffT2 % 256 == 0 && kOffT3 % 256 == 0,
              "scratch alignment");

// The scratch.  In host code this name is only a stand-in for the device
// object; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device, looked up on
// every call with that device current: after a cudaDeviceReset the module
// is loaded again and the array may sit elsewhere, so no address is kept
// between calls.  Once the module is loaded on the device the lookup
// allocates nothing; the first lookup (or launch) on a device loads it
// under CUDA's default lazy module loading, which is when the array and
// the code take their device memory.
afmm_status scratch_for_current_device(char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return AFMM_ERR_NO_DEVICE;
    }
    void* p = nullptr;
    AFMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<char*>(p);
    return AFMM_OK;
}

// Z = NaN everywhere when a conversion recorded an error (a negative or
// non-integer Rep-factor, or one outside the int8 range of the digit
// products), so a bad result cannot be mistaken for a good one.
__global__ void poison_if_flagged(double* Z, int64_t n, int64_t ldz,
                                  const int* status) {
    if (*status == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * n;
         i += (int64_t)gridDim.x * blockDim.x)
        Z[(i / n) * ldz + (i % n)] = __longlong_as_double(0x7ff8000000000000LL);
}

// Case-A form into Z (F64): X real, Y Rep-factors, scratch at `s`.
afmm_status run_case_a(char* s, int64_t n, const void* X, int xdt, int64_t ldx,
                       const void* Y, int ydt, int64_t ldy, double* Z,
                       int64_t ldz, cudaStream_t st) {
    const int64_t ld = (n + 3) / 4 * 4;
    int* status = reinterpret_cast<int*>(s + kOffStatus);
    int32_t* E = reinterpret_cast<int32_t*>(s + kOffE);
    int8_t* Q = reinterpret_cast<int8_t*>(s + kOffQ);
    int32_t* W = reinterpret_cast<int32_t*>(s + kOffW);
    int32_t* P = reinterpret_cast<int32_t*>(s + kOffP);
    AFMM_TRY(launch_exp_slice_rows_i8(X, xdt, n, ldx, E, kNoAllocSlices, kNoAllocBits, Q,
                                  ld, st));
    AFMM_TRY(launch_pack_b_i8(Y, ydt, n, ldy, W, ld, status, st, true));
    AFMM_TRY(launch_simt_dp4a(Q, ld, W, ld, P, n, (int64_t)kNoAllocSlices * n, n, n,
                              st));
    return launch_recombine_f64(P, n, E, kNoAllocSlices, kNoAllocBits, n, Z, ldz, st);
}

}  // namespace
}  // namespace afmm

using namespace afmm;

extern "C" afmm_status afmm_mul_noalloc(const afmm_desc* d, const void* X,
                                        const void* Y, void* Z, void* stream) {
    if (!d) return AFMM_ERR_INVALID_ARG;
    const int64_t n = d->n;
    if (n < 0 || d->target != AFMM_TARGET_FP64 || d->z_dtype != AFMM_F64 ||
        (d->kase != AFMM_CASE_A && d->kase != AFMM_CASE_B) || d->reserved_ != 0)
        return AFMM_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) {
        static const char msg[] =
            "afmm_mul_noalloc: n exceeds the fixed scratch limit of 256";
        set_last_error_text(msg);
        return AFMM_ERR_UNSUPPORTED;
    }
    const int64_t ldx = d->ldx ? d->ldx : n, ldy = d->ldy ? d->ldy : n,
                  ldz = d->ldz ? d->ldz : n;
    if (ldx < n || ldy < n || ldz < n) return AFMM_ERR_INVALID_ARG;
    const int rep_dt = d->kase == AFMM_CASE_A ? d->y_dtype : d->x_dtype;
    const int real_dt = d->kase == AFMM_CASE_A ? d->x_dtype : d->y_dtype;
    if (dtype_size(rep_dt) == 0 || dtype_size(real_dt) == 0 ||
        real_dt == AFMM_E4M3 || rep_dt == AFMM_F64)
        return AFMM_ERR_INVALID_ARG;
    if (n == 0) return AFMM_OK;
    if (!X || !Y || !Z) return AFMM_ERR_INVALID_ARG;
    // Device pointers of the current device only: host buffers would need
    // staging memory, and another device's memory may not be reachable.
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return AFMM_ERR_NO_DEVICE;
    }
    for (const void* p : {X, Y, static_cast<const void*>(Z)}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return AFMM_ERR_INVALID_ARG;
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return AFMM_ERR_INVALID_ARG;
        if (a.type == cudaMemoryTypeDevice && a.device != cur) return AFMM_ERR_INVALID_ARG;
    }
    char* s = nullptr;
    AFMM_TRY(scratch_for_current_device(&s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = reinterpret_cast<int*>(s + kOffStatus);
    // The array keeps the previous call's contents: the status word must
    // start at zero; every other buffer is fully rewritten below.
    AFMM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    double* Zd = static_cast<double*>(Z);
    if (d->kase == AFMM_CASE_A) {
        AFMM_TRY(run_case_a(s, n, X, d->x_dtype, ldx, Y, d->y_dtype, ldy, Zd, ldz, st));
    } else {
        // Case B: Z^T = Y^T X^T is a Case-A product of the transposes.
        void* YT = s + kOffT1;
        void* XT = s + kOffT2;
        double* ZT = reinterpret_cast<double*>(s + kOffT3);
        AFMM_TRY(launch_transpose(Y, dtype_size(d->y_dtype), n, n, ldy, YT, n, st));
        AFMM_TRY(launch_transpose(X, dtype_size(d->x_dtype), n, n, ldx, XT, n, st));
        AFMM_TRY(run_case_a(s, n, YT, d->y_dtype, n, XT, d->x_dtype, n, ZT, n, st));
        AFMM_TRY(launch_transpose(ZT, 8, n, n, n, Zd, ldz, st));
    }
    poison_if_flagged<<<64, 256, 0, st>>>(Zd, n, ldz, status);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}
