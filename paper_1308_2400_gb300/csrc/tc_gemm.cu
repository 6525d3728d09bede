// Tensor-core path (placeholder until the tcgen05 kernel lands).
#include "afmm_common.cuh"
#include "tc_gemm.cuh"

namespace afmm {
bool tc_available() { return false; }
void tc_layout(TcPlan* t, const afmm_desc& d, int slices) {
    t->n = d.n;
    t->slices = slices;
}
afmm_status tc_bind_workspace(TcPlan* t, void* a, void* b) {
    t->a = a;
    t->b = b;
    return AFMM_OK;
}
afmm_status tc_run_split(TcPlan*, const afmm_desc&, const void*, const void*,
                         void*, int*, cudaStream_t) {
    return AFMM_ERR_UNSUPPORTED;
}
}  // namespace afmm
