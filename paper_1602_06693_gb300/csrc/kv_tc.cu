// Tensor-core K.V (placeholder until the tcgen05 kernel lands).
#include "ctx.cuh"

namespace kpcg {
bool kv_tc_supported(int) { return false; }
void kv_tc_apply(Ctx&, const float*, int64_t, int, float*, int64_t, float) {
    fail(KPCG_ERR_ARG, "tensor-core K.V is not available in this build");
}
}  // namespace kpcg
