// Placeholder until the transform kernels land.
#include "bn_internal.h"

namespace bn {
struct NttPlan {};
bn_status ntt_create(NttPlan **out, bool, uint32_t, uint32_t, const bn_tuning *) {
    *out = nullptr;
    return BN_EUNSUPPORTED;
}
void ntt_destroy(NttPlan *) {}
cudaError_t ntt_launch(NttPlan *, const uint32_t *, const uint32_t *, uint32_t *, uint64_t,
                       cudaStream_t) {
    return cudaErrorNotSupported;
}
size_t ntt_scratch_bytes(const NttPlan *) { return 0; }
uint32_t ntt_length(const NttPlan *) { return 0; }
}  // namespace bn
