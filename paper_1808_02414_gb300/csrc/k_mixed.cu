// Mixed-precision step (d): placeholder until the tensor-core path lands.
#include "ccov_internal.cuh"

namespace ccov {
cudaError_t mixed_alloc(Ctx&) { return cudaErrorNotSupported; }
void mixed_free(Ctx&) {}
cudaError_t mixed_factor_inverse(Ctx&) { return cudaErrorNotSupported; }
}  // namespace ccov
