// Tensor-core ("mixed") path: not yet built in this revision; create reports
// AFQMC_ERR_UNSUPPORTED so callers fall back to nothing silently.
#include "mixed.hpp"

namespace mixed {
afqmc_status create(afqmc_kp*, cudaStream_t) { return AFQMC_ERR_UNSUPPORTED; }
void destroy(afqmc_kp*) {}
cudaError_t set_one_body(afqmc_kp*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t force_bias(afqmc_kp*, const zc*, zc*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t propagate(afqmc_kp*, zc*, const double*, double*, zc*, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t orthonormalise(afqmc_kp*, zc*, zc*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t local_energy(afqmc_kp*, const zc*, zc*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t local_energy_backward(afqmc_kp*, const zc*, const zc*, zc*, zc*, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace mixed
