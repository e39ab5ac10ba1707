// Device-side auxiliary fields (Philox4x32-10 + Box-Muller) and comb population control.
#pragma once

#include <cuda_runtime.h>

#include "handle.hpp"

namespace rng {
cudaError_t philox(const unsigned* ctr, unsigned long long seed, unsigned* out, size_t n, cudaStream_t st);
cudaError_t fields(afqmc_kp* h, unsigned long long seed, unsigned long long* counter, double* x, cudaStream_t st);
// shared memory of the comb's selection kernel (the cumulative weights)
size_t comb_smem_bytes(int W);
cudaError_t comb(afqmc_kp* h, zc* phi, double* weight, unsigned long long seed, const unsigned long long* counter,
                 int* idx, cudaStream_t st);
}  // namespace rng
