// Standard (dense) representation on the k-point kernels (dense.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace dense {
// out[g] = (L_g + L_g^dag)/2 for g < G and, unless hermitian, out[G + g] = i (L_g - L_g^dag)/2.
cudaError_t hermitian_vectors(const zc* L, zc* out, int G, int M, int hermitian, cudaStream_t st);
}  // namespace dense
