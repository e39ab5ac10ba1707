// Tensor-core ("mixed") path of the k-point AFQMC walker step.
#pragma once

#include "handle.hpp"

namespace mixed {
afqmc_status create(afqmc_kp* h, cudaStream_t st);
void destroy(afqmc_kp* h);
cudaError_t set_one_body(afqmc_kp* h, cudaStream_t st);
cudaError_t force_bias(afqmc_kp* h, const zc* phi, zc* xbar, cudaStream_t st);
cudaError_t propagate(afqmc_kp* h, zc* phi, const double* x, double* w, zc* logdet, int do_qr, cudaStream_t st);
cudaError_t orthonormalise(afqmc_kp* h, zc* phi, zc* logdet, cudaStream_t st);
cudaError_t local_energy(afqmc_kp* h, const zc* phi, zc* eloc, cudaStream_t st);
cudaError_t step(afqmc_kp* h, zc* phi, const double* x, double* w, zc* eloc, zc* logdet, int do_qr, int reuse,
                 cudaStream_t st);
cudaError_t local_energy_backward(afqmc_kp* h, const zc* phi, const zc* grad_e, zc* grad_phi, zc* grad_h1,
                                  cudaStream_t st);
// ring depth of every GEMM and the per-launch ms timed for two and three stages at create
void gemm_tuning(const afqmc_kp* h, int* depth, double* ms2, double* ms3);
}  // namespace mixed
