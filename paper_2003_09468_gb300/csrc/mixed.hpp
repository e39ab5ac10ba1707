// Tensor-core ("mixed") path of the k-point AFQMC walker step.
#pragma once

#include <functional>

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
// Several mixed handles (the same Taylor order, at most 8) advanced by one step together: the
// Taylor-term GEMMs (all = false) or every GEMM of the step (all = true) are each one launch
// over the tiles of all of them; the other work runs per handle through `each`, which calls
// its argument for every handle (index, handle, the handle's stream) between a fork from and a
// join into `st`.  phi, x, w, eloc, logdet and reuse are per handle (eloc and logdet entries
// may be NULL).  Each handle computes exactly what afqmc_kp_step computes on it alone.
constexpr int GROUP_MAX = 8;
using MemberFn = std::function<cudaError_t(int, afqmc_kp*, cudaStream_t)>;
using ForEach = std::function<cudaError_t(const MemberFn&)>;
cudaError_t group_step(afqmc_kp* const* hs, int n, zc* const* phi, const double* const* x, double* const* w,
                       zc* const* eloc, zc* const* logdet, int do_qr, const int* reuse, bool all, const ForEach& each,
                       cudaStream_t st);
// ring depth of every GEMM and the per-launch ms timed for two and three stages at create
void gemm_tuning(const afqmc_kp* h, int* depth, double* ms2, double* ms3);
// The Taylor GEMM's CTA-pair form: whether it is used, its ms at create, and whether the
// handle has it at all (more than one 128-row tile per walker).
void gemm_form(const afqmc_kp* h, int gemm, int* pair, double* ms_pair);
bool set_gemm_form(afqmc_kp* h, int gemm, int pair);
}  // namespace mixed
