// Internal state of one afqmc_kp handle (not part of the ABI).
#pragma once

#include <vector>

#include "afqmc_kp.h"
#include "common.cuh"

struct MixedState;  // tensor-core path buffers (mixed.cu)

struct afqmc_kp {
  afqmc_kp_desc d;
  int nk, M, n, G, W, NM, N, order;
  double dt, sqdt;
  std::vector<int> h_kminus, h_minus;  // host copies of the momentum tables
  int* kminus = nullptr;               // device [Nk][Nk]: index of k - Q
  int* minus = nullptr;                // device [Nk]: index of -Q

  // static data, complex128
  zc* L = nullptr;      // [Q][k][g][p][r]
  zc* LH = nullptr;     // [Q][k][g][a][r]  half-rotated
  zc* A = nullptr;      // [k][p][a]        trial
  zc* h1 = nullptr;     // [k][p][q]
  zc* AhH = nullptr;    // [k][a][q]        A[k]^dagger h[k]
  zc* v0 = nullptr;     // [k][p][q]        mean-field term
  zc* Ehalf = nullptr;  // [k][p][q]        exp(-dt/2 (h + v0))
  zc* expm_tmp = nullptr;  // [k][3][M][M]

  // workspace
  zc* S = nullptr;      // [W][2][N][N]    overlap, then LU factors
  zc* Sinv = nullptr;   // [W][2][N][N]
  zc* Gh = nullptr;     // [W][2][N][NM]   half-rotated Green's function
  zc* X = nullptr;      // [W][Nk][G]
  zc* xbar = nullptr;   // [W][2][Nk][G]
  zc* y = nullptr;      // [W][Nk][G]      sqrt(dt) * vHS coefficients
  zc* V = nullptr;      // [W][NM][NM]
  zc* T0 = nullptr;     // [W][2][NM][N]
  zc* T1 = nullptr;     // [W][2][NM][N]
  zc* acc = nullptr;    // [W][2][NM][N]
  zc* ld_old = nullptr; // [W][2]
  zc* ld_new = nullptr; // [W][2]
  int* sing_old = nullptr;  // [W][2]
  int* sing_new = nullptr;  // [W][2]
  zc* epart = nullptr;  // [W][2][Nk][Nk] exchange partials
  zc* Gam = nullptr;    // [W][2][N][NM]   dE/dGh
  zc* P = nullptr;      // [W][2][N][N]
  int* flags = nullptr; // [0] singular walkers, [1] timeouts

  MixedState* mixed = nullptr;

  // Green's function state left by afqmc_kp_step (valid for green_phi until any
  // other entry point reuses the buffers)
  bool green_valid = false;
  const void* green_phi = nullptr;

  // stage timing (afqmc_kp_profile)
  bool prof_on = false;
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;
  int open_stage = -1;
  cudaEvent_t open_event = nullptr;

  int launches = 0;     // kernel launches of the current call
  size_t bytes = 0;
  std::vector<void*> allocs;
};

// Launch bookkeeping: every kernel launch goes through AFQMC_LAUNCHED(h).
#define AFQMC_LAUNCHED(h) ((h)->launches++)

// Stage timing: no-ops unless afqmc_kp_profile enabled recording.
inline cudaEvent_t prof_event(afqmc_kp* h) {
  cudaEvent_t e = nullptr;
  if (!h->event_pool.empty()) {
    e = h->event_pool.back();
    h->event_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  return e;
}
inline void prof_begin(afqmc_kp* h, int stage, cudaStream_t st) {
  if (!h->prof_on) return;
  cudaEvent_t e = prof_event(h);
  if (!e) return;
  cudaEventRecord(e, st);
  h->open_stage = stage;
  h->open_event = e;
}
inline void prof_end(afqmc_kp* h, cudaStream_t st) {
  if (!h->prof_on || h->open_stage < 0) return;
  cudaEvent_t e = prof_event(h);
  if (!e) return;
  cudaEventRecord(e, st);
  h->recs.push_back({h->open_stage, h->open_event, e});
  h->open_stage = -1;
  h->open_event = nullptr;
}

// FP64 path (fp64.cu)
namespace fp64 {
cudaError_t setup_static(afqmc_kp* h, cudaStream_t st);
cudaError_t set_one_body(afqmc_kp* h, cudaStream_t st);
cudaError_t green(afqmc_kp* h, const zc* phi, cudaStream_t st);        // S, LU, Sinv, logdet, Gh
cudaError_t cholesky_trace(afqmc_kp* h, cudaStream_t st);              // X from Gh
cudaError_t force_bias(afqmc_kp* h, const double* x, zc* xbar_out, cudaStream_t st);
cudaError_t propagate(afqmc_kp* h, zc* phi, const double* x, double* w, zc* logdet, int do_qr,
                      cudaStream_t st);
cudaError_t orthonormalise(afqmc_kp* h, zc* phi, zc* logdet, cudaStream_t st);
cudaError_t local_energy(afqmc_kp* h, const zc* phi, zc* eloc, cudaStream_t st);
cudaError_t local_energy_backward(afqmc_kp* h, const zc* phi, const zc* grad_e, zc* grad_phi,
                                  zc* grad_h1, cudaStream_t st);
// pieces shared with the mixed path
cudaError_t grad_h1(afqmc_kp* h, const zc* grad_e, zc* grad_h1, cudaStream_t st);   // from Gh
// the projection's GEMMs in FP64, or (ff) in double-float on the FP32 pipe
cudaError_t project_gamma(afqmc_kp* h, zc* grad_phi, cudaStream_t st, bool ff);      // Gam, Gh, Sinv
cudaError_t green_ff(afqmc_kp* h, const zc* phi, cudaStream_t st);  // green() with a double-float Gh GEMM
cudaError_t overlap_lu(afqmc_kp* h, const zc* phi, zc* ld, int* sing, int want_inv, cudaStream_t st);
cudaError_t overlap_only(afqmc_kp* h, const zc* phi, cudaStream_t st);
cudaError_t lu_only(afqmc_kp* h, zc* ld, int* sing, int want_inv, cudaStream_t st);
cudaError_t weights(afqmc_kp* h, const zc* phi, const double* x, double* w, zc* logdet, cudaStream_t st);
cudaError_t qr_with(afqmc_kp* h, zc* phi, zc* scratch, cudaStream_t st);
cudaError_t qr_launch(zc* phi, zc* scratch, int rows, int cols, int nmat, cudaStream_t st);
cudaError_t weight_only(afqmc_kp* h, const double* x, double* w, zc* logdet, cudaStream_t st);
cudaError_t step(afqmc_kp* h, zc* phi, const double* x, double* w, zc* eloc, zc* logdet, int do_qr, int reuse,
                 cudaStream_t st);
}  // namespace fp64
