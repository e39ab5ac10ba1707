// C ABI entry points of the k-point AFQMC library (declared in include/afqmc_kp.h).
// Argument validation, device memory ownership and dispatch to the FP64 or the
// tensor-core (mixed) kernels.  No exception crosses this file's boundary.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "dense.hpp"
#include "handle.hpp"
#include "mixed.hpp"
#include "rng.hpp"

namespace {

thread_local char g_msg[512] = "";

afqmc_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return AFQMC_OK;
  snprintf(g_msg, sizeof(g_msg), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return AFQMC_ERR_OOM;
  if (e == cudaErrorNotSupported) return AFQMC_ERR_UNSUPPORTED;
  return AFQMC_ERR_CUDA;
}

void free_all(afqmc_kp* h) {
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

template <typename T>
cudaError_t alloc(afqmc_kp* h, T** p, size_t count) {
  void* q = nullptr;
  size_t b = count * sizeof(T);
  if (b == 0) b = 16;
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  h->bytes += b;
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

// k - Q and -Q on the Gamma-centred grid, C order over the three axes.
void momentum_tables(const int g[3], std::vector<int>& kminus, std::vector<int>& minus) {
  const int nk = g[0] * g[1] * g[2];
  kminus.assign((size_t)nk * nk, 0);
  minus.assign(nk, 0);
  auto coords = [&](int i, int c[3]) { c[2] = i % g[2]; c[1] = (i / g[2]) % g[1]; c[0] = i / (g[1] * g[2]); };
  auto lin = [&](const int c[3]) { return (c[0] * g[1] + c[1]) * g[2] + c[2]; };
  for (int k = 0; k < nk; ++k)
    for (int Q = 0; Q < nk; ++Q) {
      int ck[3], cq[3], r[3];
      coords(k, ck);
      coords(Q, cq);
      for (int d = 0; d < 3; ++d) r[d] = ((ck[d] - cq[d]) % g[d] + g[d]) % g[d];
      kminus[(size_t)k * nk + Q] = lin(r);
    }
  for (int Q = 0; Q < nk; ++Q) {
    int cq[3], r[3];
    coords(Q, cq);
    for (int d = 0; d < 3; ++d) r[d] = (g[d] - cq[d]) % g[d];
    minus[Q] = lin(r);
  }
}

bool valid_desc(const afqmc_kp_desc* d) {
  if (!d) return false;
  for (int i = 0; i < 3; ++i)
    if (d->kgrid[i] < 1 || d->kgrid[i] > 64) return false;
  const long nk = (long)d->kgrid[0] * d->kgrid[1] * d->kgrid[2];
  if (nk > 4096) return false;
  if (d->M < 1 || d->M > 128) return false;
  if (d->nocc < 1 || d->nocc > d->M) return false;
  if (d->nchol < 1 || d->nchol > 8192) return false;
  if (d->nwalkers < 1 || d->nwalkers > 65535) return false;
  if (!(d->dt > 0.0)) return false;
  if (d->taylor_order < 1 || d->taylor_order > 16) return false;
  if (d->prec != AFQMC_FP64 && d->prec != AFQMC_MIXED) return false;
  if (nk * d->nocc > 1024) return false;  // N per spin
  return true;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define MTRY_API(x)                         \
  do {                                      \
    const cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

// Complex arrays are read and written as 16-byte (re, im) vectors: NULL or 16-byte aligned.
bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool al16(const void* a, const void* b, const void* c = nullptr, const void* d = nullptr) {
  return al16(a) && al16(b) && al16(c) && al16(d);
}

// One fused step (afqmc_kp_step after validation); keeps the stored-Green bookkeeping.
cudaError_t step_impl(afqmc_kp* h, void* phi, const double* x, double* weight, void* eloc, void* logdet, int do_qr,
                      int flags, cudaStream_t st) {
  const int reuse = (flags & AFQMC_STEP_REUSE_GREEN) && h->green_valid && h->green_phi == phi;
  h->green_valid = false;
  cudaError_t e;
  if (h->mixed)
    e = mixed::step(h, static_cast<zc*>(phi), x, weight, static_cast<zc*>(eloc), static_cast<zc*>(logdet), do_qr,
                    reuse, st);
  else
    e = fp64::step(h, static_cast<zc*>(phi), x, weight, static_cast<zc*>(eloc), static_cast<zc*>(logdet), do_qr,
                   reuse, st);
  if (e == cudaSuccess) {
    h->green_valid = true;
    h->green_phi = phi;
  }
  return e;
}

bool block_args_ok(int nsteps, int qr_period, int energy_period, int flags, int comb) {
  return nsteps >= 1 && qr_period >= 1 && energy_period >= 1 && !(flags & ~AFQMC_STEP_REUSE_GREEN) &&
         (comb == 0 || comb == 1);
}

// One block (afqmc_kp_block after validation): fields, step, ..., then the comb.
cudaError_t block_impl(afqmc_kp* h, void* phi, double* weight, double* x, void* eloc_hist, double* weight_hist,
                       void* logdet, int nsteps, int qr_period, int energy_period, int flags, int comb,
                       unsigned long long seed, unsigned long long* counter, int* idx, cudaStream_t st) {
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = rng::fields(h, seed, counter, x, st);
    if (e != cudaSuccess) return e;
    const int do_qr = ((s + 1) % qr_period == 0) || s == nsteps - 1;
    const int measure = ((s + 1) % energy_period == 0) || s == nsteps - 1;
    void* el = measure ? static_cast<void*>(static_cast<zc*>(eloc_hist) + (size_t)(s / energy_period) * h->W * 3)
                       : nullptr;
    void* ld = s == nsteps - 1 ? logdet : nullptr;
    e = step_impl(h, phi, x, weight, el, ld, do_qr, s == 0 ? flags : AFQMC_STEP_REUSE_GREEN, st);
    if (e != cudaSuccess) return e;
    if (weight_hist) {
      e = cudaMemcpyAsync(weight_hist + (size_t)s * h->W, weight, sizeof(double) * h->W, cudaMemcpyDeviceToDevice,
                          st);
      if (e != cudaSuccess) return e;
    }
  }
  if (comb) {
    h->green_valid = false;
    return rng::comb(h, static_cast<zc*>(phi), weight, seed, counter, idx, st);
  }
  return cudaSuccess;
}

}  // namespace

// A group of handles stepped together: one stream per member, forked from and joined
// back to the caller's stream, so that a whole group call captures as one CUDA graph
// whose branches run concurrently.
// With `shared` set (mixed members of one Taylor order, at most mixed::GROUP_MAX of them), the
// Taylor-term GEMMs (AFQMC_GROUP_SHARED_TAYLOR) or every tensor-core GEMM of a step
// (AFQMC_GROUP_SHARED_ALL) are each one persistent launch over the tiles of all members on
// the caller's stream, and the rest of the step runs on the member streams.
struct afqmc_kp_group {
  std::vector<afqmc_kp*> members;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  int launches = 0;
  int shared = AFQMC_GROUP_PER_MEMBER;
};

namespace {

void group_free(afqmc_kp_group* g) {
  for (auto s : g->streams) cudaStreamDestroy(s);
  for (auto e : g->joins) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  delete g;
}

// Runs fn(i, member, member stream) for every member between a fork and a join on st.
// Every member that was forked is joined, also after an error.
template <typename F>
cudaError_t fork_join(afqmc_kp_group* g, cudaStream_t st, F&& fn) {
  cudaError_t e = cudaEventRecord(g->fork, st);
  if (e != cudaSuccess) return e;
  size_t forked = 0;
  cudaError_t err = cudaSuccess;
  for (size_t i = 0; i < g->members.size(); ++i) {
    e = cudaStreamWaitEvent(g->streams[i], g->fork, 0);
    if (e != cudaSuccess) { err = e; break; }
    ++forked;
    e = fn((int)i, g->members[i], g->streams[i]);
    if (e != cudaSuccess) { err = e; break; }
  }
  for (size_t i = 0; i < forked; ++i) {
    e = cudaEventRecord(g->joins[i], g->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g->joins[i], 0);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
  return err;
}

// A group call: the launch counts of the members start at 0 and add up to the group's.
template <typename F>
cudaError_t group_run(afqmc_kp_group* g, F&& body) {
  for (afqmc_kp* h : g->members) h->launches = 0;
  const cudaError_t e = body();
  g->launches = 0;
  for (afqmc_kp* h : g->members) g->launches += h->launches;
  return e;
}

bool group_shareable(const afqmc_kp_group* g) {
  if (g->members.size() > (size_t)mixed::GROUP_MAX) return false;
  for (const afqmc_kp* h : g->members)
    if (!h->mixed || h->order != g->members[0]->order) return false;
  return true;
}

// One step of every member with the shared GEMM launches (mixed::group_step); keeps each
// member's stored-Green bookkeeping as step_impl does.
cudaError_t group_step_shared(afqmc_kp_group* g, void* const* phi, const double* const* x, double* const* weight,
                              void* const* eloc, void* const* logdet, int do_qr, int flags, cudaStream_t st) {
  const size_t n = g->members.size();
  std::vector<zc*> ph(n), el(n), ld(n);
  std::vector<int> reuse(n);
  for (size_t i = 0; i < n; ++i) {
    afqmc_kp* h = g->members[i];
    ph[i] = static_cast<zc*>(phi[i]);
    el[i] = eloc ? static_cast<zc*>(eloc[i]) : nullptr;
    ld[i] = logdet ? static_cast<zc*>(logdet[i]) : nullptr;
    reuse[i] = (flags & AFQMC_STEP_REUSE_GREEN) && h->green_valid && h->green_phi == phi[i];
    h->green_valid = false;
  }
  const mixed::ForEach each = [&](const mixed::MemberFn& fn) { return fork_join(g, st, fn); };
  const cudaError_t e = mixed::group_step(g->members.data(), (int)n, ph.data(), x, weight, el.data(), ld.data(),
                                          do_qr, reuse.data(), g->shared == AFQMC_GROUP_SHARED_ALL, each, st);
  if (e == cudaSuccess)
    for (size_t i = 0; i < n; ++i) {
      g->members[i]->green_valid = true;
      g->members[i]->green_phi = phi[i];
    }
  return e;
}

// afqmc_kp_group_block with the shared GEMM launches: block_impl's sequence, every step
// through group_step_shared.
cudaError_t group_block_shared(afqmc_kp_group* g, void* const* phi, double* const* weight, double* const* x,
                               void* const* eloc_hist, double* const* weight_hist, void* const* logdet, int nsteps,
                               int qr_period, int energy_period, int flags, int comb, unsigned long long seed,
                               unsigned long long* const* counter, cudaStream_t st) {
  const size_t n = g->members.size();
  std::vector<void*> el(n), ld(n);
  for (int s = 0; s < nsteps; ++s) {
    MTRY_API(fork_join(g, st, [&](int i, afqmc_kp* h, cudaStream_t ms) {
      return rng::fields(h, seed, counter[i], x[i], ms);
    }));
    const int do_qr = ((s + 1) % qr_period == 0) || s == nsteps - 1;
    const int measure = ((s + 1) % energy_period == 0) || s == nsteps - 1;
    for (size_t i = 0; i < n; ++i) {
      el[i] = measure ? static_cast<void*>(static_cast<zc*>(eloc_hist[i]) +
                                           (size_t)(s / energy_period) * g->members[i]->W * 3)
                      : nullptr;
      ld[i] = (s == nsteps - 1 && logdet) ? logdet[i] : nullptr;
    }
    MTRY_API(group_step_shared(g, phi, x, weight, el.data(), ld.data(), do_qr,
                               s == 0 ? flags : AFQMC_STEP_REUSE_GREEN, st));
    if (weight_hist)
      MTRY_API(fork_join(g, st, [&](int i, afqmc_kp* h, cudaStream_t ms) {
        return cudaMemcpyAsync(weight_hist[i] + (size_t)s * h->W, weight[i], sizeof(double) * h->W,
                               cudaMemcpyDeviceToDevice, ms);
      }));
  }
  if (!comb) return cudaSuccess;
  return fork_join(g, st, [&](int i, afqmc_kp* h, cudaStream_t ms) {
    h->green_valid = false;
    return rng::comb(h, static_cast<zc*>(phi[i]), weight[i], seed, counter[i], nullptr, ms);
  });
}

}  // namespace

extern "C" {

const char* afqmc_last_message(void) { return g_msg; }

const char* afqmc_status_string(afqmc_status s) {
  switch (s) {
    case AFQMC_OK: return "ok";
    case AFQMC_ERR_INVALID: return "invalid argument";
    case AFQMC_ERR_OOM: return "out of device memory (or over workspace cap)";
    case AFQMC_ERR_CUDA: return "CUDA error";
    case AFQMC_ERR_SINGULAR: return "singular walker overlap";
    case AFQMC_ERR_TIMEOUT: return "bounded device wait timed out";
    case AFQMC_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

afqmc_status afqmc_kp_create(const afqmc_kp_desc* desc, const void* L, const void* h1, const void* trial,
                             void* stream, afqmc_kp_t* out) {
  if (!valid_desc(desc) || !L || !h1 || !trial || !out) return AFQMC_ERR_INVALID;
  if ((long)desc->nocc * desc->M > 1024) return AFQMC_ERR_UNSUPPORTED;
  afqmc_kp* h = new (std::nothrow) afqmc_kp();
  if (!h) return AFQMC_ERR_OOM;
  try {
    h->d = *desc;
    h->nk = desc->kgrid[0] * desc->kgrid[1] * desc->kgrid[2];
    h->M = desc->M;
    h->n = desc->nocc;
    h->G = desc->nchol;
    h->W = desc->nwalkers;
    h->NM = h->nk * h->M;
    h->N = h->nk * h->n;
    h->order = desc->taylor_order;
    h->dt = desc->dt;
    h->sqdt = sqrt(desc->dt);
    momentum_tables(desc->kgrid, h->h_kminus, h->h_minus);
    cudaStream_t st = as_stream(stream);
    const size_t nk = h->nk, M = h->M, n = h->n, G = h->G, W = h->W, NM = h->NM, N = h->N;
    cudaError_t e = cudaSuccess;
#define TRY(x)                         \
  do {                                 \
    if ((e = (x)) != cudaSuccess) {    \
      afqmc_status s_ = from_cuda(e);  \
      free_all(h);                     \
      delete h;                        \
      cudaGetLastError();              \
      return s_;                       \
    }                                  \
  } while (0)
    TRY(alloc(h, &h->kminus, nk * nk));
    TRY(alloc(h, &h->minus, nk));
    TRY(alloc(h, &h->L, nk * nk * G * M * M));
    TRY(alloc(h, &h->LH, nk * nk * G * n * M));
    TRY(alloc(h, &h->A, nk * M * n));
    TRY(alloc(h, &h->h1, nk * M * M));
    TRY(alloc(h, &h->AhH, nk * n * M));
    TRY(alloc(h, &h->v0, nk * M * M));
    TRY(alloc(h, &h->Ehalf, nk * M * M));
    TRY(alloc(h, &h->expm_tmp, nk * 3 * M * M));
    TRY(alloc(h, &h->S, W * 2 * N * N));
    TRY(alloc(h, &h->Sinv, W * 2 * N * N));
    TRY(alloc(h, &h->Gh, W * 2 * N * NM));
    TRY(alloc(h, &h->X, W * nk * G));
    TRY(alloc(h, &h->xbar, W * 2 * nk * G));
    TRY(alloc(h, &h->y, W * nk * G));
    TRY(alloc(h, &h->ld_old, W * 2));
    TRY(alloc(h, &h->ld_new, W * 2));
    TRY(alloc(h, &h->sing_old, W * 2));
    TRY(alloc(h, &h->sing_new, W * 2));
    TRY(alloc(h, &h->epart, W * 2 * nk * nk));
    TRY(alloc(h, &h->Gam, W * 2 * N * NM));
    TRY(alloc(h, &h->P, W * 2 * N * N));
    TRY(alloc(h, &h->flags, 4));
    if (desc->prec == AFQMC_FP64) {
      TRY(alloc(h, &h->V, W * NM * NM));
      TRY(alloc(h, &h->T0, W * 2 * NM * N));
      TRY(alloc(h, &h->T1, W * 2 * NM * N));
      TRY(alloc(h, &h->acc, W * 2 * NM * N));
    }
    if (desc->workspace_cap_bytes && h->bytes > desc->workspace_cap_bytes) {
      free_all(h);
      delete h;
      return AFQMC_ERR_OOM;
    }
    TRY(cudaMemcpyAsync(h->kminus, h->h_kminus.data(), sizeof(int) * nk * nk, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(h->minus, h->h_minus.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(h->L, L, sizeof(zc) * nk * nk * G * M * M, cudaMemcpyDefault, st));
    TRY(cudaMemcpyAsync(h->h1, h1, sizeof(zc) * nk * M * M, cudaMemcpyDefault, st));
    TRY(cudaMemcpyAsync(h->A, trial, sizeof(zc) * nk * M * n, cudaMemcpyDefault, st));
    TRY(cudaMemsetAsync(h->flags, 0, sizeof(int) * 4, st));
    TRY(cudaMemsetAsync(h->sing_old, 0, sizeof(int) * W * 2, st));
    TRY(cudaMemsetAsync(h->sing_new, 0, sizeof(int) * W * 2, st));
    TRY(fp64::setup_static(h, st));
    if (desc->prec == AFQMC_MIXED) {
      afqmc_status ms = mixed::create(h, st);
      if (ms != AFQMC_OK) {
        cudaStreamSynchronize(st);
        mixed::destroy(h);
        free_all(h);
        delete h;
        return ms;
      }
      if (desc->workspace_cap_bytes && h->bytes > desc->workspace_cap_bytes) {
        cudaStreamSynchronize(st);
        mixed::destroy(h);
        free_all(h);
        delete h;
        return AFQMC_ERR_OOM;
      }
    }
    TRY(cudaStreamSynchronize(st));
#undef TRY
    *out = h;
    return AFQMC_OK;
  } catch (...) {
    free_all(h);
    delete h;
    return AFQMC_ERR_OOM;
  }
}

afqmc_status afqmc_dense_create(const afqmc_dense_desc* d, const void* L, const void* h1, const void* trial,
                                void* stream, afqmc_kp_t* out) {
  if (!d || !L || !h1 || !trial || !out || (d->hermitian != 0 && d->hermitian != 1) || d->nchol < 1)
    return AFQMC_ERR_INVALID;
  const long Gp = (long)d->nchol * (d->hermitian ? 1 : 2);
  afqmc_kp_desc kd;
  memset(&kd, 0, sizeof(kd));
  kd.kgrid[0] = kd.kgrid[1] = kd.kgrid[2] = 1;
  kd.M = d->M;
  kd.nocc = d->nocc;
  kd.nchol = (int)(Gp < 1 << 30 ? Gp : 1 << 30);
  kd.nwalkers = d->nwalkers;
  kd.dt = d->dt;
  kd.taylor_order = d->taylor_order;
  kd.prec = d->prec;
  kd.workspace_cap_bytes = d->workspace_cap_bytes;
  if (!valid_desc(&kd)) return AFQMC_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  const size_t per = (size_t)d->M * d->M;
  zc* src = nullptr;
  zc* vec = nullptr;
  cudaError_t e = cudaMalloc(&src, sizeof(zc) * per * d->nchol);
  if (e == cudaSuccess) e = cudaMalloc(&vec, sizeof(zc) * per * Gp);
  if (e == cudaSuccess) e = cudaMemcpyAsync(src, L, sizeof(zc) * per * d->nchol, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = dense::hermitian_vectors(src, vec, d->nchol, d->M, d->hermitian, st);
  afqmc_status s = e == cudaSuccess ? afqmc_kp_create(&kd, vec, h1, trial, stream, out) : from_cuda(e);
  cudaError_t f = cudaStreamSynchronize(st);   // the handle has copied the vectors
  cudaFree(src);
  cudaFree(vec);
  if (s == AFQMC_OK && f != cudaSuccess) {
    afqmc_kp_destroy(*out);
    *out = nullptr;
    return from_cuda(f);
  }
  return s;
}

afqmc_status afqmc_kp_destroy(afqmc_kp_t h) {
  if (!h) return AFQMC_ERR_INVALID;
  cudaError_t e = cudaDeviceSynchronize();
  mixed::destroy(h);
  free_all(h);
  for (auto& r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto ev : h->event_pool) cudaEventDestroy(ev);
  delete h;
  return from_cuda(e);
}

afqmc_status afqmc_kp_set_one_body(afqmc_kp_t h, const void* h1, void* stream) {
  if (!h || !h1) return AFQMC_ERR_INVALID;
  h->launches = 0;
  h->green_valid = false;
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(h->h1, h1, sizeof(zc) * (size_t)h->nk * h->M * h->M, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = fp64::set_one_body(h, st);
  if (e == cudaSuccess && h->mixed) e = mixed::set_one_body(h, st);
  return from_cuda(e);
}

afqmc_status afqmc_kp_force_bias(afqmc_kp_t h, const void* phi, void* xbar, void* stream) {
  if (!h || !phi || !xbar || !al16(phi, xbar)) return AFQMC_ERR_INVALID;
  h->launches = 0;
  h->green_valid = false;
  cudaStream_t st = as_stream(stream);
  cudaError_t e;
  if (h->mixed) {
    e = mixed::force_bias(h, static_cast<const zc*>(phi), static_cast<zc*>(xbar), st);
  } else {
    e = fp64::green(h, static_cast<const zc*>(phi), st);
    if (e == cudaSuccess) e = fp64::cholesky_trace(h, st);
    if (e == cudaSuccess) e = fp64::force_bias(h, nullptr, static_cast<zc*>(xbar), st);
  }
  return from_cuda(e);
}

afqmc_status afqmc_kp_propagate(afqmc_kp_t h, void* phi, const double* x, double* weight, void* logdet,
                                int do_qr, void* stream) {
  if (!h || !phi || !x || !weight || (do_qr != 0 && do_qr != 1) || !al16(phi, logdet)) return AFQMC_ERR_INVALID;
  h->launches = 0;
  h->green_valid = false;
  cudaStream_t st = as_stream(stream);
  cudaError_t e;
  if (h->mixed)
    e = mixed::propagate(h, static_cast<zc*>(phi), x, weight, static_cast<zc*>(logdet), do_qr, st);
  else
    e = fp64::propagate(h, static_cast<zc*>(phi), x, weight, static_cast<zc*>(logdet), do_qr, st);
  return from_cuda(e);
}

afqmc_status afqmc_kp_step(afqmc_kp_t h, void* phi, const double* x, double* weight, void* eloc, void* logdet,
                           int do_qr, int flags, void* stream) {
  if (!h || !phi || !x || !weight || (do_qr != 0 && do_qr != 1) || (flags & ~AFQMC_STEP_REUSE_GREEN) ||
      !al16(phi, eloc, logdet))
    return AFQMC_ERR_INVALID;
  h->launches = 0;
  return from_cuda(step_impl(h, phi, x, weight, eloc, logdet, do_qr, flags, as_stream(stream)));
}

afqmc_status afqmc_kp_orthonormalise(afqmc_kp_t h, void* phi, void* logdet, void* stream) {
  if (!h || !phi || !al16(phi, logdet)) return AFQMC_ERR_INVALID;
  h->launches = 0;
  h->green_valid = false;
  cudaStream_t st = as_stream(stream);
  cudaError_t e;
  if (h->mixed)
    e = mixed::orthonormalise(h, static_cast<zc*>(phi), static_cast<zc*>(logdet), st);
  else
    e = fp64::orthonormalise(h, static_cast<zc*>(phi), static_cast<zc*>(logdet), st);
  return from_cuda(e);
}

afqmc_status afqmc_kp_local_energy(afqmc_kp_t h, const void* phi, void* eloc, void* stream) {
  if (!h || !phi || !eloc || !al16(phi, eloc)) return AFQMC_ERR_INVALID;
  h->launches = 0;
  h->green_valid = false;
  cudaStream_t st = as_stream(stream);
  cudaError_t e;
  if (h->mixed)
    e = mixed::local_energy(h, static_cast<const zc*>(phi), static_cast<zc*>(eloc), st);
  else
    e = fp64::local_energy(h, static_cast<const zc*>(phi), static_cast<zc*>(eloc), st);
  return from_cuda(e);
}

afqmc_status afqmc_kp_local_energy_backward(afqmc_kp_t h, const void* phi, const void* grad_e, void* grad_phi,
                                            void* grad_h1, void* stream) {
  if (!h || !phi || !grad_e || !al16(phi, grad_e, grad_phi, grad_h1)) return AFQMC_ERR_INVALID;
  h->launches = 0;
  h->green_valid = false;
  cudaStream_t st = as_stream(stream);
  cudaError_t e;
  if (h->mixed)
    e = mixed::local_energy_backward(h, static_cast<const zc*>(phi), static_cast<const zc*>(grad_e),
                                     static_cast<zc*>(grad_phi), static_cast<zc*>(grad_h1), st);
  else
    e = fp64::local_energy_backward(h, static_cast<const zc*>(phi), static_cast<const zc*>(grad_e),
                                    static_cast<zc*>(grad_phi), static_cast<zc*>(grad_h1), st);
  return from_cuda(e);
}

afqmc_status afqmc_kp_last_error(afqmc_kp_t h, void* stream, int* n_singular) {
  if (!h) return AFQMC_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return AFQMC_ERR_CUDA;
  e = cudaGetLastError();
  if (e != cudaSuccess) return AFQMC_ERR_CUDA;
  int f[4] = {0, 0, 0, 0};
  if (cudaMemcpy(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return AFQMC_ERR_CUDA;
  if (cudaMemset(h->flags, 0, sizeof(f)) != cudaSuccess) return AFQMC_ERR_CUDA;
  if (n_singular) *n_singular = f[0];
  if (f[1]) return AFQMC_ERR_TIMEOUT;
  if (f[2]) {   // the tensor-core vHS left the range of its fixed-scale fp16 format
    snprintf(g_msg, sizeof(g_msg), "vHS entry beyond the split format's range (|V| >= 58)");
    return AFQMC_ERR_UNSUPPORTED;
  }
  if (f[0]) return AFQMC_ERR_SINGULAR;
  if (f[3]) return AFQMC_ERR_INVALID;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_memory_bytes(afqmc_kp_t h, size_t* bytes) {
  if (!h || !bytes) return AFQMC_ERR_INVALID;
  *bytes = h->bytes;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_profile(afqmc_kp_t h, int enable) {
  if (!h) return AFQMC_ERR_INVALID;
  h->prof_on = enable != 0;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_stage_times(afqmc_kp_t h, double* ms, int* count) {
  if (!h || !ms || !count) return AFQMC_ERR_INVALID;
  for (int i = 0; i < AFQMC_NSTAGES; ++i) { ms[i] = 0.0; count[i] = 0; }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return from_cuda(e);
  for (auto& r : h->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.stage >= 0 && r.stage < AFQMC_NSTAGES) {
      ms[r.stage] += t;
      count[r.stage] += 1;
    }
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->recs.clear();
  return AFQMC_OK;
}

afqmc_status afqmc_philox4x32_10(const unsigned int* ctr, unsigned long long seed, unsigned int* out, size_t n,
                                 void* stream) {
  if (n > 0 && (!ctr || !out)) return AFQMC_ERR_INVALID;
  // rows of four words are moved as 16-byte vectors
  if (n > 0 && ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15u)) return AFQMC_ERR_INVALID;
  return from_cuda(rng::philox(ctr, seed, out, n, as_stream(stream)));
}

afqmc_status afqmc_kp_fields(afqmc_kp_t h, unsigned long long seed, unsigned long long* counter, double* x,
                             void* stream) {
  if (!h || !counter || !x) return AFQMC_ERR_INVALID;
  h->launches = 0;
  return from_cuda(rng::fields(h, seed, counter, x, as_stream(stream)));
}

afqmc_status afqmc_kp_comb(afqmc_kp_t h, void* phi, double* weight, unsigned long long seed,
                           const unsigned long long* counter, int* idx, void* stream) {
  if (!h || !phi || !weight || !counter || !al16(phi)) return AFQMC_ERR_INVALID;
  if (rng::comb_smem_bytes(h->W) > 227 * 1024) return AFQMC_ERR_UNSUPPORTED;
  h->launches = 0;
  h->green_valid = false;
  return from_cuda(rng::comb(h, static_cast<zc*>(phi), weight, seed, counter, idx, as_stream(stream)));
}

afqmc_status afqmc_kp_block(afqmc_kp_t h, void* phi, double* weight, double* x, void* eloc_hist,
                            double* weight_hist, void* logdet, int nsteps, int qr_period, int energy_period,
                            int flags, int comb, unsigned long long seed, unsigned long long* counter, int* idx,
                            void* stream) {
  if (!h || !phi || !weight || !x || !eloc_hist || !counter || !block_args_ok(nsteps, qr_period, energy_period, flags,
                                                                            comb) ||
      !al16(phi, eloc_hist, logdet))
    return AFQMC_ERR_INVALID;
  if (comb && rng::comb_smem_bytes(h->W) > 227 * 1024) return AFQMC_ERR_UNSUPPORTED;
  h->launches = 0;
  return from_cuda(block_impl(h, phi, weight, x, eloc_hist, weight_hist, logdet, nsteps, qr_period, energy_period,
                              flags, comb, seed, counter, idx, as_stream(stream)));
}

afqmc_status afqmc_kp_group_create(const afqmc_kp_t* systems, int nsys, afqmc_kp_group_t* out) {
  if (!systems || !out || nsys < 1 || nsys > 64) return AFQMC_ERR_INVALID;
  for (int i = 0; i < nsys; ++i) {
    if (!systems[i]) return AFQMC_ERR_INVALID;
    for (int j = 0; j < i; ++j)
      if (systems[j] == systems[i]) return AFQMC_ERR_INVALID;   // members share no workspace
  }
  afqmc_kp_group* g = new (std::nothrow) afqmc_kp_group();
  if (!g) return AFQMC_ERR_OOM;
  try {
    g->members.assign(systems, systems + nsys);
    cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    for (int i = 0; i < nsys && e == cudaSuccess; ++i) {
      cudaStream_t s = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e == cudaSuccess) g->streams.push_back(s);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) g->joins.push_back(ev);
    }
    if (e != cudaSuccess) {
      group_free(g);
      return from_cuda(e);
    }
    g->shared = group_shareable(g) ? AFQMC_GROUP_SHARED_TAYLOR : AFQMC_GROUP_PER_MEMBER;
  } catch (...) {
    group_free(g);
    return AFQMC_ERR_OOM;
  }
  *out = g;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_group_destroy(afqmc_kp_group_t g) {
  if (!g) return AFQMC_ERR_INVALID;
  cudaError_t e = cudaSuccess;
  for (auto s : g->streams) {
    cudaError_t f = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = f;
  }
  group_free(g);
  return from_cuda(e);
}

afqmc_status afqmc_kp_group_step(afqmc_kp_group_t g, void* const* phi, const double* const* x, double* const* weight,
                                 void* const* eloc, void* const* logdet, int do_qr, int flags, void* stream) {
  if (!g || !phi || !x || !weight || (do_qr != 0 && do_qr != 1) || (flags & ~AFQMC_STEP_REUSE_GREEN))
    return AFQMC_ERR_INVALID;
  for (size_t i = 0; i < g->members.size(); ++i)
    if (!phi[i] || !x[i] || !weight[i] || !al16(phi[i], eloc ? eloc[i] : nullptr, logdet ? logdet[i] : nullptr))
      return AFQMC_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  try {   // the shared path's host arrays may fail to allocate
    return from_cuda(group_run(g, [&] {
      if (g->shared) return group_step_shared(g, phi, x, weight, eloc, logdet, do_qr, flags, st);
      return fork_join(g, st, [&](int i, afqmc_kp* h, cudaStream_t s) {
        return step_impl(h, phi[i], x[i], weight[i], eloc ? eloc[i] : nullptr, logdet ? logdet[i] : nullptr, do_qr,
                         flags, s);
      });
    }));
  } catch (...) {
    return AFQMC_ERR_OOM;
  }
}

afqmc_status afqmc_kp_group_block(afqmc_kp_group_t g, void* const* phi, double* const* weight, double* const* x,
                                  void* const* eloc_hist, double* const* weight_hist, void* const* logdet, int nsteps,
                                  int qr_period, int energy_period, int flags, int comb, unsigned long long seed,
                                  unsigned long long* const* counter, void* stream) {
  if (!g || !phi || !weight || !x || !eloc_hist || !counter ||
      !block_args_ok(nsteps, qr_period, energy_period, flags, comb))
    return AFQMC_ERR_INVALID;
  for (size_t i = 0; i < g->members.size(); ++i) {
    if (!phi[i] || !weight[i] || !x[i] || !eloc_hist[i] || !counter[i] ||
        !al16(phi[i], eloc_hist[i], logdet ? logdet[i] : nullptr))
      return AFQMC_ERR_INVALID;
    if (comb && rng::comb_smem_bytes(g->members[i]->W) > 227 * 1024) return AFQMC_ERR_UNSUPPORTED;
  }
  cudaStream_t st = as_stream(stream);
  try {   // the shared path's host arrays may fail to allocate
    return from_cuda(group_run(g, [&] {
      if (g->shared)
        return group_block_shared(g, phi, weight, x, eloc_hist, weight_hist, logdet, nsteps, qr_period,
                                  energy_period, flags, comb, seed, counter, st);
      return fork_join(g, st, [&](int i, afqmc_kp* h, cudaStream_t s) {
        return block_impl(h, phi[i], weight[i], x[i], eloc_hist[i], weight_hist ? weight_hist[i] : nullptr,
                          logdet ? logdet[i] : nullptr, nsteps, qr_period, energy_period, flags, comb, seed,
                          counter[i], nullptr, s);
      });
    }));
  } catch (...) {
    return AFQMC_ERR_OOM;
  }
}

afqmc_status afqmc_kp_group_set_shared(afqmc_kp_group_t g, int shared) {
  if (!g || shared < AFQMC_GROUP_PER_MEMBER || shared > AFQMC_GROUP_SHARED_TAYLOR) return AFQMC_ERR_INVALID;
  if (shared != AFQMC_GROUP_PER_MEMBER && !group_shareable(g)) return AFQMC_ERR_UNSUPPORTED;
  g->shared = shared;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_group_shared(afqmc_kp_group_t g, int* shared) {
  if (!g || !shared) return AFQMC_ERR_INVALID;
  *shared = g->shared;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_group_launch_count(afqmc_kp_group_t g, int* launches) {
  if (!g || !launches) return AFQMC_ERR_INVALID;
  *launches = g->launches;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_gemm_tuning(afqmc_kp_t h, int* depth, double* ms2, double* ms3, int* count) {
  if (!h || !count) return AFQMC_ERR_INVALID;
  if (!h->mixed) {
    *count = 0;
    return AFQMC_OK;
  }
  if (!depth || !ms2 || !ms3) return AFQMC_ERR_INVALID;
  mixed::gemm_tuning(h, depth, ms2, ms3);
  *count = AFQMC_NGEMMS;
  return AFQMC_OK;
}

afqmc_status afqmc_kp_gemm_form(afqmc_kp_t h, int gemm, int* pair, double* ms_pair) {
  if (!h || !pair || !ms_pair || gemm < 0 || gemm >= AFQMC_NGEMMS) return AFQMC_ERR_INVALID;
  if (!h->mixed) {
    *pair = 0;
    *ms_pair = 0.0;
    return AFQMC_OK;
  }
  mixed::gemm_form(h, gemm, pair, ms_pair);
  return AFQMC_OK;
}

afqmc_status afqmc_kp_set_gemm_form(afqmc_kp_t h, int gemm, int pair) {
  if (!h || gemm < 0 || gemm >= AFQMC_NGEMMS || (pair != 0 && pair != 1)) return AFQMC_ERR_INVALID;
  if (!h->mixed) return pair ? AFQMC_ERR_UNSUPPORTED : AFQMC_OK;
  return mixed::set_gemm_form(h, gemm, pair) ? AFQMC_OK : AFQMC_ERR_UNSUPPORTED;
}

afqmc_status afqmc_kp_launch_count(afqmc_kp_t h, int* launches) {
  if (!h || !launches) return AFQMC_ERR_INVALID;
  *launches = h->launches;
  return AFQMC_OK;
}

}  // extern "C"
