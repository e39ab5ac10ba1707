/*
 * afqmc_kp.h -- C ABI of the k-point phaseless AFQMC walker step on one GPU.
 *
 * The library implements the data-parallel hot path of phaseless auxiliary-field
 * quantum Monte Carlo with momentum-blocked Cholesky vectors (Malone, Zhang and
 * Morales, "Accelerating AFQMC simulations of solids with GPUs",
 * arXiv:2003.09468): one walker step over a batch of Slater-determinant walkers
 * (Green's function, force bias, vHS, Taylor exponential, one-body halves,
 * hybrid weight, optional re-orthonormalisation) and the mixed local energy with
 * its adjoint.  Every step runs in the library's own CUDA kernels (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im) pairs of IEEE doubles ("c128");
 *   arrays are row-major (C order), with the shapes stated per argument.
 * - Symbols: Nk = kgrid[0]*kgrid[1]*kgrid[2] k-points (Gamma-centred grid,
 *   k index in C order over the three axes), M orbitals per k, n = nocc occupied
 *   orbitals per k per spin, NM = Nk*M, N = Nk*n, G = nchol Cholesky vectors
 *   per momentum transfer Q, W = nwalkers.  k - Q is taken modulo the grid.
 * - Array pointers passed to calls other than afqmc_kp_create are DEVICE pointers
 *   on the current device, owned by the caller, and must stay valid until the
 *   work enqueued on `stream` has finished.  Complex arrays (c128: interleaved
 *   (re, im) doubles) must be 16-byte aligned, as cudaMalloc and PyTorch
 *   allocations are; an unaligned complex array is refused with AFQMC_ERR_INVALID.  `stream` is a cudaStream_t (NULL
 *   means the legacy default stream).  Calls are asynchronous: they enqueue
 *   kernels and return without synchronising, except where stated.
 * - After afqmc_kp_create returns, no call allocates device memory, so every
 *   call may be captured in a CUDA graph.
 * - No C++ exception crosses the ABI.  Invalid arguments are rejected with
 *   AFQMC_ERR_INVALID before any work is enqueued.  A failed kernel launch
 *   returns AFQMC_ERR_CUDA; an asynchronous fault surfaces as AFQMC_ERR_CUDA from
 *   a later call or from afqmc_kp_last_error.
 * - A handle is not thread safe: calls on one handle must not overlap in time
 *   (they share its workspace), whatever stream they use.
 */
#ifndef AFQMC_KP_H
#define AFQMC_KP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AFQMC_OK = 0,
  AFQMC_ERR_INVALID = 1,     /* bad argument: NULL pointer, size out of range   */
  AFQMC_ERR_OOM = 2,         /* device allocation failed in afqmc_kp_create     */
  AFQMC_ERR_CUDA = 3,        /* a CUDA call or kernel launch failed             */
  AFQMC_ERR_SINGULAR = 4,    /* at least one walker had a singular overlap      */
  AFQMC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up              */
  AFQMC_ERR_UNSUPPORTED = 6  /* valid request this build does not implement     */
} afqmc_status;

typedef enum {
  /* Every contraction in complex128 on the FP64 pipes. */
  AFQMC_FP64 = 0,
  /* L-contractions (force bias, vHS, Taylor products, exchange), the Green's-
   * function product and the QR products on the tensor cores (split fp16
   * operands, FP32 accumulation); the overlap, its inverse and log-det in
   * double-float (about 48 bits) on the FP32 pipe; the weights and the energy
   * sums in FP64.  The QR is Cholesky-QR2 (the same unique Q with real positive
   * diag R as the FP64 path's Householder). */
  AFQMC_MIXED = 1
} afqmc_precision;

/* Sizes and parameters of one system; copied by afqmc_kp_create. */
typedef struct {
  int kgrid[3];        /* Monkhorst-Pack grid, each >= 1                          */
  int M;               /* orbitals per k-point, 1..128                            */
  int nocc;            /* occupied orbitals per k-point per spin, 1..M            */
  int nchol;           /* Cholesky vectors per Q, >= 1                            */
  int nwalkers;        /* walkers per call, >= 1                                  */
  double dt;           /* imaginary time step, > 0                                */
  int taylor_order;    /* terms of the exp(V) series beyond the identity, 1..16   */
  afqmc_precision prec;
  size_t workspace_cap_bytes; /* 0 = no cap; else create fails with OOM above it */
} afqmc_kp_desc;

typedef struct afqmc_kp* afqmc_kp_t;

/*
 * afqmc_kp_create -- upload a Hamiltonian and trial, precompute static data.
 *
 * Paper: Sec. 2.3, Eqs. kp_h1 and kp_h2 define h[k] and L[Q,k]; the half-rotated
 * Cholesky vectors LH[Q,k,g,a,r] = sum_p conj(A[k,p,a]) L[Q,k,g,p,r] are formed
 * once (Sec. 2.3, below Eq. kp_vhs); the one-body propagator exp(-dt/2 H1') with
 * H1' = h + v0 and v0[k] = -1/2 sum_{Q,g} L[Q,k,g] L[Q,k,g]^dagger (Sec. 2.1,
 * below Eq. hsq, and Eq. propagator) is formed by FP64 kernels.
 *
 *   desc   sizes and parameters (host pointer, copied).
 *   L      HOST or DEVICE c128 [Nk][Nk][G][M][M]: L[Q][k][g][p][r], p at k,
 *          r at k - Q.  Must satisfy L[-Q][k-Q][g] = L[Q][k][g]^dagger (Sec. 2.3);
 *          the library uses both members of each pair as given.
 *   h1     HOST or DEVICE c128 [Nk][M][M]: Hermitian one-body blocks h[k].
 *   trial  HOST or DEVICE c128 [Nk][M][n]: occupied trial orbitals A[k]
 *          (block diagonal in k, the same for both spins).
 *   stream stream used for the set-up kernels; create synchronises it before
 *          returning, so the caller's buffers may be freed afterwards.
 *   out    receives the handle; untouched on failure.
 * The library copies everything it needs and owns all its device memory.
 * Returns AFQMC_ERR_INVALID for bad sizes, AFQMC_ERR_OOM if the workspace does
 * not fit (or exceeds workspace_cap_bytes), AFQMC_ERR_UNSUPPORTED for a
 * precision mode this build lacks.
 */
afqmc_status afqmc_kp_create(const afqmc_kp_desc* desc, const void* L, const void* h1,
                             const void* trial, void* stream, afqmc_kp_t* out);

/* Sizes and parameters of one standard-representation system; copied by afqmc_dense_create. */
typedef struct {
  int M;               /* orbitals, 1..128                                          */
  int nocc;            /* occupied orbitals per spin, 1..M                          */
  int nchol;           /* Cholesky vectors G, >= 1 (2G <= 8192 unless hermitian)    */
  int nwalkers;        /* walkers per call, >= 1                                    */
  double dt;           /* imaginary time step, > 0                                  */
  int taylor_order;    /* terms of the exp(V) series beyond the identity, 1..16     */
  afqmc_precision prec;
  int hermitian;       /* 1: every L_g is Hermitian (e.g. real symmetric, real
                          orbitals at the Gamma point); 0: general complex vectors  */
  size_t workspace_cap_bytes; /* 0 = no cap                                         */
} afqmc_dense_desc;

/*
 * afqmc_dense_create -- a system in the standard (dense) representation of Sec. 2.2:
 * M orbitals, Cholesky vectors L[g][p][r] with v_{pqrs} = sum_g L_{pr,g} conj(L_{sq,g}),
 * one-body h[p][q] and trial A[p][a].  The potentials v_{g+/-} built from
 * (L_g +/- L_g^dag)/2 (Sec. 2.2) are Hermitian combinations A_g = (L_g + L_g^dag)/2 and
 * B_g = i (L_g - L_g^dag)/2 of the vectors, so the system is created as a handle with a
 * single k-point (kgrid 1x1x1) and the Hermitian vectors [A; B] (G' = 2G), or A alone
 * (G' = G) when hermitian = 1.  The exact equivalence needs the integrals to be
 * symmetric under the exchange of the two electrons (v_pqrs = v_qpsr), as Coulomb
 * integrals are.  Every entry point then applies to the returned handle, with
 * NM = M, N = nocc and fields x[W][2][1][G']: x[w][0][0][g] drives v_{g+} and, for
 * general vectors, x[w][0][0][G + g] drives v_{g-}; x[w][1] has no effect.  The force
 * bias comes back in the same layout (its second plane is zero).
 *   L      HOST or DEVICE c128 [G][M][M]
 *   h1     HOST or DEVICE c128 [M][M], Hermitian
 *   trial  HOST or DEVICE c128 [M][nocc]
 * Errors and ownership as for afqmc_kp_create (the library keeps its own copies; the
 * Hermitian set is built on the device in a temporary buffer freed before return).
 */
afqmc_status afqmc_dense_create(const afqmc_dense_desc* desc, const void* L, const void* h1,
                                const void* trial, void* stream, afqmc_kp_t* out);

/* Frees every device buffer of the handle (synchronises the device first). */
afqmc_status afqmc_kp_destroy(afqmc_kp_t h);

/*
 * afqmc_kp_set_one_body -- replace h[k] (e.g. h + lambda V1 for a response).
 * Paper: Sec. 2.3, Eq. kp_h1 (h block diagonal in k); Sec. 2.1, Eq. propagator.
 * Recomputes A[k]^dagger h[k] (energy) and exp(-dt/2 (h + v0)) (propagation).
 *   h1  DEVICE c128 [Nk][M][M], Hermitian per k (not checked).
 * Invalidates the stored Green's function.  AFQMC_ERR_INVALID on NULL arguments.
 */
afqmc_status afqmc_kp_set_one_body(afqmc_kp_t h, const void* h1, void* stream);

/*
 * afqmc_kp_force_bias -- xbar = -sqrt(dt) <psi_T|v|phi>/<psi_T|phi>.
 *
 * Paper: Sec. 2.1 (force-bias shift), Sec. 2.2 Eq. fb, Sec. 2.3 Eq. kp_vbias.
 * With X[w,Q,g] = sum_s sum_k sum_{a,r} LH[Q,k,g,a,r] Gh_s[(k,a),(k-Q,r)] and the
 * half-rotated Green's function Gh_s = (phi_s (A^dagger phi_s)^-1)^T (Eq. gfhrot):
 *   xbar[w][0][Q][g] = -sqrt(dt) * i (X[Q,g] + X[-Q,g]) / 2     ("+" fields)
 *   xbar[w][1][Q][g] = -sqrt(dt) * -(X[Q,g] - X[-Q,g]) / 2      ("-" fields)
 *   phi   DEVICE c128 [W][2][NM][N] walker orbitals, row (k,p), column (k',a).
 *   xbar  DEVICE c128 [W][2][Nk][G] output.
 */
afqmc_status afqmc_kp_force_bias(afqmc_kp_t h, const void* phi, void* xbar, void* stream);

/*
 * afqmc_kp_propagate -- one phaseless "hybrid" step of every walker.
 *
 * Paper: Sec. 2.1 Eqs. propagator and iterate_imp, the importance function I,
 * the hybrid weight and the phase; Sec. 2.2 Eq. vhs and the truncated Taylor
 * series; Sec. 2.3 Eq. kp_vhs.  Per walker:
 *   xbar from phi (as afqmc_kp_force_bias);
 *   V = sqrt(dt) sum_{Q,g} L^{Q g} y[Q,g],
 *       y = (i xt+_Q - xt-_Q)/2 + (i xt+_{-Q} + xt-_{-Q})/2,  xt = x - xbar;
 *   phi <- E * (sum_{j=0}^{taylor_order} V^j / j!) * E * phi,  E = exp(-dt/2 H1');
 *   R = prod_s det(A^dagger phi_s') / det(A^dagger phi_s), dtheta = arg R,
 *   w <- w * |R exp(sum_f x_f xbar_f - xbar_f^2 / 2)| * max(0, cos dtheta);
 *   if do_qr: phi_s <- Q of the QR factorisation with diag(R) real positive.
 *   phi     DEVICE c128 [W][2][NM][N], updated in place.
 *   x       DEVICE double [W][2][Nk][G] auxiliary fields (+ then -).
 *   weight  DEVICE double [W], updated in place.
 *   logdet  DEVICE c128 [W][2] output: log det(A^dagger phi_s) of the new
 *           walker (after QR if done), or NULL.
 *   do_qr   0 or 1.
 * A walker whose overlap matrix is singular gets weight 0 and a zero Green's
 * function; it is counted in the sticky flags read by afqmc_kp_last_error.
 */
afqmc_status afqmc_kp_propagate(afqmc_kp_t h, void* phi, const double* x, double* weight,
                                void* logdet, int do_qr, void* stream);

/* Flags of afqmc_kp_step. */
#define AFQMC_STEP_REUSE_GREEN 1

/*
 * afqmc_kp_step -- one hybrid step of every walker followed by the local
 * energy of the propagated walkers (a block of the paper's driver does many
 * such steps, Sec. 3.1).  The result equals afqmc_kp_propagate followed by
 * afqmc_kp_local_energy on the new walkers, but the Green's function of the
 * new walkers is formed once: it gives their log det for the weight update,
 * their energy, and (with AFQMC_STEP_REUSE_GREEN on the next call) the next
 * step's force bias.
 *   phi, x, weight, logdet, do_qr   as for afqmc_kp_propagate.
 *   eloc   DEVICE c128 [W][3] output: (E1, EC, EX) of the propagated walkers
 *          (a QR does not change them), or NULL for a propagation-only step: the
 *          Green's function of the new walkers is still formed (it gives their
 *          log det and the next force bias), the energy kernels are skipped.
 *   flags  0 or AFQMC_STEP_REUSE_GREEN.  With the flag, the caller promises
 *          that phi is the output of the previous afqmc_kp_step call on this
 *          handle and was not modified since; the stored Green's function,
 *          Cholesky trace and log det are then reused instead of recomputed.
 *          The library ignores the flag when another entry point ran on the
 *          handle in between or phi is a different pointer.
 */
afqmc_status afqmc_kp_step(afqmc_kp_t h, void* phi, const double* x, double* weight, void* eloc, void* logdet,
                           int do_qr, int flags, void* stream);

/*
 * afqmc_kp_orthonormalise -- phi_s <- Q factor of phi_s with diag(R) > 0
 * (the walker orthogonalisation done once per block, Sec. 3.1).
 *   phi     DEVICE c128 [W][2][NM][N], in place.
 *   logdet  DEVICE c128 [W][2] output (log det(A^dagger phi_s) after), or NULL.
 */
afqmc_status afqmc_kp_orthonormalise(afqmc_kp_t h, void* phi, void* logdet, void* stream);

/*
 * afqmc_kp_local_energy -- mixed local energy of every walker.
 *
 * Paper: Sec. 2.2 Eq. local_energy (E1 + E_C + E_X with X, X-bar, T, T-bar),
 * Sec. 2.3 Eq. kp_el, Sec. 3.2 energy steps 1-3.
 *   E1 = sum_s sum_k sum_{a,q} (A[k]^dagger h[k])[a,q] Gh_s[(k,a),(k,q)]
 *   EC = 1/2 sum_{Q,g} X[Q,g] X[-Q,g]
 *   EX = -1/2 sum_s sum_{Q,k,k'} sum_{g,a,b} T1[g,a,b] T2[g,b,a],
 *        T1 = sum_r LH[Q,k,g,a,r] Gh_s[(k'-Q,b),(k-Q,r)],
 *        T2 = sum_s LH[-Q,k'-Q,g,b,s] Gh_s[(k,a),(k',s)].
 *   phi   DEVICE c128 [W][2][NM][N].
 *   eloc  DEVICE c128 [W][3] output: (E1, EC, EX) per walker.
 */
afqmc_status afqmc_kp_local_energy(afqmc_kp_t h, const void* phi, void* eloc, void* stream);

/*
 * afqmc_kp_local_energy_backward -- adjoint of afqmc_kp_local_energy.
 *
 * Derived from Sec. 2.3 Eq. kp_el (the paper has no adjoint).  E is holomorphic
 * in phi; with upstream weights g[w][part] = dLoss/dconj(E_part) (PyTorch's
 * convention for complex tensors) the outputs are
 *   grad_phi[w] = sum_part g[w][part] * conj(dE_part[w] / dphi[w])
 *   grad_h1[k]  = sum_w g[w][0] * conj(dE1[w] / dh[k])
 *   phi       DEVICE c128 [W][2][NM][N].
 *   grad_e    DEVICE c128 [W][3].
 *   grad_phi  DEVICE c128 [W][2][NM][N] output, or NULL to skip.
 *   grad_h1   DEVICE c128 [Nk][M][M] output, or NULL to skip.
 * Exchange intermediates T2 are recomputed, never stored.
 */
afqmc_status afqmc_kp_local_energy_backward(afqmc_kp_t h, const void* phi, const void* grad_e,
                                            void* grad_phi, void* grad_h1, void* stream);

/*
 * afqmc_kp_last_error -- synchronise `stream`, read and clear the handle's
 * sticky device flags.  Returns AFQMC_ERR_SINGULAR if any walker had a singular
 * overlap since the last call (their count goes to *n_singular if non-NULL),
 * AFQMC_ERR_TIMEOUT if a bounded device wait gave up, AFQMC_ERR_UNSUPPORTED if a
 * tensor-core vHS entry left the range of its fixed-scale fp16 format (|V| >= 58;
 * the walkers of that step are not valid), AFQMC_ERR_INVALID if a comb met a total
 * weight that was not positive and finite, AFQMC_ERR_CUDA on an asynchronous CUDA
 * fault, else AFQMC_OK (precedence: CUDA, timeout, vHS range, singular, comb).
 */
afqmc_status afqmc_kp_last_error(afqmc_kp_t h, void* stream, int* n_singular);

/*
 * afqmc_kp_wait_selftest -- exercise the bounded device-side wait that every
 * mbarrier wait of the tensor-core kernels uses.  The paper has no counterpart:
 * this is a check of this library's failure handling.  A one-warp kernel
 * initialises an mbarrier for one arrival and waits on it with a limit of
 * limit_cycles SM clock cycles; with arrive = 1 the kernel makes the arrival
 * itself and the wait returns at once, with arrive = 0 nothing arrives, the wait
 * gives up after the limit and the kernel records a time-out in the handle's
 * sticky flags (afqmc_kp_last_error then returns AFQMC_ERR_TIMEOUT).  The kernel
 * issues no copy or MMA and holds no tensor memory, so the device stays usable.
 *   arrive        0 or 1.
 *   limit_cycles  1 .. 2^31 (about one second at the maximum SM clock).
 * AFQMC_ERR_INVALID on a NULL handle or arguments out of range; AFQMC_ERR_CUDA if
 * the launch fails.
 */
afqmc_status afqmc_kp_wait_selftest(afqmc_kp_t h, int arrive, long long limit_cycles, void* stream);

/* Device bytes owned by the handle (static data plus workspace). */
afqmc_status afqmc_kp_memory_bytes(afqmc_kp_t h, size_t* bytes);

/*
 * Per-stage timing with CUDA events recorded on the caller's stream around each
 * stage's kernels (the paper times its operations per block, Sec. 3.1-3.2; the
 * mechanism here is this library's own).  Stages:
 */
typedef enum {
  AFQMC_STAGE_GREEN = 0,       /* overlap, LU / inverse / log det, Green's function */
  AFQMC_STAGE_FORCE_BIAS = 1,  /* Cholesky trace X and xbar                         */
  AFQMC_STAGE_VHS = 2,         /* vHS build                                         */
  AFQMC_STAGE_TAYLOR = 3,      /* Taylor series; tensor-core path: the GEMMs alone,
                                  one interval per term (FP64 path: the one-body
                                  halves included, one interval per step)           */
  AFQMC_STAGE_WEIGHT = 4,      /* new overlap, log det and hybrid weight            */
  AFQMC_STAGE_QR = 5,          /* re-orthonormalisation                             */
  AFQMC_STAGE_ENERGY = 6,      /* E1, EC and the final sums                         */
  AFQMC_STAGE_EXCHANGE = 7,    /* the exchange contraction kernel alone             */
  AFQMC_STAGE_BACKWARD = 8,    /* adjoint kernels                                   */
  AFQMC_STAGE_ONEBODY = 9,     /* tensor-core path: the one-body halves around the
                                  Taylor series and the split of the series' input  */
  AFQMC_STAGE_ADJOINT_GEMM = 10, /* tensor-core path: the exchange adjoint GEMM alone
                                   (one interval per launch)                      */
  AFQMC_NSTAGES = 11
} afqmc_stage;

/* enable != 0 starts recording (allocates CUDA events on the host side as
 * needed; do not enable while capturing a graph); 0 stops.  */
afqmc_status afqmc_kp_profile(afqmc_kp_t h, int enable);

/* Synchronises the device, then writes for every stage the summed event time
 * in milliseconds (ms[AFQMC_NSTAGES]) and the number of recorded intervals
 * (count[AFQMC_NSTAGES]) since the last read, and clears them. */
afqmc_status afqmc_kp_stage_times(afqmc_kp_t h, double* ms, int* count);

/* Number of kernel launches the last entry point call enqueued. */
afqmc_status afqmc_kp_launch_count(afqmc_kp_t h, int* launches);

/*
 * afqmc_last_message -- NUL-terminated text of the most recent CUDA error the
 * library saw on the calling thread ("" if none).  Valid until the next call
 * on that thread; owned by the library.  The paper has no counterpart: this is
 * a diagnostic of this library.
 */
const char* afqmc_last_message(void);

/*
 * afqmc_orthonormalise_noalloc -- the walker re-orthonormalisation of
 * afqmc_kp_orthonormalise (Householder QR, phi <- Q with diag(R) real
 * positive) for callers that cannot allocate device memory: code running
 * while a CUDA graph is captured in global mode, where cudaMalloc fails, or a
 * plug-in inside a host program that owns every device byte.  It needs no
 * handle and calls no allocator; its scratch is a fixed array of
 * AFQMC_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library keeps until the process exits.  The paper has no
 * counterpart: this entry point exists only for such callers.
 *
 *   phi     DEVICE c128 [nmat][rows][cols], each matrix row-major, overwritten
 *           by its Q factor (the layout of one spin block of a walker).
 *   rows, cols, nmat   1 <= cols <= rows, cols <= 1024, nmat >= 1, and
 *           rows * cols * nmat * 16 bytes <= AFQMC_NOALLOC_SCRATCH_BYTES;
 *           larger requests return AFQMC_ERR_INVALID without doing anything.
 *   stream  cudaStream_t.
 * The first call on a device resolves the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array, so
 * calls whose work overlaps on the GPU (different streams, threads or
 * processes sharing the library image) race and must be serialised by the
 * caller.  The array keeps the last call's contents; the kernel overwrites
 * every entry it reads before reading it.
 */
#define AFQMC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
afqmc_status afqmc_orthonormalise_noalloc(void* phi, int rows, int cols, int nmat, void* stream);

/*
 * afqmc_kp_fields -- the auxiliary fields of one step drawn on the device:
 * x[w][2][Nk][G] ~ N(0,1), independent (Sec. 2.1: x is drawn from the standard
 * normal distribution at every step).  Uniform 32-bit words come from the
 * counter-based generator Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC 2011) with key = seed and counter
 * (q, w, c_lo, c_hi), q = field index / 4, c = *counter; each word pair (a, b)
 * becomes two normals by the Box-Muller transform in fp32:
 *   u1 = ((a >> 9) + 1/2) 2^-23, u2 = ((b >> 9) + 1/2) 2^-23 (exact in fp32, inside (0, 1)),
 *   r = sqrt(-2 ln u1), x = (r cos 2 pi u2, r sin 2 pi u2).
 *   seed     generator key (64 bits)
 *   counter  device pointer to one 64-bit step counter; the call draws with *counter and
 *            then increments it, in stream order, so a captured CUDA graph draws new
 *            fields on every replay
 *   x        device [W][2][Nk][G] double
 * Allocates nothing; AFQMC_ERR_INVALID on NULL arguments.
 */
afqmc_status afqmc_kp_fields(afqmc_kp_t h, unsigned long long seed, unsigned long long* counter, double* x,
                             void* stream);

/*
 * afqmc_philox4x32_10 -- the raw generator behind afqmc_kp_fields and afqmc_kp_comb:
 * out[i] = Philox4x32-10(ctr[i], key = (seed_lo, seed_hi)) for i < n (Salmon, Moraes, Dror
 * and Shaw, SC 2011: ten rounds of the multiply-and-swap bijection, the key advanced by the
 * Weyl constants between rounds).
 *   ctr   DEVICE uint32 [n][4] counters (c0, c1, c2, c3), 16-byte aligned
 *   out   DEVICE uint32 [n][4] words, 16-byte aligned
 * Needs no handle; n = 0 is a no-op; AFQMC_ERR_INVALID on NULL or unaligned pointers
 * with n > 0 (checked on the host, before any launch).
 */
afqmc_status afqmc_philox4x32_10(const unsigned int* ctr, unsigned long long seed, unsigned int* out, size_t n,
                                 void* stream);

/*
 * afqmc_kp_comb -- population control by the comb.  The walker weights are those of
 * Sec. 2.1 (the hybrid weight update); the paper leaves population control out, and
 * this is the standard comb (one uniform u per call): with cumulative
 * weights C_j = sum_{i<=j} w_i (in walker order) and total C = C_{W-1}, new walker k
 * is old walker j_k = min{ j : C_j > (k + u) C / W } and all new weights are C / W.
 * u = (a + 1/2) 2^-32 with a the first Philox4x32-10 word of counter
 * (0, 0xffffffff, c_lo, c_hi), c = *counter (the counter is not incremented; the
 * field counter of afqmc_kp_fields never takes that form while w < 2^32 - 1).
 * A total weight that is not positive and finite leaves everything as it is and is
 * counted in the sticky flags (afqmc_kp_last_error returns AFQMC_ERR_INVALID).
 *   phi     device [W][2][NM][N] complex128, in/out
 *   weight  device [W] double, in/out
 * Invalidates the stored Green's function, so the next afqmc_kp_step forms the
 * overlaps of the new population afresh.  A caller that keeps per-walker log dets
 * permutes them with the same indices: idx (device [W] int, may be NULL) receives j_k.
 * Allocates nothing (the gather goes through the handle's adjoint workspace).
 */
afqmc_status afqmc_kp_comb(afqmc_kp_t h, void* phi, double* weight, unsigned long long seed,
                           const unsigned long long* counter, int* idx, void* stream);

/*
 * afqmc_kp_block -- one block of the driver, fully on the device.  The paper's
 * block is 20 propagation steps followed by one energy evaluation and one walker
 * orthogonalisation (Sec. 3.1, Fig. timing); the hybrid weight needs no energy
 * in between.  Here, for s = 0 .. nsteps-1:
 *   afqmc_kp_fields(seed, counter, x);
 *   one hybrid step (afqmc_kp_step) of every walker, with
 *     do_qr  = ((s + 1) % qr_period == 0 or s == nsteps - 1),
 *     energy = ((s + 1) % energy_period == 0 or s == nsteps - 1), written to
 *              eloc_hist[m], m = s / energy_period (the steps without it skip the
 *              energy kernels: a propagation-only step);
 * then, when comb != 0, afqmc_kp_comb(phi, weight, seed, counter, idx).  The result
 * is bitwise that of the same calls made one by one.  Nothing synchronises with
 * the host, so the whole block can be captured in one CUDA graph and replayed
 * (the counter advances by nsteps per replay, so every replay draws new fields).
 *   phi, weight    in/out, as for afqmc_kp_step
 *   x              DEVICE double [W][2][Nk][G] scratch: the fields of the last step
 *   eloc_hist      DEVICE c128 [ceil(nsteps / energy_period)][W][3]: (E1, EC, EX)
 *   weight_hist    DEVICE double [nsteps][W]: the weights after step s, or NULL
 *   logdet         DEVICE c128 [W][2]: log dets after the last step, or NULL
 *   nsteps, qr_period, energy_period >= 1 (the paper's block: 20, 20, 20)
 *   flags          0 or AFQMC_STEP_REUSE_GREEN (applies to the first step only)
 *   comb           0 or 1; idx as for afqmc_kp_comb (NULL allowed)
 * AFQMC_ERR_INVALID on NULL required pointers or counts out of range.
 */
afqmc_status afqmc_kp_block(afqmc_kp_t h, void* phi, double* weight, double* x, void* eloc_hist,
                            double* weight_hist, void* logdet, int nsteps, int qr_period, int energy_period,
                            int flags, int comb, unsigned long long seed, unsigned long long* counter, int* idx,
                            void* stream);

/*
 * Groups: several independent systems (each its own handle, of any sizes and
 * precision) advanced by one call.  A group call forks from `stream` onto one
 * stream per member, runs every member's work there and joins back, so one
 * captured CUDA graph holds the whole group as concurrent branches and the small,
 * latency-bound kernels of different systems overlap on the GPU.  Groups of mixed
 * handles also share their GEMM launches (afqmc_kp_group_set_shared).  Each member
 * computes exactly what the same call on the member alone computes (bit for bit).
 * The walker sets of the members are the independent units of the paper's batching
 * (Sec. 3.2: operate on as many walkers at once as possible).
 */
typedef struct afqmc_kp_group* afqmc_kp_group_t;

/*
 * afqmc_kp_group_create -- a group of nsys (1..64) distinct handles.  The group
 * refers to the handles and does not own them: they must outlive the group, and
 * no other call may use them while a group call's work is in flight.  Creates one
 * non-blocking stream and one event per member.
 */
afqmc_status afqmc_kp_group_create(const afqmc_kp_t* systems, int nsys, afqmc_kp_group_t* out);

/* Synchronises the member streams and frees the group (not the member handles). */
afqmc_status afqmc_kp_group_destroy(afqmc_kp_group_t g);

/*
 * afqmc_kp_group_step -- afqmc_kp_step (Sec. 2.1-2.3, one hybrid step and the local
 * energy) on every member, batched as Sec. 3.2 advises.  phi, x, weight, eloc and
 * logdet are HOST arrays of nsys DEVICE pointers, entry i laid out as for member
 * i's afqmc_kp_step; eloc (the array, or an entry) and logdet may be NULL.
 * do_qr and flags apply to every member.
 */
afqmc_status afqmc_kp_group_step(afqmc_kp_group_t g, void* const* phi, const double* const* x,
                                 double* const* weight, void* const* eloc, void* const* logdet, int do_qr,
                                 int flags, void* stream);

/*
 * afqmc_kp_group_block -- afqmc_kp_block (the block of Sec. 3.1) on every member
 * (HOST arrays of DEVICE pointers as above; weight_hist and logdet may be NULL;
 * counter[i] is member i's step counter).  The comb acts within each member's
 * population.
 */
afqmc_status afqmc_kp_group_block(afqmc_kp_group_t g, void* const* phi, double* const* weight,
                                  double* const* x, void* const* eloc_hist, double* const* weight_hist,
                                  void* const* logdet, int nsteps, int qr_period, int energy_period,
                                  int flags, int comb, unsigned long long seed,
                                  unsigned long long* const* counter, void* stream);

/* Kernel launches of the last group call, all members together. */
afqmc_status afqmc_kp_group_launch_count(afqmc_kp_group_t g, int* launches);

/*
 * afqmc_kp_group_set_shared -- GEMM launches shared by the members in group_step and
 * group_block (Sec. 3.2: all walkers of all systems in one batched operation).
 *   AFQMC_GROUP_PER_MEMBER     every member launches its own GEMMs on its own stream;
 *   AFQMC_GROUP_SHARED_ALL     every tensor-core GEMM of a step (the Green's function, the
 *                              force bias, vHS, each Taylor term, the exchange) is one
 *                              persistent launch on `stream` over the tiles of every member,
 *                              each tile with its own member's operands, sizes and tensor maps;
 *                              the small kernels between the GEMMs run on the member streams;
 *   AFQMC_GROUP_SHARED_TAYLOR  only the six Taylor-term GEMMs are shared launches; the rest of
 *                              each member's step runs on its stream.
 * Either way each member computes bit for bit what it computes alone.  A group of 1..8 mixed
 * handles with one Taylor order starts with AFQMC_GROUP_SHARED_TAYLOR, any other group with
 * AFQMC_GROUP_PER_MEMBER; a shared mode on any other group is AFQMC_ERR_UNSUPPORTED.  GEMM
 * time-outs of a shared launch are reported by the first member's afqmc_kp_last_error.
 */
#define AFQMC_GROUP_PER_MEMBER 0
#define AFQMC_GROUP_SHARED_ALL 1
#define AFQMC_GROUP_SHARED_TAYLOR 2
afqmc_status afqmc_kp_group_set_shared(afqmc_kp_group_t g, int shared);
/* The group's mode (AFQMC_GROUP_*). */
afqmc_status afqmc_kp_group_shared(afqmc_kp_group_t g, int* shared);

/*
 * The tensor-core GEMMs of a mixed handle, and their autotuned TMA ring depth.  At create
 * the library times the step GEMMs (Green's function, force bias, vHS, a Taylor term,
 * exchange, exchange adjoint) with two- and three-stage rings on the handle's own operands
 * (three launches each, CUDA events) and keeps the faster for the handle's lifetime; the
 * depth changes how far the loads run ahead, not the arithmetic, so results do not depend on
 * it.  The QR GEMMs keep their defaults.
 */
typedef enum {
  AFQMC_GEMM_GREEN = 0,
  AFQMC_GEMM_FORCE_BIAS = 1,
  AFQMC_GEMM_VHS = 2,
  AFQMC_GEMM_TAYLOR = 3,
  AFQMC_GEMM_EXCHANGE = 4,
  AFQMC_GEMM_ADJOINT = 5,
  AFQMC_GEMM_GRAM = 6,
  AFQMC_GEMM_APPLY_R = 7,
  AFQMC_NGEMMS = 8
} afqmc_gemm;

/*
 * afqmc_kp_gemm_tuning -- the ring depth of every GEMM (depth[AFQMC_NGEMMS]) and the
 * per-launch milliseconds measured at create with two and three stages (ms2, ms3; 0 where a
 * GEMM was not timed).  HOST arrays.  *count = AFQMC_NGEMMS for a mixed handle, 0 for an
 * FP64 handle (no tensor-core GEMMs; the arrays are left untouched).
 */
afqmc_status afqmc_kp_gemm_tuning(afqmc_kp_t h, int* depth, double* ms2, double* ms3, int* count);

/*
 * afqmc_kp_gemm_form -- the tile form of one GEMM of a mixed handle.  *pair = 1: the CTA-pair
 * form (tcgen05 cta_group::2), where two SMs of a cluster compute 256-row tiles and each
 * stages its own 128 rows of A and one half (real or imaginary planes) of the paired B
 * operand, so the B operand is read from shared memory once per pair; *pair = 0: 128-row
 * tiles on one SM.  Only the Taylor-term GEMM (Sec. 3.2 step 3, more than one row tile per
 * walker) has the pair form: at create the library times it (four-stage ring) and keeps it
 * when it beats the single form at its tuned ring depth by more than 2%.  *ms_pair = that per-launch time in ms (0 if not timed, -1
 * if the device refused the cluster launch).  Both forms compute every output element with
 * the same products in the same order.  AFQMC_ERR_INVALID for NULL pointers or gemm out of
 * range; an FP64 handle reports 0.
 */
afqmc_status afqmc_kp_gemm_form(afqmc_kp_t h, int gemm, int* pair, double* ms_pair);
/*
 * afqmc_kp_set_gemm_form -- override the form chosen at create (pair 0 or 1).
 * AFQMC_ERR_UNSUPPORTED for pair = 1 on a GEMM or handle without the pair form (FP64, or
 * one row tile per walker), AFQMC_ERR_INVALID for other arguments out of range.
 */
afqmc_status afqmc_kp_set_gemm_form(afqmc_kp_t h, int gemm, int pair);

/* Static, NUL-terminated description of a status code. */
const char* afqmc_status_string(afqmc_status s);

#ifdef __cplusplus
}
#endif

#endif /* AFQMC_KP_H */
