"""FP64 CPU oracle for one k-point phaseless AFQMC walker step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the product library never
calls it and shares no code with it.

Plain, slow, obviously correct NumPy in complex128, written from the paper
(arXiv:2003.09468):

* Sec. 2.1, Eqs. hamil, hsq, hs, propagator, iterate_imp: Trotter split, the
  mean-field one-body term v0, importance sampling with the force bias, and the
  phaseless "hybrid" weight update.
* Sec. 2.2, Eqs. fb, gf, gfhrot, vhs, local_energy: Green's function, half
  rotation, force bias, vHS, Taylor-series exponential, and the local energy
  with its Coulomb (X, X-bar) and exchange (T, T-bar) intermediates.
* Sec. 2.3, Eqs. kp_h1, kp_h2, kp_vbias, kp_vhs, kp_el: the momentum-blocked
  Cholesky vectors L[Q, k] (p at k, r at k - Q), the (Q, -Q) relation and the
  k-blocked force bias, vHS and local energy.
* Sec. 3.2, energy-evaluation steps 1-3: the exchange is evaluated by looping
  over (spin, Q, k, k') and forming T1 and T2 per term.

Readings of garbled or silent passages (each is listed in the design notes):

1. Sign convention of the HS potentials: v_plus = i (L + L^dag)/2 and
   v_minus = -(L - L^dag)/2 (the paper's c_+ = 1, c_- = i times i), so that
   H2 = v0 - 1/2 sum v^2 holds with Hermitian-positive squares; x-bar =
   -sqrt(dt) <v>; the propagator acts on orbital coefficients as phi <- e^V phi.
2. Using L[Q, k]^dag = L[-Q, k-Q] every "L-bar" term becomes an L term at -Q:
   the force bias uses X_Q and X_{-Q}, the vHS uses a single contraction with
   y_Q = (i xt+_Q - xt-_Q)/2 + (i xt+_{-Q} + xt-_{-Q})/2, and T-bar of step
   2(b) is built from the half-rotated L at (-Q, k' - Q).
3. Coulomb energy E_C = 1/2 sum_{Q, g} X_{Q g} X_{-Q g} (the product of Sec.
   2.2, not a squared modulus).
4. The walker is dense in k (V couples every k to every k - Q); only the trial,
   h and the one-body propagator are block diagonal.
5. Taylor order p means sum_{j=0}^{p} V^j / j!.
6. The force bias is taken from phi at the start of the step; the overlap
   ratio covers the whole B(x - xbar), both one-body halves included; the
   phase is Delta theta = arg of that ratio; no energy shift, no capping.
7. Orthonormalisation: Householder QR with diag(R) real positive; phi <- Q;
   the log-overlap is recomputed and the weight is left alone.

Array conventions: L[Q, k, g, p, r]; LH[Q, k, g, a, r]; h[k, p, q];
A[k, p, a]; phi[s, NM, N] with row index (k, p) and column index (k', a);
Gh[s] = N x NM half-rotated Green's function with row (k, a), column (k', r);
fields x[+/-, Q, g] real; xbar[+/-, Q, g] complex.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg


# --------------------------------------------------------------------------
# k-point bookkeeping (Sec. 2.3: k - Q is taken modulo the Gamma-centred grid)
# --------------------------------------------------------------------------

def kgrid_tables(grid):
    """Return (kminus, minus): kminus[k, Q] = index of k - Q, minus[Q] = index of -Q."""
    g = np.array(grid, dtype=np.int64)
    kpts = np.array(list(itertools.product(*[range(int(v)) for v in grid])), dtype=np.int64)
    index = {tuple(v): i for i, v in enumerate(kpts)}
    nk = len(kpts)
    kminus = np.empty((nk, nk), dtype=np.int64)
    for k in range(nk):
        for Q in range(nk):
            kminus[k, Q] = index[tuple((kpts[k] - kpts[Q]) % g)]
    minus = np.array([index[tuple((-kpts[Q]) % g)] for Q in range(nk)], dtype=np.int64)
    return kminus, minus


def kplus(kminus, minus, k, Q):
    """Index of k + Q, i.e. k - (-Q)."""
    return kminus[k, minus[Q]]


# --------------------------------------------------------------------------
# Set-up quantities (computed once per Hamiltonian)
# --------------------------------------------------------------------------

def half_rotate(L, A):
    """LH[Q, k, g, a, r] = sum_p conj(A[k, p, a]) L[Q, k, g, p, r]  (Sec. 2.3, below Eq. kp_vhs)."""
    nk = L.shape[0]
    LH = np.empty(L.shape[:3] + (A.shape[2], L.shape[4]), dtype=np.complex128)
    for Q in range(nk):
        for k in range(nk):
            LH[Q, k] = np.einsum("pa,gpr->gar", A[k].conj(), L[Q, k])
    return LH


def mean_field_v0(L):
    """v0[k] = -1/2 sum_r v_{prrq} on the diagonal block k (Sec. 2.1, below Eq. hsq).

    With v_{pqrs} = sum_g L_{pr,g} L*_{sq,g} (Sec. 2.2) the sum over r gives
    -1/2 sum_{Q, g} L[Q, k, g] L[Q, k, g]^dag; momentum conservation keeps it
    block diagonal in k.
    """
    nk, M = L.shape[0], L.shape[3]
    v0 = np.zeros((nk, M, M), dtype=np.complex128)
    for Q in range(nk):
        for k in range(nk):
            for g in range(L.shape[2]):
                v0[k] -= 0.5 * L[Q, k, g] @ L[Q, k, g].conj().T
    return v0


def one_body_propagator(h, v0, dt):
    """exp(-dt/2 H1') per k with H1' = h + v0 (Sec. 2.1, Eq. propagator)."""
    return np.stack([scipy.linalg.expm(-0.5 * dt * (h[k] + v0[k])) for k in range(h.shape[0])])


class System:
    """Static data of one k-point Hamiltonian plus the quantities derived from it."""

    def __init__(self, grid, L, h, A, dt):
        self.grid = tuple(int(v) for v in grid)
        self.L = np.asarray(L, dtype=np.complex128)
        self.h = np.asarray(h, dtype=np.complex128)
        self.A = np.asarray(A, dtype=np.complex128)
        self.dt = float(dt)
        self.nk, self.nchol, self.M = self.L.shape[0], self.L.shape[2], self.L.shape[3]
        self.n = self.A.shape[2]
        self.NM, self.N = self.nk * self.M, self.nk * self.n
        self.kminus, self.minus = kgrid_tables(self.grid)
        self.LH = half_rotate(self.L, self.A)
        self.v0 = mean_field_v0(self.L)
        self.Ehalf = one_body_propagator(self.h, self.v0, self.dt)

    # block views -------------------------------------------------------
    def rows(self, k):
        return slice(k * self.n, (k + 1) * self.n)

    def cols(self, k):
        return slice(k * self.M, (k + 1) * self.M)

    def A_dense(self):
        Ad = np.zeros((self.NM, self.N), dtype=np.complex128)
        for k in range(self.nk):
            Ad[self.cols(k), self.rows(k)] = self.A[k]
        return Ad


# --------------------------------------------------------------------------
# Green's function (Sec. 2.2, Eqs. gf, gfhrot)
# --------------------------------------------------------------------------

def overlap(sys: System, phi):
    """S = A^dag phi (N x N, dense: the walker is not block diagonal in k)."""
    S = np.empty((sys.N, phi.shape[1]), dtype=np.complex128)
    for k in range(sys.nk):
        S[sys.rows(k)] = sys.A[k].conj().T @ phi[sys.cols(k)]
    return S


def log_det(S):
    """log det S as a complex number (LU with partial pivoting)."""
    sign, logabs = np.linalg.slogdet(S)
    return complex(logabs + 1j * np.angle(sign))


def green_half(sys: System, phi):
    """Half-rotated Green's function (phi (A^dag phi)^-1)^T (N x NM) and log det(A^dag phi)."""
    S = overlap(sys, phi)
    Gh = np.linalg.solve(S.T, phi.T)       # S^-T phi^T = (phi S^-1)^T
    return Gh, log_det(S)


# --------------------------------------------------------------------------
# Force bias (Sec. 2.2 Eq. fb; Sec. 2.3 Eq. kp_vbias)
# --------------------------------------------------------------------------

def cholesky_trace(sys: System, Ghs):
    """X[Q, g] = sum_s sum_k sum_{a, r} LH[Q, k, g, a, r] Gh_s[(k, a), (k - Q, r)]."""
    X = np.zeros((sys.nk, sys.nchol), dtype=np.complex128)
    for Gh in Ghs:
        for Q in range(sys.nk):
            for k in range(sys.nk):
                blk = Gh[sys.rows(k), sys.cols(sys.kminus[k, Q])]
                X[Q] += np.einsum("gar,ar->g", sys.LH[Q, k], blk)
    return X


def force_bias(sys: System, X):
    """xbar[+/-, Q, g] = -sqrt(dt) <v_{Q g +/-}> from X (reading 1 and 2)."""
    Xm = X[sys.minus]
    vplus = 0.5j * (X + Xm)
    vminus = -0.5 * (X - Xm)
    return -np.sqrt(sys.dt) * np.stack([vplus, vminus])


# --------------------------------------------------------------------------
# vHS and its exponential (Sec. 2.2 Eq. vhs and the Taylor series; Sec. 2.3 Eq. kp_vhs)
# --------------------------------------------------------------------------

def vhs_coefficients(sys: System, x, xbar):
    """y[Q, g] so that V = sqrt(dt) sum_{Q g} L^{Q g} y[Q, g] (reading 2)."""
    xt = x - xbar
    m = sys.minus
    return 0.5 * (1j * xt[0] - xt[1]) + 0.5 * (1j * xt[0][m] + xt[1][m])


def vhs(sys: System, x, xbar):
    """V[(k p), (k - Q r)] = sqrt(dt) sum_g L[Q, k, g, p, r] y[Q, g]  (NM x NM, dense in (k, k'))."""
    y = vhs_coefficients(sys, x, xbar)
    V = np.zeros((sys.NM, sys.NM), dtype=np.complex128)
    for Q in range(sys.nk):
        for k in range(sys.nk):
            V[sys.cols(k), sys.cols(sys.kminus[k, Q])] += np.sqrt(sys.dt) * np.einsum(
                "gpr,g->pr", sys.L[Q, k], y[Q])
    return V


def taylor_apply(V, phi, order):
    """sum_{j=0}^{order} V^j phi / j!  (the truncated series of Sec. 2.2)."""
    term = phi.copy()
    acc = phi.copy()
    for j in range(1, order + 1):
        term = V @ term / j
        acc = acc + term
    return acc


def one_body_apply(sys: System, phi):
    """exp(-dt/2 H1') phi, block diagonal in k."""
    out = np.empty_like(phi)
    for k in range(sys.nk):
        out[sys.cols(k)] = sys.Ehalf[k] @ phi[sys.cols(k)]
    return out


# --------------------------------------------------------------------------
# Walker step (Sec. 2.1, Eqs. propagator, iterate_imp and the hybrid weight)
# --------------------------------------------------------------------------

def hybrid_weight(w, logdet_old, logdet_new, x, xbar):
    """w |I| max(0, cos dtheta), I = ratio * exp(x.xbar - xbar.xbar/2), dtheta = arg ratio."""
    dlog = sum(logdet_new[s] - logdet_old[s] for s in range(2))
    logI = dlog + np.sum(x * xbar - 0.5 * xbar * xbar)
    return float(w * np.exp(logI.real) * max(0.0, np.cos(dlog.imag)))


def propagate_walker(sys: System, phi, x, w, taylor_order=6):
    """One hybrid step of one walker.  phi[s] (NM x N), x[+/-, Q, g] real.

    Returns (phi_new, w_new, logdet_new[2], xbar, logdet_old[2]).
    """
    Ghs, ld_old = zip(*[green_half(sys, phi[s]) for s in range(2)])
    xbar = force_bias(sys, cholesky_trace(sys, Ghs))
    V = vhs(sys, x, xbar)
    phi_new = np.empty_like(phi)
    for s in range(2):
        t = one_body_apply(sys, phi[s])
        t = taylor_apply(V, t, taylor_order)
        phi_new[s] = one_body_apply(sys, t)
    ld_new = [log_det(overlap(sys, phi_new[s])) for s in range(2)]
    w_new = hybrid_weight(w, ld_old, ld_new, x, xbar)
    return phi_new, w_new, np.array(ld_new), xbar, np.array(ld_old)


def orthonormalise(phi_s):
    """Householder QR of one spin block, with R_jj real positive; returns the Q factor."""
    Qm, R = np.linalg.qr(phi_s)
    d = np.diag(R)
    ph = d / np.abs(d)
    return Qm * ph[None, :]


# --------------------------------------------------------------------------
# Local energy (Sec. 2.2 Eq. local_energy; Sec. 2.3 Eq. kp_el; Sec. 3.2 steps 1-3)
# --------------------------------------------------------------------------

def one_body_energy(sys: System, Ghs):
    """E1 = sum_s sum_k sum_{a q} (A[k]^dag h[k])[a, q] Gh_s[(k a), (k q)]."""
    E1 = 0.0j
    for Gh in Ghs:
        for k in range(sys.nk):
            E1 += np.sum((sys.A[k].conj().T @ sys.h[k]) * Gh[sys.rows(k), sys.cols(k)])
    return complex(E1)


def coulomb_energy(sys: System, X):
    """EC = 1/2 sum_{Q g} X[Q, g] X[-Q, g]."""
    return complex(0.5 * np.sum(X * X[sys.minus]))


def exchange_energy(sys: System, Ghs, Qs=None):
    """EX = -1/2 sum_s sum_{Q k k'} sum_{g a b} T1[g, a, b] T2[g, b, a] with
    T1[g, a, b] = sum_r LH[Q, k, g, a, r] Gh_s[(k'-Q, b), (k-Q, r)] and
    T2[g, b, a] = sum_s LH[-Q, k'-Q, g, b, s] Gh_s[(k, a), (k', s)]  (Sec. 3.2 steps 2(a)-(c)).
    With Qs given, only the terms of those momentum transfers (a partial sum of EX)."""
    EX = 0.0j
    km, mq = sys.kminus, sys.minus
    Qlist = range(sys.nk) if Qs is None else Qs
    for Gh in Ghs:
        for Q in Qlist:
            for k in range(sys.nk):
                for kp in range(sys.nk):
                    T1 = np.einsum("gar,br->gab", sys.LH[Q, k],
                                   Gh[sys.rows(km[kp, Q]), sys.cols(km[k, Q])])
                    T2 = np.einsum("gbs,as->gba", sys.LH[mq[Q], km[kp, Q]],
                                   Gh[sys.rows(k), sys.cols(kp)])
                    EX += -0.5 * np.einsum("gab,gba->", T1, T2)
    return complex(EX)


def local_energy(sys: System, phi):
    """(E1, EC, EX) of one walker, complex (Sec. 2.2 Eq. local_energy; Sec. 2.3 Eq. kp_el):
    one_body_energy, coulomb_energy of the Cholesky trace X, exchange_energy."""
    Ghs = [green_half(sys, phi[s])[0] for s in range(2)]
    E1 = one_body_energy(sys, Ghs)
    EC = coulomb_energy(sys, cholesky_trace(sys, Ghs))
    EX = exchange_energy(sys, Ghs)
    return E1, EC, EX


# --------------------------------------------------------------------------
# Adjoint of the local energy (derived from Eq. kp_el; holomorphic in phi)
# --------------------------------------------------------------------------

def local_energy_grad(sys: System, phi, parts=(1.0, 1.0, 1.0), two_body=None):
    """Holomorphic derivatives of c1 E1 + c2 EC + c3 EX.

    Returns (dphi[s, NM, N], dh[k, M, M]) with dphi = d E / d phi and
    dh[k] = d E / d h[k] (entries of h treated as independent).

    Gamma_s = dE/dGh_s (N x NM):
      diagonal blocks (k, k)      += c1 A[k]^dag h[k]
      block (k, k - Q)            += c2 sum_g X[-Q, g] LH[Q, k, g]
      block (k' - Q, k - Q)[b, r] += -c3 sum_{g a} T2[g, b, a] LH[Q, k, g, a, r]
    and with S = A^dag phi_s, Theta = phi_s S^-1:
      dE/dphi_s = [S^-1 (Gamma_s - (Gamma_s Theta) A^dag)]^T
      dE/dh[k]  = c1 sum_s conj(A[k]) Gh_s[(k, .), (k, .)]
    two_body(sys, Gh, X, c2, c3, Gam) adds the Coulomb and exchange blocks (default
    gamma_two_body; a caller may pass one that sums the same blocks in another order).
    """
    c1, c2, c3 = parts
    two_body = gamma_two_body if two_body is None else two_body
    Ghs = [green_half(sys, phi[s])[0] for s in range(2)]
    X = cholesky_trace(sys, Ghs)
    Ad = sys.A_dense()
    dphi = np.empty_like(phi)
    dh = np.zeros_like(sys.h)
    for s, Gh in enumerate(Ghs):
        Gam = np.zeros_like(Gh)
        for k in range(sys.nk):
            Gam[sys.rows(k), sys.cols(k)] += c1 * (sys.A[k].conj().T @ sys.h[k])
            dh[k] += c1 * (sys.A[k].conj() @ Gh[sys.rows(k), sys.cols(k)])
        two_body(sys, Gh, X, c2, c3, Gam)
        S = overlap(sys, phi[s])
        Sinv = np.linalg.inv(S)
        Theta = phi[s] @ Sinv
        dphi[s] = (Sinv @ (Gam - (Gam @ Theta) @ Ad.conj().T)).T
    return dphi, dh


def gamma_two_body(sys: System, Gh, X, c2, c3, Gam, Qs=None):
    """Add to Gam (N x NM) the Coulomb and exchange parts of dE/dGh of one spin:
      block (k, k - Q)            += c2 sum_g X[-Q, g] LH[Q, k, g]
      block (k' - Q, k - Q)[b, r] += -c3 sum_{g a} T2[g, b, a] LH[Q, k, g, a, r]
    for every momentum transfer Q (or those in Qs: a partial sum), T2 as in exchange_energy."""
    km, mq = sys.kminus, sys.minus
    for Q in (range(sys.nk) if Qs is None else Qs):
        for k in range(sys.nk):
            Gam[sys.rows(k), sys.cols(km[k, Q])] += c2 * np.einsum(
                "g,gar->ar", X[mq[Q]], sys.LH[Q, k])
            for kp in range(sys.nk):
                T2 = np.einsum("gbs,as->gba", sys.LH[mq[Q], km[kp, Q]],
                               Gh[sys.rows(k), sys.cols(kp)])
                Gam[sys.rows(km[kp, Q]), sys.cols(km[k, Q])] += -c3 * np.einsum(
                    "gba,gar->br", T2, sys.LH[Q, k])
    return Gam


def local_energy_vjp(sys: System, phi, g, two_body=None):
    """PyTorch-convention backward: returns conj(dE/dphi) and conj(dE/dh) weighted by g[3].

    With g = dLoss/dconj(E) per part, dLoss/dconj(phi) = sum_part g_part conj(dE_part/dphi).
    """
    dphi, dh = local_energy_grad(sys, phi, parts=tuple(np.conj(g)), two_body=two_body)
    return dphi.conj(), dh.conj()
