"""FP64 CPU oracle for the standard (dense) representation of Sec. 2.2.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the product library never
calls it and shares no code with it.

Written on the standard representation's own terms, independently of the
k-point oracle: M orbitals, N occupied per spin, G Cholesky vectors L[g][p][r]
of any complex form with v_{pqrs} = sum_g L_{pr,g} conj(L_{sq,g}) (Sec. 2.2).

* Potentials: L_plus = (L + L^dag)/2, L_minus = (L - L^dag)/2 and, with the
  factor-of-i reading of the k-point oracle (reading 1 there), v_plus = i L_plus,
  v_minus = i (i L_minus) = -(L - L^dag)/2.
* Force bias from the half-rotated Green's function and Cholesky vectors:
  X_g = sum_{a r} LH[g, a, r] Gh[a, r] with LH = A^dag L_g, Xbar_g with
  LHbar = A^dag L_g^dag; <v_plus> = i (X + Xbar)/2, <v_minus> = -(X - Xbar)/2 and
  xbar = -sqrt(dt) <v> (Sec. 2.2, Eq. fb and the half-rotated form after it).
* vHS = sqrt(dt) sum_{g, +/-} (x - xbar) v (Eq. vhs); propagator
  E_half (sum_{j <= p} V^j / j!) E_half with E_half = exp(-dt/2 (h + v0)) and
  v0 = -1/2 sum_g L_g L_g^dag (Sec. 2.1, Eq. propagator).
* Local energy (Eq. local_energy): E1 = sum_s sum_{pq} h_{pq} G_s[p, q],
  E_C = 1/2 sum_g (sum_s X_s[g]) (sum_s Xbar_s[g]),
  E_X = -1/2 sum_s sum_{g a b} T_s[g, a, b] Tbar_s[g, b, a] with
  T[g, a, b] = sum_r LH[g, a, r] Gh[b, r], Tbar[g, b, a] = sum_s LHbar[g, b, s] Gh[a, s].
* Fields x[+/-][g] are real and independent per potential; the hybrid weight is the
  one of Sec. 2.1 (the k-point oracle's hybrid_weight restated here).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


class StandardSystem:
    """Static data of one standard-representation Hamiltonian and trial."""

    def __init__(self, L, h, A, dt):
        self.L = np.asarray(L, dtype=np.complex128)            # [G][M][M]
        self.h = np.asarray(h, dtype=np.complex128)            # [M][M]
        self.A = np.asarray(A, dtype=np.complex128)            # [M][N]
        self.dt = float(dt)
        self.G, self.M = self.L.shape[0], self.L.shape[1]
        self.N = self.A.shape[1]
        Ldag = self.L.conj().transpose(0, 2, 1)
        self.v_plus = 0.5j * (self.L + Ldag)
        self.v_minus = -0.5 * (self.L - Ldag)
        Ad = self.A.conj().T
        self.LH = np.einsum("ap,gpr->gar", Ad, self.L)          # A^dag L_g
        self.LHbar = np.einsum("ap,gpr->gar", Ad, Ldag)         # A^dag L_g^dag
        self.v0 = -0.5 * np.einsum("gpr,gqr->pq", self.L, self.L.conj())
        self.Ehalf = scipy.linalg.expm(-0.5 * self.dt * (self.h + self.v0))


def green_half(sys: StandardSystem, phi):
    """Gh = (phi (A^dag phi)^-1)^T (N x M) and log det(A^dag phi)."""
    S = sys.A.conj().T @ phi
    sign, logabs = np.linalg.slogdet(S)
    return np.linalg.solve(S.T, phi.T), complex(logabs + 1j * np.angle(sign))


def traces(sys: StandardSystem, Gh):
    """(X[g], Xbar[g]) of one spin's half-rotated Green's function."""
    return np.einsum("gar,ar->g", sys.LH, Gh), np.einsum("gar,ar->g", sys.LHbar, Gh)


def force_bias(sys: StandardSystem, Ghs):
    """xbar[+/-][g] = -sqrt(dt) <v_{g +/-}>, spins summed."""
    X = sum(traces(sys, Gh)[0] for Gh in Ghs)
    Xb = sum(traces(sys, Gh)[1] for Gh in Ghs)
    return -np.sqrt(sys.dt) * np.stack([0.5j * (X + Xb), -0.5 * (X - Xb)])


def vhs(sys: StandardSystem, x, xbar):
    xt = x - xbar
    return np.sqrt(sys.dt) * (np.einsum("g,gpr->pr", xt[0], sys.v_plus) + np.einsum("g,gpr->pr", xt[1], sys.v_minus))


def propagate_walker(sys: StandardSystem, phi, x, w, taylor_order=6):
    """One hybrid step: (phi_new, w_new, logdet_new[2], xbar)."""
    Ghs, ld_old = zip(*[green_half(sys, phi[s]) for s in range(2)])
    xbar = force_bias(sys, Ghs)
    V = vhs(sys, x, xbar)
    phi_new = np.empty_like(phi)
    for s in range(2):
        t = sys.Ehalf @ phi[s]
        term, acc = t.copy(), t.copy()
        for j in range(1, taylor_order + 1):
            term = V @ term / j
            acc = acc + term
        phi_new[s] = sys.Ehalf @ acc
    ld_new = [green_half(sys, phi_new[s])[1] for s in range(2)]
    dlog = sum(ld_new[s] - ld_old[s] for s in range(2))
    logI = dlog + np.sum(x * xbar - 0.5 * xbar * xbar)
    w_new = float(w * np.exp(logI.real) * max(0.0, np.cos(dlog.imag)))
    return phi_new, w_new, np.array(ld_new), xbar


def local_energy(sys: StandardSystem, phi):
    """(E1, EC, EX) of one walker from X, Xbar, T and Tbar."""
    Ghs = [green_half(sys, phi[s])[0] for s in range(2)]
    Ah = sys.A.conj().T @ sys.h
    E1 = sum(np.sum(Ah * Gh) for Gh in Ghs)
    X = sum(traces(sys, Gh)[0] for Gh in Ghs)
    Xb = sum(traces(sys, Gh)[1] for Gh in Ghs)
    EC = 0.5 * np.sum(X * Xb)
    EX = 0.0j
    for Gh in Ghs:
        T = np.einsum("gar,br->gab", sys.LH, Gh)
        Tb = np.einsum("gbs,as->gba", sys.LHbar, Gh)
        EX += -0.5 * np.einsum("gab,gba->", T, Tb)
    return complex(E1), complex(EC), complex(EX)


def hermitian_vectors(L, hermitian=False):
    """Hermitian Cholesky vectors that give the same two-body operator: L_g = A_g - i B_g
    with A_g = (L_g + L_g^dag)/2 and B_g = i (L_g - L_g^dag)/2; [A; B] (2G vectors), or A
    alone when every L_g is Hermitian."""
    L = np.asarray(L, dtype=np.complex128)
    Ldag = L.conj().transpose(0, 2, 1)
    A = 0.5 * (L + Ldag)
    if hermitian:
        return A
    return np.concatenate([A, 0.5j * (L - Ldag)])


def kpoint_fields(x, hermitian=False):
    """Standard fields x[W][+/-][G] in the layout [W][2][1][G'] of the Nk = 1 handle built from
    hermitian_vectors: plane 0 holds x_plus (and x_minus after it for general L); plane 1
    has no effect (the minus potential of a Hermitian vector is zero) and is set to zero."""
    x = np.asarray(x, dtype=np.float64)
    W, _, G = x.shape
    Gp = G if hermitian else 2 * G
    out = np.zeros((W, 2, 1, Gp))
    out[:, 0, 0, :G] = x[:, 0]
    if not hermitian:
        out[:, 0, 0, G:] = x[:, 1]
    return out
