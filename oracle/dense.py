"""Dense supercell forms of the AFQMC quantities (standard representation, Sec. 2.2).

TEST INFRASTRUCTURE ONLY (see ``afqmc_kp``).  These are the textbook,
representation-free definitions written out on full NM x NM matrices; the
k-blocked oracle must reproduce them exactly up to rounding.  They are only
usable for small systems (the ERI tensor has NM^4 entries).
"""
from __future__ import annotations

import numpy as np

from .afqmc_kp import kgrid_tables


def supercell_cholesky(L, grid):
    """L^{Q g} as dense NM x NM matrices: block (k, k - Q) = L[Q, k, g], all else zero (Sec. 2.3)."""
    nk, nchol, M = L.shape[0], L.shape[2], L.shape[3]
    kminus, _ = kgrid_tables(grid)
    Ld = np.zeros((nk, nchol, nk * M, nk * M), dtype=np.complex128)
    for Q in range(nk):
        for k in range(nk):
            kq = kminus[k, Q]
            Ld[Q, :, k * M:(k + 1) * M, kq * M:(kq + 1) * M] = L[Q, k]
    return Ld


def block_diag(blocks):
    """Dense block-diagonal matrix from a stack of equal blocks."""
    nb, r, c = blocks.shape
    out = np.zeros((nb * r, nb * c), dtype=np.complex128)
    for i in range(nb):
        out[i * r:(i + 1) * r, i * c:(i + 1) * c] = blocks[i]
    return out


def eri(Ld):
    """v_{PQRS} = sum_g L^g_{PR} conj(L^g_{SQ})  (Sec. 2.2, Cholesky form of Eq. four_ix)."""
    n = Ld.shape[-1]
    Lf = Ld.reshape(-1, n * n)                       # [g, (P R)]
    vPRSQ = (Lf.T @ Lf.conj()).reshape(n, n, n, n)   # [P, R, S, Q]
    return np.ascontiguousarray(vPRSQ.transpose(0, 3, 1, 2))


def green_full(Ad, phi):
    """G_{PR} = <c+_P c_R> = [A* (phi^T A*)^-1 phi^T]_{PR}  (Sec. 2.2, Eq. gf)."""
    return Ad.conj() @ np.linalg.inv(phi.T @ Ad.conj()) @ phi.T


def hs_potentials(Ld):
    """(v_plus, v_minus)[Q, g] = (i (L + L^dag)/2, -(L - L^dag)/2) as dense matrices."""
    Ldag = Ld.conj().swapaxes(-1, -2)
    return 0.5j * (Ld + Ldag), -0.5 * (Ld - Ldag)


def force_bias_dense(Ld, Gs, dt):
    """xbar[+/-, Q, g] = -sqrt(dt) sum_s Tr(v_{Q g +/-} G_s^T)  (Sec. 2.2, Eq. fb)."""
    vp, vm = hs_potentials(Ld)
    G = sum(Gs)
    return -np.sqrt(dt) * np.stack([np.einsum("qgPR,PR->qg", vp, G),
                                    np.einsum("qgPR,PR->qg", vm, G)])


def vhs_dense(Ld, x, xbar, dt):
    """V = sqrt(dt) sum_{Q g +/-} (x - xbar)_{+/- Q g} v_{Q g +/-}  (Sec. 2.2, Eq. vhs)."""
    vp, vm = hs_potentials(Ld)
    xt = x - xbar
    return np.sqrt(dt) * (np.einsum("qg,qgPR->PR", xt[0], vp) + np.einsum("qg,qgPR->PR", xt[1], vm))


def v0_dense(v):
    """v0_{pq} = -1/2 sum_r v_{prrq}  (Sec. 2.1, below Eq. hsq)."""
    return -0.5 * np.einsum("prrq->pq", v)


def local_energy_dense(H1, v, Gs):
    """(E1, EC, EX) from Eq. local_energy with the full ERI tensor."""
    E1 = sum(np.sum(H1 * G) for G in Gs)
    EC = 0.0j
    EX = 0.0j
    for a in range(2):
        for b in range(2):
            EC += 0.5 * np.einsum("pqrs,pr,qs->", v, Gs[a], Gs[b])
        EX -= 0.5 * np.einsum("pqrs,ps,qr->", v, Gs[a], Gs[a])
    return complex(E1), complex(EC), complex(EX)
