"""Fock-space brute force for tiny systems (Jordan-Wigner, sparse 2^nso operators).

TEST INFRASTRUCTURE ONLY.  Builds second-quantised operators explicitly and
evaluates the definitions of Sec. 2.1-2.2 without any Green's-function algebra:
the Hamiltonian of Eq. hamil, the mixed expectation <psi_T|O|phi>/<psi_T|phi>,
and exponentials of one-body operators.  The spin-orbital index is P + s * NM
for spatial orbital P and spin s.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def annihilators(nso):
    """Sparse Jordan-Wigner annihilation operators c_j (2^nso x 2^nso, CSR)."""
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    I2 = sp.identity(2, format="csr")
    ops = []
    for j in range(nso):
        m = sp.csr_matrix(np.array([[1.0]]))
        for i in range(nso):
            m = sp.kron(m, Z if i < j else (a if i == j else I2), format="csr")
        ops.append(m.astype(np.complex128))
    return ops


class FockSpace:
    def __init__(self, NM):
        self.NM = NM
        self.nso = 2 * NM
        self.c = annihilators(self.nso)
        self.cd = [m.T.tocsr() for m in self.c]
        self.dim = 2 ** self.nso

    def so(self, P, s):
        return P + s * self.NM

    def zero(self):
        return sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)

    def one_body(self, O, spins=(0, 1)):
        """sum_{PR s} O_{PR} c+_{P s} c_{R s}."""
        out = self.zero()
        for s in spins:
            for P in range(self.NM):
                for R in range(self.NM):
                    if O[P, R] != 0:
                        out = out + O[P, R] * (self.cd[self.so(P, s)] @ self.c[self.so(R, s)])
        return out.tocsr()

    def two_body(self, v, tol=0.0):
        """1/2 sum_{PQRS s s'} v_{PQRS} c+_{P s} c+_{Q s'} c_{S s'} c_{R s}  (Eq. hamil)."""
        out = self.zero()
        NM = self.NM
        for P, Q, R, S in itertools.product(range(NM), repeat=4):
            if abs(v[P, Q, R, S]) <= tol:
                continue
            for a in range(2):
                for b in range(2):
                    out = out + 0.5 * v[P, Q, R, S] * (
                        self.cd[self.so(P, a)] @ self.cd[self.so(Q, b)]
                        @ self.c[self.so(S, b)] @ self.c[self.so(R, a)])
        return out.tocsr()

    def slater(self, orbitals):
        """prod_s prod_a (sum_P orb_s[P, a] c+_{P s}) |0>."""
        st = np.zeros(self.dim, dtype=np.complex128)
        st[0] = 1.0
        for s, mat in enumerate(orbitals):
            for a in range(mat.shape[1]):
                op = self.zero()
                for P in range(self.NM):
                    op = op + mat[P, a] * self.cd[self.so(P, s)]
                st = op @ st
        return st

    @staticmethod
    def mixed(bra, op, ket):
        return complex((bra.conj() @ (op @ ket)) / (bra.conj() @ ket))

    @staticmethod
    def expm_apply(op, vec):
        return spla.expm_multiply(op.tocsc(), vec)
