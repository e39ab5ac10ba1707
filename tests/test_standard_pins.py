"""Pins of the standard-representation oracle (Sec. 2.2) against things other than itself.

* Fock-space brute force (Jordan-Wigner) on tiny systems, for real symmetric and for
  complex (adjoint-paired) Cholesky vectors: the local energy, the force bias, the operator
  identity H2 = v0 - 1/2 sum v^2, and the overlap ratio of the whole propagator.
* The X, Xbar, T, Tbar forms of the energy against the energy from the full ERI tensor.
* Reduction to the k-point oracle at Nk = 1: Hermitian vectors as they are, and general
  vectors through the Hermitian pair A_g = (L + L^dag)/2, B_g = i (L - L^dag)/2 with the
  fields mapped one to one (the layout the library's dense handles use).
"""
import numpy as np
import pytest
import scipy.linalg

import gen
from oracle import afqmc_kp as ok
from oracle import dense, fock
from oracle import standard as so

TINY = {
    "real-M3": gen.DenseSpec(M=3, nocc=1, nchol=4, nwalkers=1, real=True, random_trial=True, seed=1),
    "complex-M3": gen.DenseSpec(M=3, nocc=1, nchol=4, nwalkers=1, real=False, random_trial=True, seed=2),
    "complex-M4": gen.DenseSpec(M=4, nocc=2, nchol=2, nwalkers=1, real=False, random_trial=True, seed=3),
}


def system(spec):
    return so.StandardSystem(gen.dense_cholesky(spec), gen.dense_one_body(spec), gen.dense_trial(spec), spec.dt)


class Case:
    def __init__(self, spec):
        self.spec = spec
        self.sys = system(spec)
        s = self.sys
        self.phi = gen.dense_walkers(spec, 1)[0]
        self.v = dense.eri(s.L[None])                      # v_{pqrs} = sum_g L_{pr,g} conj(L_{sq,g})
        self.F = fock.FockSpace(s.M)
        self.psiT = self.F.slater([s.A, s.A])
        self.ket = self.F.slater([self.phi[0], self.phi[1]])
        self.H2 = self.F.two_body(self.v, tol=1e-300)
        self.vops = [[self.F.one_body(s.v_plus[g]) for g in range(s.G)],
                     [self.F.one_body(s.v_minus[g]) for g in range(s.G)]]


@pytest.fixture(scope="module", params=list(TINY))
def case(request):
    return Case(TINY[request.param])


def test_energy_matches_fock_space(case):
    s = case.sys
    E1, EC, EX = so.local_energy(s, case.phi)
    assert abs(E1 - case.F.mixed(case.psiT, case.F.one_body(s.h), case.ket)) < 1e-11
    e2 = case.F.mixed(case.psiT, case.H2, case.ket)
    assert abs(EC + EX - e2) < 1e-11 * max(1.0, abs(e2))


def test_force_bias_matches_fock_space(case):
    s = case.sys
    Ghs = [so.green_half(s, case.phi[sp])[0] for sp in range(2)]
    xbar = so.force_bias(s, Ghs)
    for pm in range(2):
        for g in range(s.G):
            ref = -np.sqrt(s.dt) * case.F.mixed(case.psiT, case.vops[pm][g], case.ket)
            assert abs(xbar[pm, g] - ref) < 1e-12


def test_hs_operator_identity(case):
    """H2 = v0 - 1/2 sum_{g, +/-} v^2 (adjoint-closed vector sets make the commutators cancel)."""
    s = case.sys
    rhs = case.F.one_body(s.v0)
    for pm in range(2):
        for op in case.vops[pm]:
            rhs = rhs - 0.5 * (op @ op)
    diff = (case.H2 - rhs).tocoo()
    assert (np.abs(diff.data).max() if diff.nnz else 0.0) < 1e-13


def test_propagator_overlap_ratio_matches_fock_space(case):
    s = case.sys
    x = np.random.default_rng(4).standard_normal((2, s.G))
    _, _, ld_new, xbar = so.propagate_walker(s, case.phi, x, 1.0, taylor_order=40)
    ld_old = np.array([so.green_half(s, case.phi[sp])[1] for sp in range(2)])
    ratio = np.exp(np.sum(ld_new - ld_old))
    H1p = case.F.one_body(s.h + s.v0)
    op = case.F.zero()
    for pm in range(2):
        for g in range(s.G):
            op = op + np.sqrt(s.dt) * (x[pm, g] - xbar[pm, g]) * case.vops[pm][g]
    st = case.F.expm_apply(-0.5 * s.dt * H1p, case.ket)
    st = case.F.expm_apply(op, st)
    st = case.F.expm_apply(-0.5 * s.dt * H1p, st)
    ref = (case.psiT.conj() @ st) / (case.psiT.conj() @ case.ket)
    assert abs(ratio - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("real", [True, False])
def test_energy_forms_match_eri(real):
    spec = gen.DenseSpec(M=10, nocc=3, nchol=12, nwalkers=2, real=real, random_trial=True, seed=5)
    s = system(spec)
    v = dense.eri(s.L[None])
    for phi in gen.dense_walkers(spec):
        Gs = [dense.green_full(s.A, phi[sp]) for sp in range(2)]
        ref = dense.local_energy_dense(s.h, v, Gs)
        got = so.local_energy(s, phi)
        for a, b in zip(got, ref):
            assert abs(a - b) < 1e-11 * max(1.0, abs(b))


def kpoint_system(s, hermitian):
    Lh = so.hermitian_vectors(s.L, hermitian=hermitian)
    return ok.System((1, 1, 1), Lh[None, None], s.h[None], s.A[None], s.dt)


@pytest.mark.parametrize("real", [True, False])
def test_reduces_to_kpoint_oracle_at_one_kpoint(real):
    """One step and the energy: the standard oracle with vectors L and fields x against the
    k-point oracle at Nk = 1 with the Hermitian vectors and the mapped fields."""
    spec = gen.DenseSpec(M=9, nocc=3, nchol=10, nwalkers=2, real=real, random_trial=True, seed=6)
    s = system(spec)
    ks = kpoint_system(s, hermitian=real)
    assert np.abs(ks.v0[0] - s.v0).max() < 1e-13
    xs = gen.dense_fields(spec, 0)
    xk = so.kpoint_fields(xs, hermitian=real)
    for w, phi in enumerate(gen.dense_walkers(spec)):
        p1, w1, ld1, xb1 = so.propagate_walker(s, phi, xs[w], 0.8)
        p2, w2, ld2, xb2, _ = ok.propagate_walker(ks, phi, xk[w], 0.8)
        assert np.abs(p1 - p2).max() < 1e-12
        assert abs(w1 - w2) < 1e-12
        assert np.abs(ld1 - ld2).max() < 1e-12
        assert np.abs(so.kpoint_fields(xb1.real[None], real)[0] + 1j * so.kpoint_fields(xb1.imag[None], real)[0]
                      - xb2).max() < 1e-13
        e1, e2 = so.local_energy(s, phi), ok.local_energy(ks, phi)
        assert np.abs(np.array(e1) - np.array(e2)).max() < 1e-11


def test_taylor_step_approaches_expm():
    spec = TINY["complex-M4"]
    s = system(spec)
    phi = gen.dense_walkers(spec, 1)[0]
    x = np.random.default_rng(9).standard_normal((2, s.G))
    Ghs = [so.green_half(s, phi[sp])[0] for sp in range(2)]
    V = so.vhs(s, x, so.force_bias(s, Ghs))
    exact = s.Ehalf @ scipy.linalg.expm(V) @ s.Ehalf @ phi[0]
    p6 = so.propagate_walker(s, phi, x, 1.0, taylor_order=6)[0][0]
    nv = np.linalg.norm(V, 2)
    bound = nv ** 7 / 5040 * np.exp(nv) * np.linalg.norm(s.Ehalf, 2) ** 2 * np.linalg.norm(phi[0], 2)
    assert np.linalg.norm(p6 - exact, 2) <= bound * (1 + 1e-6) + 1e-14
