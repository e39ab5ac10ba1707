"""Pins of the FP64 oracle against things other than itself.

* Fock-space brute force (Jordan-Wigner) on tiny systems: the local energy, the
  force bias, the Hubbard-Stratonovich operator identity, the Thouless overlap
  and the whole propagator B(x - xbar) (Sec. 2.1, 2.2).
* Dense supercell definitions (standard representation, Sec. 2.2) against the
  k-blocked forms (Sec. 2.3) at the 2x2x2 size, plus momentum conservation.
* Library routines with error bounds (scipy expm for the Taylor series).
* Invariances, special cases, central finite differences for the adjoint and
  hand-constructed weight updates.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import gen
from oracle import afqmc_kp as ok
from oracle import dense, fock
from oracle_util import oracle_system, rel, tiny

FOCK_SPECS = {
    "1x1x2-identity-trial": tiny((1, 1, 2), M=2, nocc=1, nchol=3, random_trial=False),
    "1x1x2-random-trial": tiny((1, 1, 2), M=2, nocc=1, nchol=3, random_trial=True),
    "1x1x3-random-trial": tiny((1, 1, 3), M=2, nocc=1, nchol=2, random_trial=True, seed=4),
}


class FockCase:
    def __init__(self, spec):
        self.spec = spec
        self.sys = oracle_system(spec)
        s = self.sys
        self.Ld = dense.supercell_cholesky(s.L, s.grid)
        self.v = dense.eri(self.Ld)
        self.H1 = dense.block_diag(s.h)
        self.Ad = s.A_dense()
        self.phi = gen.walkers(spec, 1)[0]
        self.F = fock.FockSpace(s.NM)
        self.psiT = self.F.slater([self.Ad, self.Ad])
        self.ket = self.F.slater([self.phi[0], self.phi[1]])
        self.H2op = self.F.two_body(self.v, tol=1e-300)
        vp, vm = dense.hs_potentials(self.Ld)
        self.vhat = [(0, Q, g, self.F.one_body(vp[Q, g])) for Q in range(s.nk) for g in range(s.nchol)]
        self.vhat += [(1, Q, g, self.F.one_body(vm[Q, g])) for Q in range(s.nk) for g in range(s.nchol)]


@pytest.fixture(scope="module", params=list(FOCK_SPECS))
def fc(request):
    return FockCase(FOCK_SPECS[request.param])


def test_local_energy_matches_fock_space(fc):
    E1, EC, EX = ok.local_energy(fc.sys, fc.phi)
    e1 = fc.F.mixed(fc.psiT, fc.F.one_body(fc.H1), fc.ket)
    e2 = fc.F.mixed(fc.psiT, fc.H2op, fc.ket)
    assert abs(E1 - e1) < 1e-11 * max(1, abs(e1))
    assert abs((EC + EX) - e2) < 1e-11 * max(1, abs(e2))


def test_hs_operator_identity(fc):
    """H2 = v0 - 1/2 sum v^2 with the sign reading of the HS potentials (Eq. hsq)."""
    v0 = dense.v0_dense(fc.v)
    rhs = fc.F.one_body(v0)
    for _, _, _, op in fc.vhat:
        rhs = rhs - 0.5 * (op @ op)
    diff = (fc.H2op - rhs).tocoo()
    assert (np.abs(diff.data).max() if diff.nnz else 0.0) < 1e-13
    # k-blocked v0 of the oracle equals -1/2 sum_r v_prrq from the ERI
    assert np.abs(dense.block_diag(fc.sys.v0) - v0).max() < 1e-14


def test_force_bias_matches_fock_space(fc):
    Ghs = [ok.green_half(fc.sys, fc.phi[s])[0] for s in range(2)]
    xbar = ok.force_bias(fc.sys, ok.cholesky_trace(fc.sys, Ghs))
    for pm, Q, g, op in fc.vhat:
        ref = -np.sqrt(fc.sys.dt) * fc.F.mixed(fc.psiT, op, fc.ket)
        assert abs(xbar[pm, Q, g] - ref) < 1e-12


def test_green_function_matches_fock_space(fc):
    s = fc.sys
    for spin in range(2):
        Gh, _ = ok.green_half(s, fc.phi[spin])
        G = fc.Ad.conj() @ Gh
        for P in range(s.NM):
            for R in range(s.NM):
                op = fc.F.cd[fc.F.so(P, spin)] @ fc.F.c[fc.F.so(R, spin)]
                assert abs(G[P, R] - fc.F.mixed(fc.psiT, op, fc.ket)) < 1e-12


def test_thouless_and_vhs_orientation(fc):
    """<psiT| exp(sqrt(dt) xt.v) |phi> = prod_s det(A^dag e^V phi_s) with V from the k-blocked vHS."""
    s = fc.sys
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, s.nk, s.nchol))
    Ghs = [ok.green_half(s, fc.phi[sp])[0] for sp in range(2)]
    xbar = ok.force_bias(s, ok.cholesky_trace(s, Ghs))
    V = ok.vhs(s, x, xbar)
    assert np.abs(V - dense.vhs_dense(fc.Ld, x, xbar, s.dt)).max() < 1e-14
    xt = x - xbar
    op = fc.F.zero()
    for pm, Q, g, vop in fc.vhat:
        op = op + np.sqrt(s.dt) * xt[pm, Q, g] * vop
    lhs = fc.psiT.conj() @ fc.F.expm_apply(op, fc.ket)
    eV = scipy.linalg.expm(V)
    rhs = np.prod([np.linalg.det(fc.Ad.conj().T @ eV @ fc.phi[sp]) for sp in range(2)])
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_propagator_overlap_ratio_matches_fock_space(fc):
    """Whole B(x - xbar) incl. both one-body halves: ratio of overlaps vs Fock space."""
    s = fc.sys
    rng = np.random.default_rng(11)
    x = rng.standard_normal((2, s.nk, s.nchol))
    _, _, ld_new, xbar, ld_old = ok.propagate_walker(s, fc.phi, x, 1.0, taylor_order=40)
    ratio = np.exp(np.sum(ld_new - ld_old))
    H1p = fc.F.one_body(fc.H1 + dense.v0_dense(fc.v))
    xt = x - xbar
    op = fc.F.zero()
    for pm, Q, g, vop in fc.vhat:
        op = op + np.sqrt(s.dt) * xt[pm, Q, g] * vop
    st = fc.F.expm_apply(-0.5 * s.dt * H1p, fc.ket)
    st = fc.F.expm_apply(op, st)
    st = fc.F.expm_apply(-0.5 * s.dt * H1p, st)
    ref = (fc.psiT.conj() @ st) / (fc.psiT.conj() @ fc.ket)
    assert abs(ratio - ref) < 1e-11 * abs(ref)


# ---------------------------------------------------------------------------
# 2x2x2 size: dense supercell definitions vs k-blocked forms
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small():
    spec = gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=2, random_trial=True)
    s = oracle_system(spec)
    Ld = dense.supercell_cholesky(s.L, s.grid)
    return spec, s, Ld, dense.eri(Ld)


def test_kblocked_energy_matches_dense_eri(small):
    spec, s, Ld, v = small
    H1 = dense.block_diag(s.h)
    Ad = s.A_dense()
    for phi in gen.walkers(spec, 2):
        Gs = [dense.green_full(Ad, phi[sp]) for sp in range(2)]
        ref = dense.local_energy_dense(H1, v, Gs)
        got = ok.local_energy(s, phi)
        for a, b in zip(got, ref):
            assert abs(a - b) < 1e-11 * max(1.0, abs(b))


def test_momentum_conservation_and_time_reversal(small):
    spec, s, Ld, v = small
    kp = gen.kpoints(s.grid)
    kof = np.repeat(np.arange(s.nk), s.M)
    K = kp[kof]
    g = np.array(s.grid)
    # v_PQRS = 0 unless k_P - k_R + k_Q - k_S = 0 mod grid
    bad = ((K[:, None, None, None] - K[None, None, :, None] + K[None, :, None, None]
            - K[None, None, None, :]) % g).any(axis=-1)
    assert np.abs(v[bad]).max() == 0.0
    assert np.abs(v[~bad]).max() > 1e-3
    # L^{Q g dagger} = L^{-Q g}
    _, minus = ok.kgrid_tables(s.grid)
    for Q in range(s.nk):
        assert np.abs(Ld[Q].conj().swapaxes(-1, -2) - Ld[minus[Q]]).max() == 0.0


def test_force_bias_and_vhs_match_dense(small):
    spec, s, Ld, v = small
    Ad = s.A_dense()
    phi = gen.walkers(spec, 1)[0]
    Gs = [dense.green_full(Ad, phi[sp]) for sp in range(2)]
    Ghs = [ok.green_half(s, phi[sp])[0] for sp in range(2)]
    for sp in range(2):
        assert np.abs(Ad.conj() @ Ghs[sp] - Gs[sp]).max() < 1e-12
    xbar = ok.force_bias(s, ok.cholesky_trace(s, Ghs))
    assert rel(xbar, dense.force_bias_dense(Ld, Gs, s.dt)) < 1e-13
    x = gen.fields(spec, 0, 1)[0]
    assert rel(ok.vhs(s, x, xbar), dense.vhs_dense(Ld, x, xbar, s.dt)) < 1e-13
    assert np.abs(dense.block_diag(s.v0) - dense.v0_dense(v)).max() < 1e-13


def test_single_kpoint_reduces_to_standard_representation():
    spec = gen.SystemSpec(grid=(1, 1, 1), M=6, nocc=2, nchol=10, nwalkers=1, random_trial=True, seed=3)
    s = oracle_system(spec)
    Ld = dense.supercell_cholesky(s.L, s.grid)
    phi = gen.walkers(spec, 1)[0]
    Gs = [dense.green_full(s.A_dense(), phi[sp]) for sp in range(2)]
    ref = dense.local_energy_dense(dense.block_diag(s.h), dense.eri(Ld), Gs)
    for a, b in zip(ok.local_energy(s, phi), ref):
        assert abs(a - b) < 1e-12 * max(1.0, abs(b))


def test_taylor_series_vs_expm_bound(small):
    spec, s, Ld, v = small
    phi = gen.walkers(spec, 1)[0][0]
    x = gen.fields(spec, 0, 1)[0]
    xbar = np.zeros_like(x)
    V = ok.vhs(s, x, xbar)
    nV = np.linalg.norm(V, 2)
    E = scipy.linalg.expm(V) @ phi
    for p in (2, 4, 6):
        err = np.linalg.norm(ok.taylor_apply(V, phi, p) - E, 2)
        bound = nV ** (p + 1) * np.exp(nV) / math.factorial(p + 1)
        assert err <= bound * np.linalg.norm(phi, 2) * (1 + 1e-9)
        assert err > 1e-15   # truncated, not the exact exponential
    assert np.linalg.norm(ok.taylor_apply(V, phi, 30) - E) < 1e-13


def test_energy_and_force_bias_invariant_under_orbital_rotation(small):
    spec, s, Ld, v = small
    phi = gen.walkers(spec, 1)[0]
    rng = np.random.default_rng(2)
    U = rng.standard_normal((s.N, s.N)) + 1j * rng.standard_normal((s.N, s.N))
    phiU = np.stack([phi[0] @ U, phi[1] @ U.T])
    E0 = ok.local_energy(s, phi)
    E1 = ok.local_energy(s, phiU)
    for a, b in zip(E0, E1):
        assert abs(a - b) < 1e-10 * max(1.0, abs(b))
    phiQ = np.stack([ok.orthonormalise(phi[sp] @ U) for sp in range(2)])
    for a, b in zip(E0, ok.local_energy(s, phiQ)):
        assert abs(a - b) < 1e-10 * max(1.0, abs(b))
    X0 = ok.cholesky_trace(s, [ok.green_half(s, phi[sp])[0] for sp in range(2)])
    X1 = ok.cholesky_trace(s, [ok.green_half(s, phiU[sp])[0] for sp in range(2)])
    assert rel(X1, X0) < 1e-10


def test_trial_walker_special_case(small):
    """phi = psi_T: Hermitian G, so E_L is real and X_{-Q} = conj(X_Q)."""
    spec, s, Ld, v = small
    Ad = s.A_dense()
    phi = np.stack([Ad, Ad])
    E = ok.local_energy(s, phi)
    assert all(abs(e.imag) < 1e-12 for e in E)
    X = ok.cholesky_trace(s, [ok.green_half(s, phi[sp])[0] for sp in range(2)])
    assert np.abs(X[s.minus] - X.conj()).max() < 1e-13
    # textbook closed-shell energy from the density matrix P = A A^dag (per spin)
    P = Ad @ Ad.conj().T
    H1 = dense.block_diag(s.h)
    J = np.einsum("pqrs,qs->pr", v, P.T)     # Coulomb from both spins: 2 * J below
    K = np.einsum("pqrs,qr->ps", v, P.T)
    e_rhf = 2 * np.sum(H1 * P.T) + 0.5 * np.sum((2 * J) * (2 * P.T)) - np.sum(K * P.T)
    assert abs(sum(E) - e_rhf) < 1e-11 * abs(e_rhf)


def test_orthonormalise_is_unique_qr():
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((20, 6)) + 1j * rng.standard_normal((20, 6))
    Qm = ok.orthonormalise(Z)
    assert np.abs(Qm.conj().T @ Qm - np.eye(6)).max() < 1e-14
    R = Qm.conj().T @ Z
    assert np.abs(np.tril(R, -1)).max() < 1e-13
    assert np.all(np.abs(np.diag(R).imag) < 1e-13) and np.all(np.diag(R).real > 0)


# ---------------------------------------------------------------------------
# Adjoint: central finite differences
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def grad_case():
    spec = gen.SystemSpec(grid=(2, 2, 1), M=5, nocc=2, nchol=12, nwalkers=1, random_trial=True, seed=3)
    return spec, oracle_system(spec), gen.walkers(spec, 1)[0]


@pytest.mark.parametrize("part", [0, 1, 2])
def test_energy_adjoint_vs_finite_differences(grad_case, part):
    spec, s, phi = grad_case
    parts = [0.0, 0.0, 0.0]
    parts[part] = 1.0
    dphi, _ = ok.local_energy_grad(s, phi, parts=parts)
    rng = np.random.default_rng(9)
    h = 1e-5
    for spin in range(2):
        D = rng.standard_normal(phi[0].shape) + 1j * rng.standard_normal(phi[0].shape)
        for fac in (1.0, 1j):
            pp, pm = phi.copy(), phi.copy()
            pp[spin] += h * fac * D
            pm[spin] -= h * fac * D
            fd = (ok.local_energy(s, pp)[part] - ok.local_energy(s, pm)[part]) / (2 * h)
            an = np.sum(dphi[spin] * fac * D)
            assert abs(fd - an) < 1e-5 * abs(an)


def test_one_body_perturbation_response(grad_case):
    spec, s, phi = grad_case
    V1 = gen.perturbation(spec)
    _, dh = ok.local_energy_grad(s, phi)
    h = 1e-3
    sp = ok.System(s.grid, s.L, s.h + h * V1, s.A, s.dt)
    sm = ok.System(s.grid, s.L, s.h - h * V1, s.A, s.dt)
    fd = (sum(ok.local_energy(sp, phi)) - sum(ok.local_energy(sm, phi))) / (2 * h)
    an = np.sum(dh * V1)
    assert abs(fd - an) < 1e-8 * abs(an)


def test_vjp_convention(grad_case):
    """Real loss l = Re(c E): PyTorch grad wrt conj(phi) equals conj(c) conj(dE/dphi) / 2 * 2."""
    spec, s, phi = grad_case
    g = np.array([0.3 - 0.2j, 0.0, 1.1 + 0.4j])
    gphi, _ = ok.local_energy_vjp(s, phi, g)
    # directional check: d/dt l(phi + t D) for l = Re(sum_p conj(g_p) E_p) equals Re <gphi, D> * 2 / 2
    rng = np.random.default_rng(1)
    D = rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape)
    h = 1e-5
    loss = lambda p: float(np.real(np.sum(np.conj(g) * np.array(ok.local_energy(s, p)))))
    fd = (loss(phi + h * D) - loss(phi - h * D)) / (2 * h)
    an = float(np.real(np.sum(np.conj(gphi) * D)))
    assert abs(fd - an) < 1e-5 * abs(an)


# ---------------------------------------------------------------------------
# Hybrid weight update: hand-constructed cases
# ---------------------------------------------------------------------------

def test_hybrid_weight_cases():
    x = np.zeros((2, 1, 1))
    xbar = np.zeros((2, 1, 1), dtype=complex)
    eps = 1e-6
    old = [0.0j, 0.0j]
    # phase pi/2 - eps is kept (cos > 0), pi/2 + eps is killed
    assert ok.hybrid_weight(2.0, old, [1j * (np.pi / 2 - eps), 0.0j], x, xbar) > 0
    assert ok.hybrid_weight(2.0, old, [1j * (np.pi / 2 + eps), 0.0j], x, xbar) == 0.0
    # pure modulus change: w |ratio|
    assert abs(ok.hybrid_weight(1.5, old, [0.3, -0.1], x, xbar) - 1.5 * np.exp(0.2)) < 1e-15
    # phase split over the spins, 60 degrees in total: cos = 1/2
    w = ok.hybrid_weight(1.0, old, [1j * np.pi / 6, 1j * np.pi / 6], x, xbar)
    assert abs(w - 0.5) < 1e-15
    # force-bias factor exp(x xbar - xbar^2 / 2) enters only through its modulus
    x1 = np.array([[[1.0]], [[0.0]]])
    xb1 = np.array([[[0.5 + 0.25j]], [[0.0]]])
    expo = 1.0 * (0.5 + 0.25j) - 0.5 * (0.5 + 0.25j) ** 2
    assert abs(ok.hybrid_weight(1.0, old, [0.0j, 0.0j], x1, xb1) - np.exp(expo.real)) < 1e-15


def test_generator_time_reversal_blocks():
    spec = gen.SystemSpec(grid=(3, 1, 2), M=3, nocc=1, nchol=4, nwalkers=1)
    L = gen.cholesky(spec)
    kminus, minus = ok.kgrid_tables(spec.grid)
    for Q in range(spec.nk):
        for k in range(spec.nk):
            assert np.array_equal(L[minus[Q], kminus[k, Q]], L[Q, k].conj().transpose(0, 2, 1))
