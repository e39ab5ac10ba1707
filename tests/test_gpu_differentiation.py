"""The differentiation workload: the 3x3x3 grid, M = 26, n = 4, 208 vectors per Q, 64 walkers,
the local-energy adjoint with respect to the walker orbitals and to a Hermitian one-body
perturbation lambda V1 (V1[k] Hermitised complex N(0, 0.01)), on both paths, against the
oracle's gradient and against central finite differences.

With upstream g = (g1, g2, g3) on walker 0 only, the library returns
  grad_phi = sum_part g_part conj(dE_part/dphi)  and  grad_h1 = g1 conj(dE1/dh),
so d(E1)/d lambda = sum_k sum_pq conj(grad_h1[k][p][q]) V1[k][p][q] / conj(g1) (E1 is the only
part that depends on h, and linearly).  Bars: the oracle's gradient 1e-10 (FP64) and 1e-5 of ||dE/dphi|| (mixed);
d lambda against the oracle 1e-10 on both paths (the h-gradient comes from the double-float
Green's function on the mixed path); central differences of the FP64 path at h = 1e-5 along a
random complex direction of walker 0 within 1e-5 relative, and in lambda (E1 is linear in h:
the difference quotient is exact up to rounding) within 1e-6 at lambda = 1e-5 and 1e-10 at
lambda = 0.5.
"""
import numpy as np
import pytest

import gen
from oracle import afqmc_kp as ok

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make, rel  # noqa: E402

pytestmark = pytest.mark.gpu

SPEC = gen.DIAMOND_3x3x3


@pytest.fixture(scope="module")
def setup():
    phis = gen.near_trial_walkers(SPEC)
    V1 = gen.perturbation(SPEC)
    g = np.zeros((SPEC.nwalkers, 3), dtype=np.complex128)
    g[0] = gen.upstream(SPEC)[0]
    osys = ok.System(SPEC.grid, gen.cholesky(SPEC), gen.one_body(SPEC), gen.trial(SPEC), SPEC.dt)
    ref_phi, ref_h = ok.local_energy_vjp(osys, phis[0], g[0])
    ref_dlam = np.sum(ref_h.conj() * V1) / np.conj(g[0][0])
    return phis, V1, g, ref_phi, ref_dlam


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_against_oracle(setup, prec):
    phis, V1, g, ref_phi, ref_dlam = setup
    sys_, _ = make(SPEC, prec)
    gphi, gh1 = sys_.local_energy_backward(dev(phis), dev(g))
    got_phi, got_h = host(gphi), host(gh1)
    assert np.abs(got_phi[1:]).max() == 0.0
    bar = 1e-10 if prec == "fp64" else 1e-5
    assert rel(got_phi[0], ref_phi) < bar
    dlam = np.sum(got_h.conj() * V1) / np.conj(g[0][0])
    assert abs(dlam - ref_dlam) < 1e-10 * abs(ref_dlam), (dlam, ref_dlam)
    assert sys_.last_error() == (0, 0)
    sys_.close()


def test_fp64_adjoint_against_finite_differences(setup):
    phis, V1, g, _, _ = setup
    sys_, _ = make(SPEC, "fp64")
    gphi, gh1 = sys_.local_energy_backward(dev(phis), dev(g))
    got_phi, got_h = host(gphi)[0], host(gh1)
    c = g[0]

    def loss(p, hh=None):
        if hh is not None:
            sys_.set_one_body(dev(hh))
        e = host(sys_.local_energy(dev(p)))[0]
        return float((np.conj(c) * e).real.sum())   # L = Re sum conj(g) E: dL/dconj(phi) = grad_phi

    # along a random complex direction of walker 0
    rng = np.random.default_rng(17)
    d = rng.standard_normal(phis[0].shape) + 1j * rng.standard_normal(phis[0].shape)
    h = 1e-5
    pp, pm = phis.copy(), phis.copy()
    pp[0] += h * d
    pm[0] -= h * d
    fd = (loss(pp) - loss(pm)) / (2 * h)
    an = float((np.conj(got_phi) * d).real.sum())
    assert abs(fd - an) < 1e-5 * abs(an), (fd, an)
    # in lambda: E1 is linear in h, so the central difference is exact up to rounding; at
    # lambda = 1e-5 the FP64 rounding of E1 (~50 Ha, ~1e-13 absolute) over 2e-5 bounds it to
    # ~1e-8 absolute (3e-7 of the derivative), at lambda = 0.5 to ~1e-13
    h1 = gen.one_body(SPEC)
    an_lam = np.sum(got_h.conj() * V1) / np.conj(c[0])
    for lam, bar in ((1e-5, 1e-6), (0.5, 1e-10)):
        e_p = host(_energy_with(sys_, phis, h1 + lam * V1))[0][0]
        e_m = host(_energy_with(sys_, phis, h1 - lam * V1))[0][0]
        fd_lam = (e_p - e_m) / (2 * lam)
        assert abs(fd_lam - an_lam) < bar * abs(an_lam), (lam, fd_lam, an_lam)
    sys_.close()


def _energy_with(sys_, phis, h1):
    sys_.set_one_body(dev(h1))
    return sys_.local_energy(dev(phis))
