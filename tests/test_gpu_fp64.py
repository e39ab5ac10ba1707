"""FP64 GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Bar: 1e-10 relative (normwise over the batch) on every output."""
import numpy as np
import pytest

import gen
from oracle import afqmc_kp as ok

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make, oracle_energy, oracle_xbar, rel, wrap_phase  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10

SPECS = {
    # 2x2x2 grid, 8 orbitals per k (identity and random trials)
    "2x2x2": gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16),
    "2x2x2-rtrial": gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=5, random_trial=True, seed=7),
    # ragged, non-cubic grid with Q != -Q pairs and odd sizes (several GEMM tiles plus a tail)
    "3x1x2-ragged": gen.SystemSpec(grid=(3, 1, 2), M=7, nocc=3, nchol=11, nwalkers=3, random_trial=True, seed=3),
    # single k-point, single walker (standard representation special case)
    "1x1x1": gen.SystemSpec(grid=(1, 1, 1), M=5, nocc=2, nchol=4, nwalkers=1, random_trial=True, seed=5),
    # the largest orbital count per k-point and the largest nocc M the handle accepts
    "1x1x1-M128": gen.SystemSpec(grid=(1, 1, 1), M=128, nocc=8, nchol=16, nwalkers=2, random_trial=True, seed=6),
    # 3x3x3 grid with small bands (Q != -Q everywhere but Q = 0)
    "3x3x3-small": gen.SystemSpec(grid=(3, 3, 3), M=4, nocc=1, nchol=9, nwalkers=2, random_trial=True, seed=11),
}


@pytest.fixture(scope="module", params=list(SPECS))
def case(request):
    spec = SPECS[request.param]
    sys_, osys = make(spec, "fp64")
    yield spec, sys_, osys
    sys_.close()


def test_local_energy(case):
    spec, sys_, osys = case
    phis = gen.walkers(spec)
    e = host(sys_.local_energy(dev(phis)))
    ref = oracle_energy(osys, phis)
    for part in range(3):
        assert rel(e[:, part], ref[:, part]) < TOL, part


def test_force_bias(case):
    spec, sys_, osys = case
    phis = gen.walkers(spec)
    xb = host(sys_.force_bias(dev(phis)))
    ref = np.array([oracle_xbar(osys, p) for p in phis])
    assert rel(xb, ref) < TOL


@pytest.mark.parametrize("do_qr", [False, True])
def test_propagate(case, do_qr):
    spec, sys_, osys = case
    phis = gen.walkers(spec)
    x = gen.fields(spec, 3)
    w0 = np.linspace(0.5, 1.5, spec.nwalkers)
    phi, w = dev(phis), dev(w0)
    ld = torch.empty((spec.nwalkers, 2), dtype=torch.complex128, device="cuda")
    sys_.propagate(phi, dev(x), w, logdet=ld, do_qr=do_qr)
    phi_g, w_g, ld_g = host(phi), host(w), host(ld)
    ref_phi, ref_w, ref_ld = [], [], []
    for i in range(spec.nwalkers):
        pn, wn, ldn, _, _ = ok.propagate_walker(osys, phis[i], x[i], w0[i])
        if do_qr:
            pn = np.stack([ok.orthonormalise(pn[s]) for s in range(2)])
            ldn = np.array([ok.log_det(ok.overlap(osys, pn[s])) for s in range(2)])
        ref_phi.append(pn)
        ref_w.append(wn)
        ref_ld.append(ldn)
    ref_phi, ref_w, ref_ld = np.array(ref_phi), np.array(ref_w), np.array(ref_ld)
    assert rel(phi_g, ref_phi) < TOL
    assert rel(w_g, ref_w) < TOL
    assert rel(ld_g.real, ref_ld.real) < TOL
    assert np.abs(wrap_phase(ld_g.imag - ref_ld.imag)).max() < 1e-9


def test_orthonormalise(case):
    spec, sys_, osys = case
    rng = np.random.default_rng(4)
    phis = gen.walkers(spec)
    mix = rng.standard_normal((spec.N, spec.N)) + 1j * rng.standard_normal((spec.N, spec.N))
    phis = phis @ (np.eye(spec.N) + 0.3 * mix)
    phi = dev(phis)
    sys_.orthonormalise(phi)
    ref = np.array([[ok.orthonormalise(p[s]) for s in range(2)] for p in phis])
    assert rel(host(phi), ref) < TOL


def test_backward(case):
    spec, sys_, osys = case
    phis = gen.walkers(spec)
    g = gen.upstream(spec)
    gphi, gh1 = sys_.local_energy_backward(dev(phis), dev(g))
    gphi, gh1 = host(gphi), host(gh1)
    ref_phi = np.array([ok.local_energy_vjp(osys, phis[w], g[w])[0] for w in range(spec.nwalkers)])
    ref_h1 = sum(ok.local_energy_vjp(osys, phis[w], g[w])[1] for w in range(spec.nwalkers))
    # dE1/dh has only the E1 part, weighted by g[w][0]
    ref_h1_only = sum(ok.local_energy_vjp(osys, phis[w], np.array([g[w][0], 0, 0]))[1]
                      for w in range(spec.nwalkers))
    assert rel(ref_h1, ref_h1_only) < 1e-14
    assert rel(gphi, ref_phi) < TOL
    assert rel(gh1, ref_h1) < TOL


def test_singular_walker_gets_zero_weight():
    spec = SPECS["2x2x2-rtrial"]
    sys_, osys = make(spec, "fp64")
    phis = gen.walkers(spec)
    phis[1, 0][:, 0] = 0.0          # walker 1, spin up: a zero column makes A^dag phi singular
    w = dev(np.ones(spec.nwalkers))
    sys_.propagate(dev(phis), dev(gen.fields(spec, 0)), w)
    status, nsing = sys_.last_error()
    wg = host(w)
    assert status == 4 and nsing >= 1
    assert wg[1] == 0.0 and np.all(np.isfinite(wg)) and np.all(wg[[0, 2, 3, 4]] > 0)
    assert sys_.last_error() == (0, 0)   # flags are cleared by the read
    sys_.close()


def test_full_size_sampled_energy():
    """3x3x3, M=26, n=4, nchol=208, 64 walkers (the diamond-sized workload), FP64:
    two sampled walkers against the oracle, and the batch is finite."""
    spec = gen.DIAMOND_3x3x3
    sys_, osys = make(spec, "fp64")
    phis = gen.walkers(spec)
    e = host(sys_.local_energy(dev(phis)))
    assert np.all(np.isfinite(e))
    for w in (0, spec.nwalkers - 1):
        ref = np.array(ok.local_energy(osys, phis[w]))
        assert rel(e[w], ref) < TOL
    sys_.close()
