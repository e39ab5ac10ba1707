"""Standard (dense) representation on the library (afqmc_dense_create) against the standard
oracle of Sec. 2.2, through the C ABI, on both paths.

Inputs and fields are in the standard layout; the handle takes the fields mapped onto its
Hermitian vectors (oracle.standard.kpoint_fields).  Bars as for the k-point systems: FP64
path 1e-10 normwise; mixed path walkers 1e-6, weights 1e-5, force bias 1e-6 normwise,
energies within 1e-5 Ha per part on near-trial walkers and max(1e-5, 2e-6 |E|) on random
walkers (the conditioning stress case), gradients within 1e-5 of the summed part norms.
"""
import numpy as np
import pytest

import gen
from oracle import afqmc_kp as ok
from oracle import standard as so

torch = pytest.importorskip("torch")
from gpu_util import dev, host, rel  # noqa: E402

pytestmark = pytest.mark.gpu

SPECS = {
    "real-M12": gen.DenseSpec(M=12, nocc=3, nchol=20, nwalkers=5, real=True, random_trial=True, seed=31),
    "complex-M10": gen.DenseSpec(M=10, nocc=2, nchol=8, nwalkers=4, real=False, random_trial=True, seed=32),
    # more walker-spins than one row tile, ragged column tiles
    "complex-M20-many": gen.DenseSpec(M=20, nocc=5, nchol=14, nwalkers=70, real=False, seed=33),
}
BARS = {"fp64": dict(phi=1e-10, w=1e-10, e_abs=1e-10, e_rel=1e-10, xbar=1e-10),
        "mixed": dict(phi=1e-6, w=1e-5, e_abs=1e-5, e_rel=2e-6, xbar=1e-6)}


def make_dense(spec, precision):
    from paper_2003_09468_gb300 import DenseAFQMC
    L, h, A = gen.dense_cholesky(spec), gen.dense_one_body(spec), gen.dense_trial(spec)
    sys_ = DenseAFQMC(L, h, A, spec.nwalkers, spec.dt, precision=precision, hermitian=spec.real)
    return sys_, so.StandardSystem(L, h, A, spec.dt)


def energy_ok(got, ref, bar):
    err = np.abs(got - ref).max(axis=0)
    allowed = np.maximum(bar["e_abs"], bar["e_rel"] * np.abs(ref).max(axis=0))
    return bool(np.all(err < allowed)), err, allowed


@pytest.mark.parametrize("walkers", ["near_trial", "random"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(SPECS))
def test_step_force_bias_and_energy(name, prec, walkers):
    spec = SPECS[name]
    bar = dict(BARS[prec])
    if walkers == "near_trial" and prec == "mixed":
        bar["e_rel"] = 0.0
    sys_, osys = make_dense(spec, prec)
    assert sys_.field_shape == (spec.nwalkers, 2, 1, spec.nchol * (1 if spec.real else 2))
    phis = gen.dense_near_trial_walkers(spec) if walkers == "near_trial" else gen.dense_walkers(spec)
    # force bias, in the handle's layout
    xb = host(sys_.force_bias(dev(phis)))
    ref_xb = []
    for i in range(spec.nwalkers):
        r = so.force_bias(osys, [so.green_half(osys, phis[i][sp])[0] for sp in range(2)])
        ref_xb.append(so.kpoint_fields(r.real[None], spec.real)[0] + 1j * so.kpoint_fields(r.imag[None], spec.real)[0])
    assert rel(xb, np.array(ref_xb)) < bar["xbar"]
    # one step: walkers, weights and the new walkers' energies
    x = gen.dense_fields(spec, 0)
    w0 = np.linspace(0.7, 1.3, spec.nwalkers)
    phi, w = dev(phis), dev(w0)
    e = host(sys_.step(phi, dev(so.kpoint_fields(x, spec.real)), w, reuse=False))
    got_phi, got_w = host(phi), host(w)
    ref = [so.propagate_walker(osys, phis[i], x[i], w0[i]) for i in range(spec.nwalkers)]
    assert rel(got_phi, np.array([r[0] for r in ref])) < bar["phi"]
    assert rel(got_w, np.array([r[1] for r in ref])) < bar["w"]
    ref_e = np.array([so.local_energy(osys, got_phi[i]) for i in range(spec.nwalkers)])
    ok_, err, allowed = energy_ok(e, ref_e, bar)
    assert ok_, (err, allowed)
    assert sys_.last_error() == (0, 0)
    sys_.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint(prec):
    spec = SPECS["complex-M10"]
    sys_, osys = make_dense(spec, prec)
    ks = ok.System((1, 1, 1), so.hermitian_vectors(osys.L, spec.real)[None, None], osys.h[None], osys.A[None], spec.dt)
    phis = gen.dense_walkers(spec)
    g = gen.upstream(gen.SMALL_2x2x2, spec.nwalkers, seed_offset=7)
    gphi, gh1 = sys_.local_energy_backward(dev(phis), dev(g))
    full = np.array([ok.local_energy_vjp(ks, phis[w], g[w])[0] for w in range(spec.nwalkers)])
    parts = []
    for j in range(3):
        m = np.zeros(3)
        m[j] = 1.0
        parts.append(np.array([ok.local_energy_vjp(ks, phis[w], g[w] * m)[0] for w in range(spec.nwalkers)]))
    err = np.linalg.norm(host(gphi) - full) / sum(np.linalg.norm(p) for p in parts)
    assert err < (1e-10 if prec == "fp64" else 1e-5)
    ref_h1 = sum(ok.local_energy_vjp(ks, phis[w], g[w])[1] for w in range(spec.nwalkers))
    assert rel(host(gh1), ref_h1) < 1e-10
    sys_.close()


def test_dense_supercell_workload_sampled():
    """The two-cell Gamma-point workload (M = 52, N = 8, 416 real vectors, 64 walkers) on the
    tensor-core path: sampled walkers against the standard oracle, and a device-driven block."""
    spec = gen.DENSE_1x1x2
    sys_, osys = make_dense(spec, "mixed")
    phis = gen.dense_walkers(spec)
    x = gen.dense_fields(spec, 0)
    phi, w = dev(phis), dev(np.ones(spec.nwalkers))
    e = host(sys_.step(phi, dev(so.kpoint_fields(x, True)), w, reuse=False))
    got_phi, got_w = host(phi), host(w)
    for i in (0, spec.nwalkers - 1):
        pn, wn, _, _ = so.propagate_walker(osys, phis[i], x[i], 1.0)
        assert rel(got_phi[i], pn) < BARS["mixed"]["phi"]
        assert abs(got_w[i] - wn) <= BARS["mixed"]["w"] * abs(wn)   # a walker the phaseless cut kills is 0 on both sides
        ok_, err, allowed = energy_ok(e[i:i + 1], np.array([so.local_energy(osys, got_phi[i])]), BARS["mixed"])
        assert ok_, (i, err, allowed)
    xs = torch.empty(sys_.field_shape, dtype=torch.float64, device="cuda")
    eh = torch.empty((1, spec.nwalkers, 3), dtype=torch.complex128, device="cuda")
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    sys_.block(phi, w, xs, eh, counter, seed=5, nsteps=10, qr_period=5, energy_period=10)
    assert np.all(np.isfinite(host(eh))) and np.all(host(w) > 0)
    assert sys_.last_error() == (0, 0)
    sys_.close()
