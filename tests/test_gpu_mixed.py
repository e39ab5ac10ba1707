"""Tensor-core (mixed) path vs the FP64 CPU oracle, through the C ABI.

Two walker sets per system (both seeded, both from the input recipe):
  near-trial  orthonormalised trial + small noise, the walkers a projection carries
              (Sec. 2.1 starts from the trial): the task's bars, absolute;
  random      orthonormalised complex Gaussians far from the trial (cond(A^dag phi) up
              to ~50 on the small systems): a conditioning stress case with the bars
              derived below.

Bars on near-trial walkers (the task's):
  force bias      normwise relative 1e-6
  E_L             every part within 1e-5 Ha per cell, max_w |E_gpu - E_ref| / Nk
  propagated phi  normwise relative 1e-6
  weights         relative 1e-5; log det 1e-5 absolute (real part)
  dE/dphi         normwise relative 1e-5 against the oracle's dE/dphi itself
  dE/dh           1e-10 (the FP64-class double-float Green's function)
Bars on random walkers (stress):
  E_L             the FP32-class relative error 2e-6 of each part, or 1e-5 Ha per cell,
                  whichever is larger (these walkers carry 20-60 Ha per cell)
  dE/dphi         1e-5 of the sum of the norms of the three parts' gradients (E1, E_C,
                  E_X taken one at a time): the Coulomb and exchange gradients of such
                  walkers nearly cancel, so the total's norm hides the size of the
                  operands; both ratios are printed
  force bias, phi, weights as above
QR (both sets): Cholesky-QR2 against the Householder Q, normwise max(1e-6, 2e-7 cond(phi))
(the QR with diag(R) > 0 is unique, so an orthonormal-to-u result differs by ~u cond),
and orthonormal to 1e-6.
"""
import numpy as np
import pytest

import gen
from oracle import afqmc_kp as ok

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make, oracle_energy, oracle_xbar, rel  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_XBAR = 1e-6
TOL_E_PER_CELL = 1e-5
TOL_PHI = 1e-6
TOL_W = 1e-5

SPECS = {
    "2x2x2": gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16),
    "2x2x2-rtrial": gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=5, random_trial=True, seed=7),
    "3x1x2-ragged": gen.SystemSpec(grid=(3, 1, 2), M=7, nocc=3, nchol=11, nwalkers=3, random_trial=True, seed=3),
    "1x1x1": gen.SystemSpec(grid=(1, 1, 1), M=5, nocc=2, nchol=4, nwalkers=1, random_trial=True, seed=5),
    # the largest orbital count per k-point and the largest nocc M the handle accepts
    "1x1x1-M128": gen.SystemSpec(grid=(1, 1, 1), M=128, nocc=8, nchol=16, nwalkers=2, random_trial=True, seed=6),
    "3x3x3-small": gen.SystemSpec(grid=(3, 3, 3), M=4, nocc=1, nchol=9, nwalkers=2, random_trial=True, seed=11),
    # more than 128 walker-spins: two row tiles in every walker-batched GEMM
    "2x1x1-many-walkers": gen.SystemSpec(grid=(2, 1, 1), M=6, nocc=2, nchol=10, nwalkers=70, seed=2),
    # N = 128 occupied orbitals: the overlap inverse is too large for shared memory and
    # runs on its global-memory variant
    "2x2x2-N128": gen.SystemSpec(grid=(2, 2, 2), M=20, nocc=16, nchol=10, nwalkers=2, random_trial=True, seed=9),
    # N = 256 occupied orbitals, the count of the 4x4x4 workload: the global-memory overlap
    # inverse and the global-memory Cholesky of the QR
    "2x2x4-N256": gen.SystemSpec(grid=(2, 2, 4), M=20, nocc=16, nchol=6, nwalkers=2, random_trial=True, seed=12),
}


@pytest.fixture(scope="module", params=list(SPECS))
def case(request):
    spec = SPECS[request.param]
    sys_, osys = make(spec, "mixed")
    yield spec, sys_, osys
    sys_.close()


WALKER_SETS = {"near_trial": gen.near_trial_walkers, "random": gen.walkers}

TOL_E_REL = 2e-6


def energy_error_per_cell(e, ref, nk):
    return np.abs(e - ref).max(axis=0) / nk


def energy_bar_per_cell(ref, nk, walkers="random"):
    if walkers == "near_trial":
        return np.full(3, TOL_E_PER_CELL)
    return np.maximum(TOL_E_PER_CELL, TOL_E_REL * np.abs(ref).max(axis=0) / nk)


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_local_energy(case, walkers):
    spec, sys_, osys = case
    phis = WALKER_SETS[walkers](spec)
    e = host(sys_.local_energy(dev(phis)))
    ref = oracle_energy(osys, phis)
    err = energy_error_per_cell(e, ref, spec.nk)
    bar = energy_bar_per_cell(ref, spec.nk, walkers)
    assert np.all(err < bar), (err, bar)
    assert sys_.last_error() == (0, 0)


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_force_bias(case, walkers):
    spec, sys_, osys = case
    phis = WALKER_SETS[walkers](spec)
    xb = host(sys_.force_bias(dev(phis)))
    ref = np.array([oracle_xbar(osys, p) for p in phis])
    assert rel(xb, ref) < TOL_XBAR


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_propagate(case, walkers):
    spec, sys_, osys = case
    phis = WALKER_SETS[walkers](spec)
    x = gen.fields(spec, 1)
    w0 = np.linspace(0.5, 1.5, spec.nwalkers)
    phi, w = dev(phis), dev(w0)
    ld = torch.empty((spec.nwalkers, 2), dtype=torch.complex128, device="cuda")
    sys_.propagate(phi, dev(x), w, logdet=ld)
    phi_g, w_g, ld_g = host(phi), host(w), host(ld)
    ref = [ok.propagate_walker(osys, phis[i], x[i], w0[i]) for i in range(spec.nwalkers)]
    w_ref = np.array([r[1] for r in ref])
    assert rel(phi_g, np.array([r[0] for r in ref])) < TOL_PHI
    if walkers == "near_trial":
        # every walker's weight on its own (none is near the phaseless cut cos = 0)
        assert np.all(w_ref > 0)
        assert np.all(np.abs(w_g - w_ref) <= TOL_W * w_ref), np.abs(w_g - w_ref) / w_ref
    else:
        assert rel(w_g, w_ref) < TOL_W
    assert np.abs(ld_g.real - np.array([r[2] for r in ref]).real).max() < TOL_W
    assert sys_.last_error() == (0, 0)


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_orthonormalise(case, walkers):
    spec, sys_, osys = case
    rng = np.random.default_rng(4)
    phis = WALKER_SETS[walkers](spec)
    mix = rng.standard_normal((spec.N, spec.N)) + 1j * rng.standard_normal((spec.N, spec.N))
    phis = phis @ (np.eye(spec.N) + 0.3 * mix)
    phi = dev(phis)
    sys_.orthonormalise(phi)
    got = host(phi)
    ref = np.array([[ok.orthonormalise(p[s]) for s in range(2)] for p in phis])
    # CholeskyQR2 is orthonormal to the working precision u ~ 1e-7; by uniqueness of the QR
    # with diag(R) > 0 its Q then differs from the Householder Q by about u cond(phi)
    cond = max(np.linalg.cond(p[s]) for p in phis for s in range(2))
    assert rel(got, ref) < max(TOL_PHI, 2e-7 * cond), cond
    q = got.reshape(-1, spec.NM, spec.N)
    assert np.abs(np.einsum("bij,bik->bjk", q.conj(), q) - np.eye(spec.N)).max() < TOL_PHI


TOL_GRAD = 1e-5


def oracle_grads(osys, phis, g, walkers):
    """The oracle's dE/dphi for upstream g, and the same for each energy part alone."""
    full = np.array([ok.local_energy_vjp(osys, phis[w], g[w])[0] for w in walkers])
    parts = []
    for j in range(3):
        mask = np.zeros(3)
        mask[j] = 1.0
        parts.append(np.array([ok.local_energy_vjp(osys, phis[w], g[w] * mask)[0] for w in walkers]))
    return full, parts


def grad_errors(got, full, parts):
    """(error relative to ||dE/dphi||, error relative to the sum of the parts' norms)."""
    d = np.linalg.norm(got - full)
    return d / np.linalg.norm(full), d / sum(np.linalg.norm(p) for p in parts)


def check_grad(got, full, parts, walkers):
    own, summed = grad_errors(got, full, parts)
    print(f"dE/dphi error: {own:.3e} of ||dE/dphi||, {summed:.3e} of the sum of the parts' norms")
    if walkers == "near_trial":
        assert own < TOL_GRAD, (own, summed)
    else:
        assert summed < TOL_GRAD, (own, summed)


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_backward(case, walkers):
    spec, sys_, osys = case
    phis = WALKER_SETS[walkers](spec)
    g = gen.upstream(spec)
    gphi, gh1 = sys_.local_energy_backward(dev(phis), dev(g))
    idx = range(spec.nwalkers)
    full, parts = oracle_grads(osys, phis, g, idx)
    ref_h1 = sum(ok.local_energy_vjp(osys, phis[w], g[w])[1] for w in idx)
    check_grad(host(gphi), full, parts, walkers)
    assert rel(host(gh1), ref_h1) < 1e-10
    # the gradient of the total energy (every part weighted alike)
    ones = np.ones_like(g)
    gphi1, _ = sys_.local_energy_backward(dev(phis), dev(ones), want_h1=False)
    full1, parts1 = oracle_grads(osys, phis, ones, idx)
    check_grad(host(gphi1), full1, parts1, walkers)


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_backward_diamond_sampled(walkers):
    """The adjoint at the 3x3x3, M=26, n=4, nchol=208, 64-walker size: walker 0 against
    the oracle (the other walkers' upstream gradients are zero)."""
    spec = gen.DIAMOND_3x3x3
    sys_, osys = make(spec, "mixed")
    phis = WALKER_SETS[walkers](spec)
    g = np.zeros((spec.nwalkers, 3), dtype=np.complex128)
    g[0] = gen.upstream(spec)[0]
    gphi, _ = sys_.local_energy_backward(dev(phis), dev(g), want_h1=False)
    got = host(gphi)
    full, parts = oracle_grads(osys, phis, g, [0])
    check_grad(got[:1], full, parts, walkers)
    assert np.abs(got[1:]).max() == 0.0
    assert sys_.last_error() == (0, 0)
    sys_.close()


def test_energy_invariant_under_orbital_rotation(case):
    """E_L depends on phi only through its column space (Sec. 2.2): the GPU energies of phi
    and phi U agree with each other and with the oracle."""
    spec, sys_, osys = case
    rng = np.random.default_rng(8)
    phis = gen.near_trial_walkers(spec)
    U, _ = np.linalg.qr(rng.standard_normal((spec.N, spec.N)) + 1j * rng.standard_normal((spec.N, spec.N)))
    e0 = host(sys_.local_energy(dev(phis)))
    e1 = host(sys_.local_energy(dev(phis @ U)))
    ref = oracle_energy(osys, phis)
    assert np.all(energy_error_per_cell(e1, ref, spec.nk) < TOL_E_PER_CELL)
    assert np.all(energy_error_per_cell(e0, e1, spec.nk) < 2 * TOL_E_PER_CELL)


@pytest.mark.parametrize("walkers", list(WALKER_SETS))
def test_diamond_size_sampled(walkers):
    """3x3x3 grid, M=26, n=4, nchol=208, 64 walkers: the benchmark workload in the
    benchmark's launch configuration.  Sampled walkers against the oracle at the task's bars
    (the seeded random walkers meet them too; one step later they no longer can, see the
    trajectory tests)."""
    spec = gen.DIAMOND_3x3x3
    sys_, osys = make(spec, "mixed")
    phis = WALKER_SETS[walkers](spec)
    e = host(sys_.local_energy(dev(phis)))
    xb = host(sys_.force_bias(dev(phis)))
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(xb))
    for w in (0, spec.nwalkers - 1):
        ref = np.array(ok.local_energy(osys, phis[w]))
        assert np.all(np.abs(e[w] - ref) / spec.nk < TOL_E_PER_CELL), (w, e[w] - ref)
        assert rel(xb[w], oracle_xbar(osys, phis[w])) < TOL_XBAR
    x = gen.fields(spec, 0)
    phi, wt = dev(phis), dev(np.ones(spec.nwalkers))
    sys_.propagate(phi, dev(x), wt)
    phi_g, w_g = host(phi), host(wt)
    # random walkers: walker 5 (the overlap of a random walker after one step has cond ~ 7000,
    # and its weight moves by ~2e-5 under a 4e-8 relative change of the walker: walker 0's
    # weight is not determined to 1e-5 by any 22-bit arithmetic)
    for w in ((0, 5) if walkers == "near_trial" else (5,)):
        pn, wn, _, _, _ = ok.propagate_walker(osys, phis[w], x[w], 1.0)
        assert rel(phi_g[w], pn) < TOL_PHI, w
        assert abs(w_g[w] - wn) <= TOL_W * abs(wn), (w, abs(w_g[w] - wn) / abs(wn))
    assert sys_.last_error() == (0, 0)
    sys_.close()


def test_singular_walker_gets_zero_weight():
    spec = SPECS["2x2x2-rtrial"]
    sys_, _ = make(spec, "mixed")
    phis = gen.walkers(spec)
    phis[1, 0][:, 0] = 0.0          # walker 1, spin up: a zero column makes A^dag phi singular
    w = dev(np.ones(spec.nwalkers))
    sys_.propagate(dev(phis), dev(gen.fields(spec, 0)), w)
    status, nsing = sys_.last_error()
    wg = host(w)
    assert status == 4 and nsing >= 1
    assert wg[1] == 0.0 and np.all(np.isfinite(wg)) and np.all(wg[[0, 2, 3, 4]] > 0)
    assert sys_.last_error() == (0, 0)
    sys_.close()


def test_gemm_autotuning(case):
    """Every step GEMM was timed at create with both ring depths and runs the faster one (the
    policy default unless the other is more than 2% faster); the QR GEMMs keep their defaults."""
    spec, sys_, _ = case
    t = sys_.gemm_tuning()
    assert set(t) == set(sys_.GEMMS)
    for name, v in t.items():
        assert v["ring_depth"] in (2, 3), (name, v)
        if name in ("gram", "apply_r"):
            assert v["ms_2_stages"] == 0.0 and v["ms_3_stages"] == 0.0
            continue
        assert v["ms_2_stages"] > 0.0 and v["ms_3_stages"] > 0.0, (name, v)
        fast = 2 if v["ms_2_stages"] < v["ms_3_stages"] else 3
        if v["ring_depth"] != fast:   # the default kept within the 2% margin
            assert min(v["ms_2_stages"], v["ms_3_stages"]) >= 0.98 * max(v["ms_2_stages"], v["ms_3_stages"]) - 1e-9



def test_taylor_cta_pair_form():
    """The Taylor GEMM's CTA-pair form (256-row tiles over a cluster of two SMs, each staging half
    of the paired B operand) gives bit for bit the single form's walkers, weights and energies;
    the form chosen at create is the faster one (the single form unless the pair form is more
    than 2% faster), and the override is refused where the pair form does not exist."""
    from paper_2003_09468_gb300 import AfqmcError
    # N = 80 occupied orbitals per spin: R = 2N = 160 rows per walker, two row tiles
    spec = gen.SystemSpec(grid=(2, 2, 2), M=12, nocc=10, nchol=16, nwalkers=8, random_trial=True, seed=41)
    sys_, osys = make(spec, "mixed")
    chosen, ms_pair = sys_.gemm_form("taylor")
    t = sys_.gemm_tuning()["taylor"]
    assert ms_pair > 0.0 and t["ms_cta_pair"] == ms_pair and t["cta_pair"] == chosen
    single = t["ms_2_stages"] if t["ring_depth"] == 2 else t["ms_3_stages"]   # at the tuned depth
    assert chosen == (ms_pair < 0.98 * single)
    phi0 = gen.near_trial_walkers(spec)
    outs = []
    for pair in (False, True):
        sys_.set_gemm_form("taylor", pair)
        assert sys_.gemm_form("taylor")[0] == pair
        phi, w = dev(phi0), dev(np.linspace(0.8, 1.2, spec.nwalkers))
        el = torch.empty((spec.nwalkers, 3), dtype=torch.complex128, device="cuda")
        for s in range(3):
            sys_.step(phi, dev(gen.fields(spec, s)), w, el, do_qr=(s == 1), reuse=s > 0)
        outs.append((host(phi), host(w), host(el)))
        assert sys_.last_error() == (0, 0)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    pn, _, _, _, _ = ok.propagate_walker(osys, phi0[0], gen.fields(spec, 0)[0], 1.0)
    sys_.set_gemm_form("taylor", True)
    phi = dev(phi0)
    sys_.step(phi, dev(gen.fields(spec, 0)), dev(np.ones(spec.nwalkers)), reuse=False)
    assert rel(host(phi)[0], pn) < TOL_PHI
    with pytest.raises(AfqmcError):
        sys_.set_gemm_form("exchange", True)
    sys_.close()
    # one row tile per walker (2N = 8): no pair form
    small, _ = make(SPECS["2x2x2"], "mixed")
    assert small.gemm_form("taylor") == (False, 0.0)
    with pytest.raises(AfqmcError):
        small.set_gemm_form("taylor", True)
    small.close()
    fp64, _ = make(SPECS["2x2x2"], "fp64")
    assert fp64.gemm_form("taylor") == (False, 0.0)
    with pytest.raises(AfqmcError):
        fp64.set_gemm_form("taylor", True)
    fp64.close()
