"""The largest workload: 4x4x4 grid (Nk = 64), M = 52 orbitals per k, n = 4, 416 Cholesky
vectors per Q, 256 walkers, mixed path, in the launch configuration of the benchmark
(`bench.py --workload diamond-4x4x4`).

The handle holds ~270 GB of device memory (the split Cholesky vectors, the precontracted
exchange tensor of all 262 144 triples, the walker workspace), so this test needs the whole
GPU.  The oracle follows walker 0 at the task's bars:
  the seeded walker's force bias (1e-6 normwise) and E1, E_C, E_X (1e-5 Ha per cell);
  after one fused step, the walker (1e-6), its weight (1e-5 relative), its log det (1e-5,
  against the oracle's log det of the GPU's walker) and E1, E_C, E_X (1e-5 Ha per cell);
  the adjoint of the seeded walker's local energy (dE/dphi within 1e-5 of ||dE/dphi||, dE/dh
  within 1e-10).
The oracle's exchange sum of one walker at this size (2 x 64^3 terms) and the exchange blocks of
its gradient are split over Q across spawned processes, each running the oracle's own
functions on its momentum transfers.
"""
import gc
import os
import sys

import numpy as np
import pytest

import gen
from oracle import afqmc_kp as ok

torch = pytest.importorskip("torch")
from gpu_util import dev, host, rel  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL_E, TOL_XBAR, TOL_PHI, TOL_W, TOL_LD = 1e-5, 1e-6, 1e-6, 1e-5, 1e-5


def test_diamond_4x4x4_sampled():
    sys.path.insert(0, ROOT)
    import bench   # the benchmark's oracle helpers: the pooled exchange sum
    from paper_2003_09468_gb300 import KPointAFQMC
    spec = gen.DIAMOND_4x4x4
    gc.collect()
    torch.cuda.empty_cache()
    L, h1, A = gen.cholesky(spec), gen.one_body(spec), gen.trial(spec)
    sys_ = KPointAFQMC(spec.grid, L, h1, A, spec.nwalkers, spec.dt, precision="mixed")
    assert sys_.memory_bytes() < 285e9
    phis = gen.near_trial_walkers(spec)
    phi = dev(phis)
    e0 = host(sys_.local_energy(phi))
    xb0 = host(sys_.force_bias(phi))
    x = gen.fields(spec, 0)
    w = dev(np.ones(spec.nwalkers))
    ld = torch.empty((spec.nwalkers, 2), dtype=torch.complex128, device="cuda")
    e1 = host(sys_.step(phi, dev(x), w, logdet=ld, do_qr=False, reuse=False))
    phi_g, w_g, ld_g = host(phi[:1]), host(w), host(ld)
    assert np.all(np.isfinite(e0)) and np.all(np.isfinite(e1)) and np.all(w_g > 0)
    # the adjoint of the seeded walkers' energy, walker 0's upstream weights only
    g = np.zeros((spec.nwalkers, 3), dtype=np.complex128)
    g[0] = gen.upstream(spec)[0]
    phi.copy_(torch.from_numpy(phis))
    gphi, gh1 = sys_.local_energy_backward(phi, dev(g))
    gphi0, gh1_h = host(gphi[:1])[0], host(gh1)
    del gphi
    assert sys_.last_error() == (0, 0)
    sys_.close()
    del phi
    torch.cuda.empty_cache()

    osys = ok.System(spec.grid, L, h1, A, spec.dt)
    workers = os.cpu_count() or 1

    def energy(p):
        Ghs = [ok.green_half(osys, p[s])[0] for s in range(2)]
        return np.array([ok.one_body_energy(osys, Ghs), ok.coulomb_energy(osys, ok.cholesky_trace(osys, Ghs)),
                         bench.exchange_in_pool(osys, Ghs, workers)])

    # the seeded walker
    Ghs = [ok.green_half(osys, phis[0][s])[0] for s in range(2)]
    assert rel(xb0[0], ok.force_bias(osys, ok.cholesky_trace(osys, Ghs))) < TOL_XBAR
    err = np.abs(e0[0] - energy(phis[0])) / spec.nk
    assert np.all(err < TOL_E), err
    # one step
    pn, wn, _, _, _ = ok.propagate_walker(osys, phis[0], x[0], 1.0)
    assert rel(phi_g[0], pn) < TOL_PHI
    assert abs(w_g[0] - wn) < TOL_W * wn
    ld_own = np.array([ok.log_det(ok.overlap(osys, phi_g[0][s])) for s in range(2)])
    assert np.abs(ld_g[0].real - ld_own.real).max() < TOL_LD
    err = np.abs(e1[0] - energy(pn)) / spec.nk
    assert np.all(err < TOL_E), err
    # the adjoint
    ref_phi, ref_h = ok.local_energy_vjp(osys, phis[0], g[0], two_body=bench.gamma_in_pool(workers))
    assert rel(gphi0, ref_phi) < 1e-5
    assert rel(gh1_h, ref_h) < 1e-10
