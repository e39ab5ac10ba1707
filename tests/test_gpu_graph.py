"""The fused walker step (afqmc_kp_step) captured into a CUDA graph.

A step allocates nothing and synchronises nothing, and its kernels are deterministic (no
floating-point atomics), so a graph replay must reproduce the eager steps bit for bit.
The log-determinant buffers of the handle alternate between steps, so one graph holds two
steps and is replayed with fresh fields copied into its static input buffers."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
from gpu_util import dev, make  # noqa: E402

pytestmark = pytest.mark.gpu

SPEC = gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16, random_trial=True, seed=4)


def run(precision: str, graph: bool):
    sys_, _ = make(SPEC, precision)
    phi = dev(gen.walkers(SPEC))
    w = torch.ones(SPEC.nwalkers, dtype=torch.float64, device="cuda")
    eloc = torch.empty((SPEC.nwalkers, 3), dtype=torch.complex128, device="cuda")
    xs = [dev(gen.fields(SPEC, i)) for i in range(5)]
    sys_.step(phi, xs[0], w, eloc, reuse=False)          # first step eager in both runs
    if not graph:
        for i in range(1, 5):
            sys_.step(phi, xs[i], w, eloc, do_qr=(i % 2 == 0))
    else:
        xa, xb = torch.empty_like(xs[0]), torch.empty_like(xs[0])
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sys_.step(phi, xa, w, eloc, do_qr=False)
            sys_.step(phi, xb, w, eloc, do_qr=True)
        for i in (1, 3):
            xa.copy_(xs[i])
            xb.copy_(xs[i + 1])
            g.replay()
    torch.cuda.synchronize()
    out = (phi.cpu().numpy(), w.cpu().numpy(), eloc.cpu().numpy(), sys_.last_error())
    sys_.close()
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_graph_replay_matches_eager_steps(precision):
    eager = run(precision, graph=False)
    graph = run(precision, graph=True)
    for a, b in zip(eager[:3], graph[:3]):
        assert np.array_equal(a, b)
    assert eager[3] == (0, 0) and graph[3] == (0, 0)
    assert np.all(np.isfinite(graph[2]))
