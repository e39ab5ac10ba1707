"""The adjoint behind torch.autograd (binding.LocalEnergy).

FP64 path: the gradients PyTorch reports for a real loss L = Re sum c E match central finite
differences of L along random complex directions of the walkers and of a Hermitian one-body
perturbation (E is linear in h, so the h-derivative is exact up to rounding).  Mixed path: the
same gradients as the FP64 path within the mixed adjoint's bar (1e-5 of the gradient norm).
"""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
from gpu_util import dev, make  # noqa: E402

pytestmark = pytest.mark.gpu

SPEC = gen.SystemSpec(grid=(2, 2, 1), M=6, nocc=2, nchol=12, nwalkers=3, random_trial=True, seed=41)


def loss_and_grads(sys_, phi0, h0, c):
    from paper_2003_09468_gb300 import LocalEnergy
    phi = phi0.clone().requires_grad_(True)
    h1 = h0.clone().requires_grad_(True)
    E = LocalEnergy.apply(phi, h1, sys_)
    L = (E * c).real.sum()
    L.backward()
    return float(L.detach()), phi.grad.detach().clone(), h1.grad.detach().clone()


def loss_at(sys_, phi, h1, c):
    sys_.set_one_body(h1.contiguous())
    return float((sys_.local_energy(phi.contiguous()) * c).real.sum())


def test_fp64_autograd_matches_finite_differences():
    sys_, _ = make(SPEC, "fp64")
    rng = np.random.default_rng(3)
    phi0 = dev(gen.walkers(SPEC))
    h0 = dev(gen.one_body(SPEC))
    c = dev(rng.standard_normal((SPEC.nwalkers, 3)) + 1j * rng.standard_normal((SPEC.nwalkers, 3)))
    _, gphi, gh = loss_and_grads(sys_, phi0, h0, c)
    hstep = 1e-6
    for _ in range(2):
        d = dev(rng.standard_normal(phi0.shape) + 1j * rng.standard_normal(phi0.shape))
        fd = (loss_at(sys_, phi0 + hstep * d, h0, c) - loss_at(sys_, phi0 - hstep * d, h0, c)) / (2 * hstep)
        an = float((gphi.conj() * d).real.sum())
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)
    dh = rng.standard_normal(h0.shape) + 1j * rng.standard_normal(h0.shape)
    dh = dev(0.5 * (dh + dh.conj().transpose(0, 2, 1)))
    fd = (loss_at(sys_, phi0, h0 + dh, c) - loss_at(sys_, phi0, h0 - dh, c)) / 2.0
    an = float((gh.conj() * dh).real.sum())
    assert abs(fd - an) < 1e-10 * max(1.0, abs(an)), (fd, an)
    sys_.close()


def test_mixed_autograd_matches_fp64():
    rng = np.random.default_rng(4)
    phi0 = dev(gen.walkers(SPEC))
    h0 = dev(gen.one_body(SPEC))
    c = dev(rng.standard_normal((SPEC.nwalkers, 3)) + 1j * rng.standard_normal((SPEC.nwalkers, 3)))
    out = {}
    for prec in ("fp64", "mixed"):
        sys_, _ = make(SPEC, prec)
        out[prec] = loss_and_grads(sys_, phi0, h0, c)
        # the autograd path is the library's adjoint, unchanged
        gphi, gh = sys_.local_energy_backward(phi0, c.conj().resolve_conj())
        with pytest.raises(ValueError):      # a lazy conjugate view is refused, not misread
            sys_.local_energy_backward(phi0, c.conj())
        assert torch.equal(gphi, out[prec][1]) and torch.equal(gh, out[prec][2])
        sys_.close()
    (l64, g64, h64), (lmx, gmx, hmx) = out["fp64"], out["mixed"]
    assert abs(lmx - l64) < 2e-6 * max(1.0, abs(l64))
    assert float(torch.linalg.vector_norm(gmx - g64) / torch.linalg.vector_norm(g64)) < 1e-5
    assert float(torch.linalg.vector_norm(hmx - h64) / torch.linalg.vector_norm(h64)) < 1e-10
