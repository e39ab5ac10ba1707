"""afqmc_orthonormalise_noalloc: the re-orthonormalisation for callers that cannot
allocate device memory (graph capture in global mode, hosts that own every device
byte).  It must give the same walkers as afqmc_kp_orthonormalise, the handle-based
entry point, at the FP64 bar of the other tests (1e-10), on two calls in a row that
share the library's fixed scratch array.  Kept in a file that pytest collects last."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make, rel  # noqa: E402

pytestmark = pytest.mark.gpu


def noalloc(phi: "torch.Tensor", rows: int, cols: int, nmat: int) -> int:
    from paper_2003_09468_gb300 import load_library
    lib = load_library()
    return lib.afqmc_orthonormalise_noalloc(phi.data_ptr(), rows, cols, nmat,
                                            torch.cuda.current_stream().cuda_stream)


def skewed_walkers(spec, seed):
    rng = np.random.default_rng(seed)
    mix = rng.standard_normal((spec.N, spec.N)) + 1j * rng.standard_normal((spec.N, spec.N))
    return gen.walkers(spec) @ (np.eye(spec.N) + 0.3 * mix)


def test_noalloc_matches_handle_entry_point_on_two_calls():
    spec = gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=6, nwalkers=5, random_trial=True, seed=7)
    sys_, _ = make(spec, "fp64")
    for call, seed in enumerate((1, 2)):
        phis = skewed_walkers(spec, seed)
        ref = dev(phis)
        sys_.orthonormalise(ref)
        got = dev(phis)
        assert noalloc(got, spec.NM, spec.N, 2 * spec.nwalkers) == 0, call
        g, r = host(got), host(ref)
        assert rel(g, r) < 1e-10, call
        # orthonormal columns
        q = g.reshape(2 * spec.nwalkers, spec.NM, spec.N)
        gram = np.einsum("bij,bik->bjk", q.conj(), q)
        assert np.abs(gram - np.eye(spec.N)).max() < 1e-12
    sys_.close()


def test_noalloc_rejects_oversized_requests():
    phi = torch.zeros(16, dtype=torch.complex128, device="cuda")
    too_many = (32 * 1024 * 1024) // 16 + 1          # one element beyond the scratch array
    assert noalloc(phi, too_many, 1, 1) == 1
    assert noalloc(phi, 4, 8, 1) == 1                 # cols > rows
    assert noalloc(phi, 2048, 1025, 1) == 1           # cols beyond the kernel's limit
    # an 8-byte-aligned complex array (a C double complex pointer may be one) is refused on the
    # host: the kernel moves (re, im) pairs as 16-byte vectors
    base = torch.zeros(40, dtype=torch.float64, device="cuda")
    from paper_2003_09468_gb300 import load_library
    lib = load_library()
    assert lib.afqmc_orthonormalise_noalloc(base.data_ptr() + 8, 4, 2, 1,
                                            torch.cuda.current_stream().cuda_stream) == 1
