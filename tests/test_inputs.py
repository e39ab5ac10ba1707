"""The input recipe (gen/): the near-trial walker set the parity bars and the benchmark use.
CPU only; the recipe holds no method arithmetic, these check its stated properties."""
import numpy as np

import gen
from oracle import afqmc_kp as ok
from oracle_util import oracle_system


def test_near_trial_walkers_are_orthonormal_and_seeded():
    spec = gen.SystemSpec(grid=(2, 1, 3), M=7, nocc=3, nchol=5, nwalkers=4, random_trial=True, seed=3)
    a = gen.near_trial_walkers(spec)
    b = gen.near_trial_walkers(spec, 2, first=2)
    assert a.shape == (4, 2, spec.NM, spec.N)
    assert np.array_equal(a[2:], b)                         # any walker regenerates alone
    q = a.reshape(-1, spec.NM, spec.N)
    assert np.abs(np.einsum("bij,bik->bjk", q.conj(), q) - np.eye(spec.N)).max() < 1e-13
    # close to the trial: the overlap with the (orthonormal) trial is well conditioned
    A = gen.trial_dense(spec)
    for p in q:
        s = np.linalg.svd(A.conj().T @ p, compute_uv=False)
        assert s.min() > 0.9 and s.max() <= 1.0 + 1e-12
    # the random set is far from it
    r = gen.walkers(spec).reshape(-1, spec.NM, spec.N)
    assert min(np.linalg.svd(A.conj().T @ p, compute_uv=False).min() for p in r) < 0.5


def test_trial_dense_places_the_blocks():
    spec = gen.SystemSpec(grid=(1, 2, 2), M=5, nocc=2, nchol=3, nwalkers=1, random_trial=True, seed=1)
    A, Ad = gen.trial(spec), gen.trial_dense(spec)
    for k in range(spec.nk):
        for k2 in range(spec.nk):
            blk = Ad[k * spec.M:(k + 1) * spec.M, k2 * spec.nocc:(k2 + 1) * spec.nocc]
            assert np.array_equal(blk, A[k] if k == k2 else np.zeros_like(blk))


def test_near_trial_walkers_stay_alive_over_ten_steps():
    """Over ten oracle steps (QR every fifth) the near-trial walkers keep positive weights and
    well-conditioned overlaps: the benchmark's timed regime is a live population."""
    spec = gen.SMALL_2x2x2
    osys = oracle_system(spec)
    for i in (0, 7):
        phi, w = gen.near_trial_walkers(spec, 1, first=i)[0], 1.0
        for s in range(10):
            phi, w, _, _, _ = ok.propagate_walker(osys, phi, gen.fields(spec, s, 1, first=i)[0], w)
            if (s + 1) % 5 == 0:
                phi = np.stack([ok.orthonormalise(phi[sp]) for sp in range(2)])
            assert w > 0
        assert max(np.linalg.cond(ok.overlap(osys, phi[sp])) for sp in range(2)) < 2.0


def test_dense_near_trial_walkers():
    spec = gen.DenseSpec(M=12, nocc=3, nchol=4, nwalkers=3, random_trial=True, seed=5)
    q = gen.dense_near_trial_walkers(spec).reshape(-1, spec.M, spec.N)
    A = gen.dense_trial(spec)
    assert np.abs(np.einsum("bij,bik->bjk", q.conj(), q) - np.eye(spec.N)).max() < 1e-13
    assert min(np.linalg.svd(A.conj().T @ p, compute_uv=False).min() for p in q) > 0.9
