"""Pins of the CPU restatement of the field generator and of the comb.

* Philox4x32-10 against the known-answer values published with the generator
  (tests/golden/philox4x32_10_kat.txt), plus the bijection property of a fixed-key
  Philox and bit-balance statistics.
* Box-Muller against its own geometry (z0^2 + z1^2 = -2 ln u1, atan2(z1, z0) = 2 pi u2)
  and the moments and distribution function of the standard normal.
* The comb against a brute-force scan of its definition, the systematic-resampling
  multiplicity bound, unbiasedness over u, and its degenerate cases.
"""
import os

import numpy as np
import pytest

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        left, right = line.split("|")
        a = [int(v, 16) for v in left.split()]
        rows.append((a[:4], a[4:], [int(v, 16) for v in right.split()]))
    return rows


def test_philox_known_answers():
    rows = kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = rng.philox4x32_10(np.array(ctr), np.array(key))
        assert [int(v) for v in got] == want


def test_philox_fixed_key_is_a_bijection_of_the_counter():
    n = 1 << 16
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = 7
    out = rng.philox4x32_10(ctr, rng.key_of(12345)).astype(np.uint64)
    packed = (out[:, 0] << np.uint64(32)) | out[:, 1]
    assert np.unique(packed).size == n        # 64 of the 128 bits already distinct


def test_philox_bit_balance_and_counter_avalanche():
    n = 1 << 15
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n)
    out = rng.philox4x32_10(ctr, rng.key_of(0xDEADBEEFCAFEF00D))
    bits = np.unpackbits(out.view(np.uint8), axis=-1).reshape(n, -1).astype(np.float64)
    p = bits.mean(axis=0)
    assert np.all(np.abs(p - 0.5) < 5 * 0.5 / np.sqrt(n))
    # flipping one counter bit changes about half the output bits
    ctr2 = ctr.copy()
    ctr2[:, 1] ^= np.uint64(1)
    out2 = rng.philox4x32_10(ctr2, rng.key_of(0xDEADBEEFCAFEF00D))
    flips = np.unpackbits((out ^ out2).view(np.uint8), axis=-1).reshape(n, -1).sum(axis=1)
    assert abs(flips.mean() - 64.0) < 0.5


def test_philox_key_schedule_matters():
    ctr = np.array([1, 2, 3, 4])
    a = rng.philox4x32_10(ctr, np.array([1, 0]))
    b = rng.philox4x32_10(ctr, np.array([0, 1]))
    assert not np.array_equal(a, b)


def test_uniform_range_and_extremes():
    u = rng.uniform23(np.array([0, 511, 512, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24 and u[2] == 3 * 2.0 ** -24
    assert u[3] == 1.0 - 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in float32
    z0, z1, r = rng.box_muller(np.array([0, 0xFFFFFFFF]), np.array([0xFFFFFFFF, 0]))
    assert np.all(np.isfinite(z0)) and np.all(np.isfinite(z1))
    assert abs(r[0] - np.sqrt(48 * np.log(2.0))) < 1e-12          # u1 = 2^-24


def test_box_muller_geometry():
    g = np.random.default_rng(5)
    a = g.integers(0, 2 ** 32, 4096, dtype=np.uint64)
    b = g.integers(0, 2 ** 32, 4096, dtype=np.uint64)
    z0, z1, r = rng.box_muller(a, b)
    u1, u2 = rng.uniform23(a), rng.uniform23(b)
    assert np.allclose(z0 ** 2 + z1 ** 2, -2.0 * np.log(u1), rtol=3e-7, atol=1e-12)
    ang = np.mod(np.arctan2(z1, z0), 2 * np.pi)
    d = np.abs(ang - 2 * np.pi * u2)
    d = np.minimum(d, 2 * np.pi - d)
    assert np.max(d * np.maximum(r, 1e-3)) < 1e-6


def test_fields_are_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    x = rng.fields(2024, 3, (64, 2, 8, 64)).ravel()      # 65536 draws
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
    assert scipy_stats.kstest(x, "norm").pvalue > 1e-4
    # neighbouring fields of one walker and the same field of neighbouring walkers
    y = rng.fields(2024, 3, (64, 2, 8, 64)).reshape(64, -1)
    assert abs(np.corrcoef(y[:, :-1].ravel(), y[:, 1:].ravel())[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(y[:-1].ravel(), y[1:].ravel())[0, 1]) < 5 / np.sqrt(n)


def test_fields_differ_by_counter_seed_and_walker():
    a = rng.fields(1, 0, (4, 2, 1, 6))
    assert not np.array_equal(a, rng.fields(1, 1, (4, 2, 1, 6)))
    assert not np.array_equal(a, rng.fields(2, 0, (4, 2, 1, 6)))
    assert not np.array_equal(a[0], a[1])
    # the field count need not be a multiple of four: the shorter draw is a prefix
    b = rng.fields(1, 0, (4, 2, 1, 5))
    assert np.array_equal(b.reshape(4, -1), a.reshape(4, -1)[:, :10])


def comb_brute(w, u):
    W = len(w)
    C, s = [], 0.0
    for v in w:
        s += v
        C.append(s)
    out = []
    for k in range(W):
        t = ((k + u) * s) / W
        j = next((j for j in range(W) if C[j] > t), W - 1)
        out.append(j)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_comb_matches_brute_force_definition(seed):
    g = np.random.default_rng(seed)
    W = int(g.integers(1, 40))
    w = g.exponential(size=W) * (g.random(W) > 0.2)
    if w.sum() == 0:
        w[0] = 1.0
    u = float(g.random())
    idx, wnew = rng.comb_indices(w, u)
    assert list(idx) == comb_brute(list(w), u)
    assert wnew == pytest.approx(w.sum() / W, rel=1e-15)
    assert np.all(np.diff(idx) >= 0)
    assert np.all(w[idx] > 0)                    # a zero-weight walker is never chosen


def test_comb_multiplicities_and_unbiasedness():
    g = np.random.default_rng(11)
    W = 32
    w = g.exponential(size=W)
    expect = w * W / w.sum()
    mean = np.zeros(W)
    us = (np.arange(4096) + 0.5) / 4096
    for u in us:
        idx, _ = rng.comb_indices(w, u)
        cnt = np.bincount(idx, minlength=W)
        assert np.all(cnt >= np.floor(expect) - 1e-9) and np.all(cnt <= np.ceil(expect) + 1e-9)
        mean += cnt
    mean /= len(us)
    assert np.max(np.abs(mean - expect)) < 2e-3


def test_comb_degenerate_cases():
    idx, wnew = rng.comb_indices(np.ones(9), 0.999)
    assert list(idx) == list(range(9)) and wnew == 1.0
    for bad in (np.zeros(5), -np.ones(5), np.array([1.0, np.inf, 1.0]), np.array([1.0, np.nan])):
        idx, wnew = rng.comb_indices(bad, 0.5)
        assert wnew is None and list(idx) == list(range(len(bad)))
    idx, wnew = rng.comb_indices(np.array([0.0, 0.0, 3.0]), 0.1)
    assert list(idx) == [2, 2, 2] and wnew == 1.0


def test_comb_uniform_uses_the_reserved_counter():
    u = rng.comb_uniform(77, 5)
    a = int(rng.philox4x32_10(np.array([0, 0xFFFFFFFF, 5, 0]), rng.key_of(77))[0])
    assert u == (a + 0.5) * 2.0 ** -32 and 0.0 < u < 1.0
