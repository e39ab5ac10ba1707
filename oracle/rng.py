"""CPU restatement of the device field generator and of the comb.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the product library never
calls it and shares no code with it.

* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC 2011, Sec. 3-4): ten rounds
  of a multiply-and-swap bijection of a 128-bit counter under a 64-bit key that
  advances by the Weyl constants between rounds.  Written with numpy uint64
  products, so the high and low 32-bit halves are exact.
* Box-Muller (Box and Muller 1958): two uniforms inside (0, 1) give two
  independent standard normals r cos(2 pi u2), r sin(2 pi u2), r = sqrt(-2 ln u1).
  The uniforms are the top 23 bits of each word plus one half, times 2^-23; the
  transform is evaluated in float64 and rounded to float32, which is the precision
  the device path delivers.
* The auxiliary fields are drawn from the standard normal distribution at every
  step (Sec. 2.1); each walker's field vector comes from its own counter
  (q, w, c_lo, c_hi), q indexing groups of four fields.
* Comb population control (the paper leaves population control out): with the
  running sums C_j of the weights and C the total, new walker k is old walker
  min{j : C_j > (k + u) C / W} and every new weight is C / W.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57          # round multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85          # key increments (golden ratio, sqrt(3) - 1)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr[..., 4] (uint32) under keys key[..., 2]; returns uint32 [..., 4]."""
    c = np.asarray(ctr, dtype=np.uint64) & _MASK
    k = np.broadcast_to(np.asarray(key, dtype=np.uint64) & _MASK, c.shape[:-1] + (2,)).copy()
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & _MASK
            k1 = (k1 + np.uint64(W1)) & _MASK
        p0 = np.uint64(M0) * c0            # < 2^64: exact
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def key_of(seed: int) -> np.ndarray:
    seed &= (1 << 64) - 1
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def uniform23(a) -> np.ndarray:
    """((a >> 9) + 1/2) 2^-23: exact in float32, inside (0, 1)."""
    return ((np.asarray(a, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(a, b):
    """Two standard normals per word pair, float64 arithmetic rounded to float32."""
    u1, u2 = uniform23(a), uniform23(b)
    r = np.sqrt(-2.0 * np.log(u1))
    z0 = (r * np.cos(2.0 * np.pi * u2)).astype(np.float32)
    z1 = (r * np.sin(2.0 * np.pi * u2)).astype(np.float32)
    return z0.astype(np.float64), z1.astype(np.float64), r


def field_words(seed: int, counter: int, W: int, F: int) -> np.ndarray:
    """Philox words [W][ceil(F/4)][4] of one step's fields."""
    nq = (F + 3) // 4
    ctr = np.zeros((W, nq, 4), dtype=np.uint64)
    ctr[..., 0] = np.arange(nq, dtype=np.uint64)[None, :]
    ctr[..., 1] = np.arange(W, dtype=np.uint64)[:, None]
    ctr[..., 2] = counter & 0xFFFFFFFF
    ctr[..., 3] = (counter >> 32) & 0xFFFFFFFF
    return philox4x32_10(ctr, key_of(seed))


def fields(seed: int, counter: int, shape) -> np.ndarray:
    """x[W][2][Nk][G] for one step; shape = (W, 2, Nk, G)."""
    W = shape[0]
    F = int(np.prod(shape[1:]))
    w = field_words(seed, counter, W, F)
    z0, z1, _ = box_muller(w[..., 0], w[..., 1])
    z2, z3, _ = box_muller(w[..., 2], w[..., 3])
    x = np.stack([z0, z1, z2, z3], axis=-1).reshape(W, -1)[:, :F]
    return x.reshape(shape)


def comb_uniform(seed: int, counter: int) -> float:
    """u = (a + 1/2) 2^-32, a the first word at counter (0, 0xffffffff, c_lo, c_hi)."""
    ctr = np.array([0, 0xFFFFFFFF, counter & 0xFFFFFFFF, (counter >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    a = int(philox4x32_10(ctr, key_of(seed))[0])
    return (a + 0.5) * 2.0 ** -32


def comb_indices(weight, u: float):
    """Old-walker index of each new walker and the new common weight (None if the total is unusable)."""
    w = np.asarray(weight, dtype=np.float64)
    W = w.size
    C = np.cumsum(w)                      # running sums in walker order
    tot = C[-1] if W else 0.0
    if not (tot > 0.0 and np.isfinite(tot)):
        return np.arange(W), None
    t = ((np.arange(W, dtype=np.float64) + u) * tot) / float(W)
    j = np.searchsorted(C, t, side="right")
    return np.minimum(j, W - 1), tot / W


def comb(phi, weight, seed: int, counter: int):
    """(phi, weight, idx) after the comb."""
    idx, wnew = comb_indices(weight, comb_uniform(seed, counter))
    if wnew is None:
        return phi.copy(), np.asarray(weight, dtype=np.float64).copy(), idx
    return phi[idx].copy(), np.full(len(idx), wnew), idx
