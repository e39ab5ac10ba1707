"""Seeded synthetic inputs for the k-point phaseless AFQMC walker step.

This module is the input recipe shared by the FP64 oracle and the CUDA path.
It holds no step of the method's arithmetic: it only draws random numbers and
places them with the symmetry the paper states for the inputs.

Recipe (all complex normals are (a + i b)/sqrt(2) with a, b ~ N(0, 1)):

* Cholesky vectors L[Q, k, g, p, r] (Sec. 2.3, Eq. kp_h2): p lives at k-point k,
  r at k - Q.  Each block is complex N(0, 1) scaled by exp(-g/16)/sqrt(Nk*M).
  The pair (Q, k) and (-Q, k - Q) is tied by the time-reversal relation
  L[-Q, k-Q][g] = L[Q, k][g]^dagger (Sec. 2.3); the block with the lexicographically
  smaller (Q, k) is drawn and its partner is the conjugate transpose.  The one
  self-partnered case, Q = 0, is Hermitised as (R + R^dagger)/2.
* One-body h[k] (Sec. 2.3, Eq. kp_h1): diag(linspace(0, 4, M)) plus 0.1 times a
  Hermitised complex normal off the diagonal.
* Trial A[k] (M x n per k-point, block diagonal in k, Sec. 2.3): the first n
  columns of the identity, or of a random unitary when ``random_trial``.
* Walkers phi[w, s] (NM x N per spin, dense in k): complex normal matrix with
  orthonormal columns ("random" walkers, far from the trial: a stress case for
  conditioning).
* Near-trial walkers: the orthonormalised columns of A + eps Z / sqrt(NM), with
  A the trial placed block-diagonally in the dense NM x N layout and Z complex
  normal, so that every column is moved by about eps of its length (eps = 0.1
  by default).  A projection starts from the trial (Sec. 2.1), so
  these are the walkers a simulation actually carries: well-conditioned
  overlaps, small phases, weights that stay positive over many steps.
* Auxiliary fields x[w, +/-, Q, g]: real N(0, 1) (Sec. 2.1, Eq. hs).
* Perturbation V1[k]: Hermitised complex N(0, 0.01).

Every block is drawn from ``numpy.random.default_rng(SeedSequence([seed, tag,
i, j]))`` so that any single (Q, k) block of L, walker or field row can be
regenerated alone, which lets the oracle stream systems whose L does not fit in
host memory.
"""
from __future__ import annotations

import itertools
import os
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

TAG_L = 1
TAG_H1 = 2
TAG_TRIAL = 3
TAG_WALKER = 4
TAG_FIELD = 5
TAG_V1 = 6
TAG_NEAR = 7


@dataclass(frozen=True)
class SystemSpec:
    """Sizes and seed of one synthetic k-point system."""

    grid: Tuple[int, int, int]
    M: int
    nocc: int
    nchol: int
    nwalkers: int
    dt: float = 0.005
    seed: int = 0
    random_trial: bool = False

    @property
    def nk(self) -> int:
        return int(np.prod(self.grid))

    @property
    def NM(self) -> int:
        return self.nk * self.M

    @property
    def N(self) -> int:
        return self.nk * self.nocc


# Workload shapes of the paper's diamond-carbon runs, restated as synthetic systems.
# 2x2x2 grid, 8 orbitals per k (small case the oracle finishes in seconds).
SMALL_2x2x2 = SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16)
# 3x3x3 grid with 26 orbitals per k: 702 basis functions and 2 x 108 electrons,
# the size of the DZVP 3x3x3 system used for the walker-batching study (Sec. 3.2).
DIAMOND_3x3x3 = SystemSpec(grid=(3, 3, 3), M=26, nocc=4, nchol=208, nwalkers=64)
# 4x4x4 grid, 52 orbitals per k (the synthetic analogue of the 4x4x4 TZVP run).
DIAMOND_4x4x4 = SystemSpec(grid=(4, 4, 4), M=52, nocc=4, nchol=416, nwalkers=256)
# Eight uneven systems run as one group (1024 walkers in all): grids 2x2x2 .. 3x3x3,
# M in {16, 26}, n in {2, 4}, 8M Cholesky vectors per Q, each with its own seed.
BATCHED_UNEVEN = [
    SystemSpec(grid=g, M=m, nocc=n, nchol=8 * m, nwalkers=w, seed=100 + i)
    for i, (g, m, n, w) in enumerate([
        ((2, 2, 2), 16, 2, 256), ((2, 2, 2), 26, 4, 128), ((2, 2, 3), 16, 2, 160), ((2, 2, 3), 26, 4, 96),
        ((2, 3, 3), 16, 4, 128), ((2, 3, 3), 26, 2, 96), ((3, 3, 3), 16, 2, 128), ((3, 3, 3), 26, 4, 32)])
]


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), *[int(v) for v in key]]))


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def kpoints(grid) -> np.ndarray:
    """Integer coordinates of the Gamma-centred grid, C order (last axis fastest)."""
    return np.array(list(itertools.product(*[range(int(g)) for g in grid])), dtype=np.int64)


def _partner(grid, Q: int, k: int) -> Tuple[int, int]:
    """(-Q, k - Q) for the time-reversal pairing of the synthetic blocks."""
    g = np.array(grid, dtype=np.int64)
    kp = kpoints(grid)
    mq = (-kp[Q]) % g
    kmq = (kp[k] - kp[Q]) % g
    lin = lambda v: int((v[0] * g[1] + v[1]) * g[2] + v[2])
    return lin(mq), lin(kmq)


def chol_block(spec: SystemSpec, Q: int, k: int) -> np.ndarray:
    """L[Q, k] as an (nchol, M, M) complex128 array."""
    scale = np.exp(-np.arange(spec.nchol) / 16.0) / np.sqrt(spec.nk * spec.M)
    Q2, k2 = _partner(spec.grid, Q, k)
    if (Q2, k2) == (Q, k):
        R = _cnormal(_rng(spec.seed, TAG_L, Q, k), (spec.nchol, spec.M, spec.M))
        R = R * scale[:, None, None]
        return 0.5 * (R + R.conj().transpose(0, 2, 1))
    if (Q, k) < (Q2, k2):
        R = _cnormal(_rng(spec.seed, TAG_L, Q, k), (spec.nchol, spec.M, spec.M))
        return R * scale[:, None, None]
    R = _cnormal(_rng(spec.seed, TAG_L, Q2, k2), (spec.nchol, spec.M, spec.M))
    return (R * scale[:, None, None]).conj().transpose(0, 2, 1).copy()


def cholesky(spec: SystemSpec, dtype=np.complex128, threads: int | None = None) -> np.ndarray:
    """All blocks L[Q, k, g, p, r] (Nk, Nk, nchol, M, M).  Every block comes from its own
    seeded stream, so the blocks are drawn on `threads` threads (default: every core; NumPy's
    generators and array arithmetic release the GIL) with the same result as one thread."""
    from concurrent.futures import ThreadPoolExecutor
    nk = spec.nk
    out = np.empty((nk, nk, spec.nchol, spec.M, spec.M), dtype=dtype)

    def fill(i):
        Q, k = divmod(i, nk)
        out[Q, k] = chol_block(spec, Q, k)

    nthreads = threads or os.cpu_count() or 1
    if nthreads <= 1 or nk * nk == 1:
        for i in range(nk * nk):
            fill(i)
    else:
        with ThreadPoolExecutor(min(nthreads, nk * nk)) as ex:
            list(ex.map(fill, range(nk * nk)))
    return out


def one_body(spec: SystemSpec) -> np.ndarray:
    """h[k, p, q] (Nk, M, M), Hermitian per k."""
    out = np.empty((spec.nk, spec.M, spec.M), dtype=np.complex128)
    for k in range(spec.nk):
        R = 0.1 * _cnormal(_rng(spec.seed, TAG_H1, k), (spec.M, spec.M))
        np.fill_diagonal(R, 0.0)
        out[k] = np.diag(np.linspace(0.0, 4.0, spec.M)) + 0.5 * (R + R.conj().T)
    return out


def trial(spec: SystemSpec) -> np.ndarray:
    """A[k, p, a] (Nk, M, nocc): occupied trial orbitals per k-point."""
    out = np.empty((spec.nk, spec.M, spec.nocc), dtype=np.complex128)
    for k in range(spec.nk):
        if spec.random_trial:
            U, _ = np.linalg.qr(_cnormal(_rng(spec.seed, TAG_TRIAL, k), (spec.M, spec.M)))
            out[k] = U[:, : spec.nocc]
        else:
            out[k] = np.eye(spec.M)[:, : spec.nocc]
    return out


def walkers(spec: SystemSpec, nw: int | None = None, first: int = 0) -> np.ndarray:
    """phi[w, s, NM, N] for walkers first .. first+nw-1, orthonormal columns."""
    nw = spec.nwalkers if nw is None else nw
    out = np.empty((nw, 2, spec.NM, spec.N), dtype=np.complex128)
    for i in range(nw):
        for s in range(2):
            Z = _cnormal(_rng(spec.seed, TAG_WALKER, first + i, s), (spec.NM, spec.N))
            out[i, s], _ = np.linalg.qr(Z)
    return out


def trial_dense(spec: SystemSpec) -> np.ndarray:
    """The trial as one dense NM x N matrix: A[k] at rows (k, p), columns (k, a)."""
    A = trial(spec)
    out = np.zeros((spec.NM, spec.N), dtype=np.complex128)
    for k in range(spec.nk):
        out[k * spec.M:(k + 1) * spec.M, k * spec.nocc:(k + 1) * spec.nocc] = A[k]
    return out


def near_trial_walkers(spec: SystemSpec, nw: int | None = None, first: int = 0, eps: float = 0.1) -> np.ndarray:
    """phi[w, s, NM, N] for walkers first .. first+nw-1: orthonormal columns spanning
    A + eps Z / sqrt(NM) (Z complex normal, its own stream per walker and spin)."""
    nw = spec.nwalkers if nw is None else nw
    A = trial_dense(spec)
    eps = eps / np.sqrt(spec.NM)
    out = np.empty((nw, 2, spec.NM, spec.N), dtype=np.complex128)
    for i in range(nw):
        for s in range(2):
            Z = _cnormal(_rng(spec.seed, TAG_NEAR, first + i, s), (spec.NM, spec.N))
            out[i, s], _ = np.linalg.qr(A + eps * Z)
    return out


def fields(spec: SystemSpec, step: int, nw: int | None = None, first: int = 0) -> np.ndarray:
    """x[w, +/-, Q, g] real N(0, 1) auxiliary fields for one time step."""
    nw = spec.nwalkers if nw is None else nw
    out = np.empty((nw, 2, spec.nk, spec.nchol), dtype=np.float64)
    for i in range(nw):
        out[i] = _rng(spec.seed, TAG_FIELD, step, first + i).standard_normal((2, spec.nk, spec.nchol))
    return out


def perturbation(spec: SystemSpec) -> np.ndarray:
    """V1[k, p, q] (Nk, M, M): Hermitian one-body perturbation, entries ~ N(0, 0.01)."""
    out = np.empty((spec.nk, spec.M, spec.M), dtype=np.complex128)
    for k in range(spec.nk):
        R = 0.01 * _cnormal(_rng(spec.seed, TAG_V1, k), (spec.M, spec.M))
        out[k] = 0.5 * (R + R.conj().T)
    return out


def upstream(spec: SystemSpec, nw: int | None = None, seed_offset: int = 0) -> np.ndarray:
    """Complex weights g[w, 3] for the three energy parts (upstream gradient)."""
    nw = spec.nwalkers if nw is None else nw
    return _cnormal(_rng(spec.seed + seed_offset, TAG_V1, 10_000), (nw, 3))


# ---------------------------------------------------------------------------
# Standard (dense) representation: one cell at the Gamma point, M orbitals,
# N occupied per spin, G Cholesky vectors L[g][p][r].
# ---------------------------------------------------------------------------
TAG_DENSE = 20


@dataclass(frozen=True)
class DenseSpec:
    """Sizes and seed of one synthetic standard-representation system.  real=True draws real
    symmetric Cholesky vectors (real orbitals, as for a Gamma-point supercell); otherwise the
    vectors come in adjoint pairs (L, L^dag), a set closed under the adjoint, as the vectors
    of a complex Hamiltonian's electron repulsion integrals are."""

    M: int
    nocc: int
    nchol: int
    nwalkers: int
    dt: float = 0.005
    seed: int = 0
    real: bool = True
    random_trial: bool = False

    @property
    def N(self) -> int:
        return self.nocc


# A two-cell Gamma-point supercell of the 1x1x2 k-point system with M = 26 per cell:
# M = 52, N = 8 per spin, 8M real vectors.
DENSE_1x1x2 = DenseSpec(M=52, nocc=8, nchol=416, nwalkers=64, real=True)
# the same cells in the k-point representation
KPOINT_1x1x2 = SystemSpec(grid=(1, 1, 2), M=26, nocc=4, nchol=208, nwalkers=64)


def dense_cholesky(spec: DenseSpec) -> np.ndarray:
    """L[g, p, r] (nchol, M, M), entries of size exp(-g / 2M) / sqrt(M)."""
    G, M = spec.nchol, spec.M
    scale = np.exp(-np.arange(G) / (2.0 * M)) / np.sqrt(M)
    r = _rng(spec.seed, TAG_DENSE, 0)
    if spec.real:
        R = r.standard_normal((G, M, M))
        return (0.5 * (R + R.transpose(0, 2, 1)) * scale[:, None, None]).astype(np.complex128)
    if G % 2:
        raise ValueError("adjoint pairs need an even number of vectors")
    R = _cnormal(r, (G // 2, M, M)) * scale[0::2, None, None]   # one size per pair
    out = np.empty((G, M, M), dtype=np.complex128)
    out[0::2] = R
    out[1::2] = R.conj().transpose(0, 2, 1)
    return out


def dense_one_body(spec: DenseSpec) -> np.ndarray:
    """h[p, q] (M, M): diagonal 0..4 plus a small Hermitian (real symmetric if real) part."""
    r = _rng(spec.seed, TAG_DENSE, 1)
    R = 0.1 * (r.standard_normal((spec.M, spec.M)) if spec.real else _cnormal(r, (spec.M, spec.M)))
    np.fill_diagonal(R, 0.0)
    return (np.diag(np.linspace(0.0, 4.0, spec.M)) + 0.5 * (R + R.conj().T)).astype(np.complex128)


def dense_trial(spec: DenseSpec) -> np.ndarray:
    """A[p, a] (M, nocc): the first nocc orbitals, or nocc columns of a random unitary."""
    if not spec.random_trial:
        return np.eye(spec.M, spec.nocc, dtype=np.complex128)
    Z = _cnormal(_rng(spec.seed, TAG_DENSE, 2), (spec.M, spec.M))
    Qm, _ = np.linalg.qr(Z)
    return np.ascontiguousarray(Qm[:, :spec.nocc])


def dense_walkers(spec: DenseSpec, nw: int | None = None, first: int = 0) -> np.ndarray:
    """phi[w, s, M, N], orthonormal columns."""
    nw = spec.nwalkers if nw is None else nw
    out = np.empty((nw, 2, spec.M, spec.N), dtype=np.complex128)
    for i in range(nw):
        for s in range(2):
            Qm, _ = np.linalg.qr(_cnormal(_rng(spec.seed, TAG_DENSE, 3, first + i, s), (spec.M, spec.N)))
            out[i, s] = Qm
    return out


def dense_near_trial_walkers(spec: DenseSpec, nw: int | None = None, first: int = 0, eps: float = 0.1) -> np.ndarray:
    """phi[w, s, M, N]: orthonormal columns spanning A + eps Z / sqrt(M), Z complex normal."""
    nw = spec.nwalkers if nw is None else nw
    A = dense_trial(spec)
    out = np.empty((nw, 2, spec.M, spec.N), dtype=np.complex128)
    for i in range(nw):
        for s in range(2):
            Z = _cnormal(_rng(spec.seed, TAG_DENSE, 5, first + i, s), (spec.M, spec.N))
            out[i, s], _ = np.linalg.qr(A + (eps / np.sqrt(spec.M)) * Z)
    return out


def dense_fields(spec: DenseSpec, step: int, nw: int | None = None, first: int = 0) -> np.ndarray:
    """x[w, +/-, g] real N(0, 1) fields of one step."""
    nw = spec.nwalkers if nw is None else nw
    out = np.empty((nw, 2, spec.nchol))
    for i in range(nw):
        out[i] = _rng(spec.seed, TAG_DENSE, 4, step, first + i).standard_normal((2, spec.nchol))
    return out

