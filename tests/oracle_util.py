"""Helpers shared by the test files: build oracle systems from the seeded generator."""
from __future__ import annotations

import numpy as np

import gen
from oracle import afqmc_kp as ok


def oracle_system(spec: gen.SystemSpec) -> ok.System:
    return ok.System(spec.grid, gen.cholesky(spec), gen.one_body(spec), gen.trial(spec), spec.dt)


def tiny(grid=(1, 1, 2), M=2, nocc=1, nchol=3, nw=2, random_trial=True, seed=1):
    return gen.SystemSpec(grid=grid, M=M, nocc=nocc, nchol=nchol, nwalkers=nw, dt=0.01,
                          seed=seed, random_trial=random_trial)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
