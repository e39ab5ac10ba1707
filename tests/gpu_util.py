"""Helpers for the GPU parity tests: build handles from seeded inputs, oracle references."""
from __future__ import annotations

import numpy as np
import torch

import gen
from oracle import afqmc_kp as ok


def make(spec: gen.SystemSpec, precision: str = "fp64", taylor_order: int = 6):
    from paper_2003_09468_gb300 import KPointAFQMC
    L, h1, A = gen.cholesky(spec), gen.one_body(spec), gen.trial(spec)
    sys_ = KPointAFQMC(spec.grid, L, h1, A, spec.nwalkers, spec.dt, taylor_order=taylor_order, precision=precision)
    osys = ok.System(spec.grid, L, h1, A, spec.dt)
    return sys_, osys


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_energy(osys, phis, walkers=None):
    idx = range(len(phis)) if walkers is None else walkers
    return np.array([ok.local_energy(osys, phis[w]) for w in idx])


def oracle_xbar(osys, phi):
    Ghs = [ok.green_half(osys, phi[s])[0] for s in range(2)]
    return ok.force_bias(osys, ok.cholesky_trace(osys, Ghs))


def wrap_phase(a):
    return np.angle(np.exp(1j * np.asarray(a)))
