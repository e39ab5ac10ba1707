"""Multi-process replica reduction (Sec. 2.1 mixed estimator) on CPU ranks with gloo:
two ranks holding disjoint walker sets must give the single-process estimate over the
union, and a rank whose walkers all have zero weight must not disturb it."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2003_09468_gb300.replicas import block_energy  # noqa: E402


def data(rank: int, nwalk: int = 7):
    rng = np.random.default_rng(100 + rank)
    e = rng.standard_normal((nwalk, 3)) + 1j * rng.standard_normal((nwalk, 3))
    w = rng.uniform(0.1, 2.0, nwalk)
    if rank == 1:
        w[::3] = 0.0   # dead walkers stay in the batch with zero weight
    return torch.from_numpy(e), torch.from_numpy(w)


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        e, w = data(rank)
        est, tot = block_energy(e, w)
        out[rank] = (est.real, est.imag, tot)
    finally:
        dist.destroy_process_group()


def test_two_rank_block_energy_matches_union():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(worker, args=(world, free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    es = [data(r) for r in range(world)]
    e = np.concatenate([x[0].numpy() for x in es])
    w = np.concatenate([x[1].numpy() for x in es])
    ref = (w * e.sum(axis=1)).sum() / w.sum()
    for r in range(world):
        got = complex(res[r][0], res[r][1])
        assert abs(got - ref) < 1e-12 * abs(ref)
        assert abs(res[r][2] - w.sum()) < 1e-12 * w.sum()


def test_single_process_and_dead_batch():
    e, w = data(0)
    est, tot = block_energy(e, w)
    ref = (w.numpy() * e.numpy().sum(axis=1)).sum() / w.numpy().sum()
    assert abs(est - ref) < 1e-12 * abs(ref) and abs(tot - w.sum().item()) < 1e-12
    est0, tot0 = block_energy(e, torch.zeros_like(w))
    assert tot0 == 0.0 and np.isnan(est0.real)
