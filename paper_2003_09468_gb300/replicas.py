"""Walker replicas across processes (one per GPU).

Walkers are independent between the energy measurements, so a multi-GPU run gives every
rank its own walkers and a full copy of the Hamiltonian; nothing crosses ranks inside a
step.  The one exchange is the block's energy estimate, the weighted (mixed) estimator of
Sec. 2.1,

    E_block = sum_w W_w E_L(w) / sum_w W_w,

reduced as two numbers per rank (the weighted complex energy sum and the weight sum) with
one all-reduce over the ranks of `group`.  This module is plain PyTorch: the per-walker
energies and weights come from the library, the reduction is torch.distributed.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def local_sums(eloc: torch.Tensor, weight: torch.Tensor) -> torch.Tensor:
    """[Re sum_w W_w E_L(w), Im sum_w W_w E_L(w), sum_w W_w] of this rank's walkers.

    eloc: [W, 3] complex (E1, E_C, E_X per walker, as afqmc_kp_local_energy returns them);
    weight: [W] real.  Float64 on the device of `eloc`.
    """
    e = eloc.sum(dim=-1)
    w = weight.to(torch.float64)
    num = (w * e.real).sum(), (w * e.imag).sum()
    return torch.stack([num[0], num[1], w.sum()]).to(torch.float64)


def block_energy(eloc: torch.Tensor, weight: torch.Tensor, group=None) -> tuple[complex, float]:
    """Mixed estimator over the walkers of every rank in `group` (all of this rank's
    walkers when torch.distributed is not initialised): (E_block, total weight).
    A total weight of zero (every walker dead) gives E_block = nan."""
    s = local_sums(eloc, weight)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    num = complex(float(s[0]), float(s[1]))
    den = float(s[2])
    return (num / den if den != 0.0 else complex(float("nan"), float("nan"))), den
