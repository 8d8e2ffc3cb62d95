"""Several GPUs, one process each: how the evaluation shards.

Every lattice point, sector, kinematic point and random shift of the method
is independent, so ranks need no exchange inside an evaluation pass.

* Adaptive integration (qmc_integrate): each pass splits the (kinematic
  point, sector) slots to evaluate over the ranks by cost; each rank
  evaluates its share on its GPU, and one sum over the ranks per pass
  (``allreduce_fn``, installed with ``set_ranks``) gives every rank the same
  per-shift sums, so that all ranks take the same allocation decisions and
  return the one-rank result.
* The throughput bench: rank r evaluates the same jobs as every other rank
  with its own shift streams (seed = base seed + r): the ranks' shifts
  together are N x m independent random shifts of each lattice (weak
  scaling: per-rank work is fixed). The timing of a step is the slowest
  rank's.

The collectives are torch.distributed calls on host tensors (gloo) or device
tensors (nccl); nothing here computes any part of the method.
"""
from __future__ import annotations

import numpy as np


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s shift streams."""
    return int(base_seed) + int(rank)


def gather_shift_sums(local, group=None, device=None):
    """All-gather per-shift sums [jobs][m][orders][2] from every rank and
    concatenate them along the shift axis in rank order: [jobs][N m][orders][2]."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(np.ascontiguousarray(local, dtype=np.float64))
    if device is not None:
        t = t.to(device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    return np.concatenate([p.cpu().numpy() for p in parts], axis=1)


def max_over_ranks(value: float, group=None, device=None) -> float:
    """The largest `value` over all ranks (step time of the slowest rank)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def allreduce_fn(group=None, device=None):
    """A function summing a float64 numpy array in place over all ranks (the
    exchange of a rank-partitioned qmc_integrate pass)."""
    import torch
    import torch.distributed as dist

    def reduce(buf):
        t = torch.from_numpy(np.array(buf, dtype=np.float64, copy=True))
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        buf[:] = t.cpu().numpy()

    return reduce


def set_ranks(ctx, group=None, device=None):
    """Make qmc_integrate on `ctx` one rank of a partitioned integration over
    the ranks of the process group."""
    import torch.distributed as dist

    from . import qmc

    qmc.qmc_set_ranks(ctx, dist.get_rank(group), dist.get_world_size(group), allreduce_fn(group, device))
