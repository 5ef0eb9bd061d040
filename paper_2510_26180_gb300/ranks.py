"""Multi-GPU layout of a solve: one process per GPU, sample shards, no
data-path collective.

The samples of the method are independent (each runs its own Algorithm 2 on
its own coefficient field), so N GPUs take N disjoint batches: rank r draws
its batch from the seed ``seed + 1000 r`` and solves it alone.  The only
cross-rank traffic is the job's timing: the units all ranks processed are
summed and divided by the slowest rank's time (MAX over ranks), which is
the whole-job throughput of a weak-scaling run.
"""
from __future__ import annotations

import os


def world() -> tuple:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank ``rank``'s batch (rank 0 keeps the workload's own seed)."""
    return int(seed) + 1000 * int(rank)


def job_rate(local_units: float, local_ms: float, device=None) -> tuple:
    """(units per second of the whole job, slowest rank's ms, units of all
    ranks).  With an initialized process group of more than one rank, the
    time is reduced with MAX and the units with SUM; otherwise the local
    values are returned."""
    import torch
    import torch.distributed as dist
    ms = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    units = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        dist.all_reduce(units, op=dist.ReduceOp.SUM)
    ms_max = float(ms.item())
    total = float(units.item())
    return total / (ms_max / 1e3), ms_max, total
