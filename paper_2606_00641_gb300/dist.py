"""Multi-rank helpers for independent-domain runs (one process per GPU).

The VLBM path shards into independent domains (each rank advances its own
periodic domain, or its own subset of a batch of domains); there is no data
exchange between ranks, so the only collectives are the timing and counting
reductions done here.  Works with any torch.distributed backend (NCCL on
GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import os


def env_ranks():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def weak_scaling_rate(ms_local: float, cells_local: int, steps: int, device=None):
    """Whole-job cell updates per second over all ranks.

    The job time is the slowest rank's time (max over ranks); the work is the
    sum of every rank's cells x steps.  Returns (rate in GLUPS, max ms, total
    cells).  Without an initialised process group it is the local figure."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return cells_local * steps / (ms_local * 1e-3) / 1e9, ms_local, cells_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    ms, cells = float(t.item()), int(c.item())
    return cells * steps / (ms * 1e-3) / 1e9, ms, cells


def shard_domains(sizes, world: int, rank: int):
    """Indices of the domains rank `rank` owns: greedy largest-first packing by
    cell count, so that every rank gets close to the same number of cells."""
    order = sorted(range(len(sizes)), key=lambda d: (-sizes[d], d))
    load = [0] * world
    owner = {}
    for d in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[d] = r
        load[r] += sizes[d]
    return [d for d in range(len(sizes)) if owner[d] == rank]
