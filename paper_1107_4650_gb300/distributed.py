"""Multi-process host logic: one process per GPU, no collective on the data path.

The single-grid step does not shard here (one grid per GPU, replicas); the batched Klein ensemble is a
set of independent runs, so a job of N ranks draws N x runs_per_rank runs once and gives each rank an
equal number of them with about equal work.  The only collectives are the timing reduction (the slowest
rank's time) and barriers around the timed region.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def run_cost(run) -> float:
    """Point-steps of one run (side^2 x steps): the quantity the batched kernel's time follows."""
    return float(run.side) * float(run.side) * float(run.nsteps)


def ensemble_shard(runs_per_rank: int, rank: int, world: int, seed: int = W.SEED + 1):
    """This rank's share of one global draw of runs_per_rank * world ensemble runs.

    Runs are sorted by cost (largest first, ties by draw index) and dealt in a snake order 0..N-1, N-1..0,
    so every rank gets exactly runs_per_rank runs and the costs differ by at most the largest run's.
    Returns (runs, indices into the global draw, the global draw's deviation log)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    runs, log = W.klein_ensemble(nruns=runs_per_rank * world, seed=seed)
    cost = np.array([run_cost(r) for r in runs])
    order = sorted(range(len(runs)), key=lambda i: (-cost[i], i))
    mine = []
    for pos, i in enumerate(order):
        lap, k = divmod(pos, world)
        owner = k if lap % 2 == 0 else world - 1 - k
        if owner == rank:
            mine.append(i)
    mine.sort()
    return [runs[i] for i in mine], mine, log


def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """The largest value of x over all ranks (all-reduce MAX); x itself with one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
