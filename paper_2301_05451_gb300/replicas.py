"""Multi-GPU execution of the contraction: replicas.

The path shards naturally -- batch rows, parameter-shift copies and slices
are independent and meet in one sum -- and each box here has one GPU, so N
processes run N independent replicas of the workload (weak scaling, no
data-path collective).  What they share is the timing protocol: a barrier
before and after the timed steps and the maximum of the ranks' times.
"""
from __future__ import annotations

import os

import torch


def env():
    """(rank, world size, local rank) from the launcher's environment."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, dist=None, device=None):
    """The largest of every rank's value (a float); `dist` is
    torch.distributed when a process group is up, else None."""
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, seconds, dist=None, device=None):
    """Whole-job throughput: units processed by all ranks divided by the
    slowest rank's time."""
    world = dist.get_world_size() if dist is not None else 1
    return units_per_rank * world / max_over_ranks(seconds, dist, device)


def row_range(n_rows, rank, world):
    """Contiguous share of n_rows for `rank` (used when a batch is split over
    ranks instead of replicated)."""
    per = (n_rows + world - 1) // world
    lo = min(n_rows, rank * per)
    return lo, min(n_rows, lo + per)
