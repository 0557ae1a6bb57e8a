"""Multi-rank plumbing: one process per GPU, no collective on the data path.

A single Poisson problem does not shard without a halo exchange at every
stage of every level, so one problem runs on one GPU and N ranks run N
replicas.  Independent problems of a batch are split across ranks by cost
(unknowns); the only collective is the max of the per-rank step time that a
benchmark reports.
"""

from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device: torch.device | None = None) -> float:
    """The maximum of a per-rank scalar (e.g. a step time) over all ranks."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or torch.device("cpu"))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_by_cost(costs, rank: int, nranks: int) -> list[int]:
    """Indices of the items rank `rank` handles: largest items first, each to
    the rank with the least total cost so far (ties to the lower rank).  Every
    rank computes the same assignment; every item goes to exactly one rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * nranks
    owner = [0] * len(costs)
    for i in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]
