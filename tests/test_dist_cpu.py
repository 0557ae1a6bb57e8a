"""Multi-rank logic on CPU with the gloo backend (world size 2): the max over
ranks used for the reported step time, and the cost-balanced split of a batch
of independent problems (every problem on exactly one rank)."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_math_9907190_gb300 import dist as D
from paper_math_9907190_gb300 import inputs as I


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = D.max_over_ranks(1.5 + rank)
        sides = I.batch_sides(512)
        mine = D.shard_by_cost([n * n for n in sides], rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = (m, gathered)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_batch_sharding_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    sides = I.batch_sides(512)
    costs = [n * n for n in sides]
    for rank in range(world):
        m, gathered = out[rank]
        assert m == 2.5
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(len(sides)))
        loads = [sum(costs[i] for i in part) for part in gathered]
        assert max(loads) - min(loads) <= max(costs)
    assert out[0][1] == out[1][1]


def test_single_rank_defaults():
    assert D.max_over_ranks(3.0) == 3.0
    assert D.shard_by_cost([5, 1, 3], 0, 1) == [0, 1, 2]
    assert D.world()[1] >= 1
