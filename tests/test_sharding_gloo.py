"""Multi-rank host logic on CPU (gloo, world size 2): the snapshot split and
the timing reductions the benchmark uses when it runs on several GPUs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2601_23002_gb300.sharding import shard, snapshot_cost, max_over_ranks, sum_over_ranks
from workloads import batch_cells


def test_shard_covers_every_snapshot_once_and_balances():
    cells = batch_cells(64)
    costs = [snapshot_cost(c.n) for c in cells]
    for world in (1, 2, 3, 8):
        parts = [shard(costs, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs) + 1e-6 * sum(costs)


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard([1.0], 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [snapshot_cost(c.n) for c in batch_cells(16)]
        mine = shard(costs, world, rank)
        t = 1.0 + rank          # this rank's time
        out[rank] = (max_over_ranks(t), sum_over_ranks(len(mine)), tuple(mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_count():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of a threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.0            # the slowest rank's time
    assert out[0][1] == out[1][1] == 16.0           # every snapshot counted once
    assert not set(out[0][2]) & set(out[1][2])


def test_without_a_process_group_the_reductions_are_identities():
    assert max_over_ranks(3.5) == 3.5 and sum_over_ranks(7) == 7.0
