"""Multi-GPU host logic.  Snapshots (cells) are independent, so ranks take
disjoint sets of them and exchange only their timings: no collective on the
data path.  A single cell does not shard (its 3-D FFTs would need an
all-to-all per transform); there every rank runs a replica."""
from __future__ import annotations

import math


def snapshot_cost(n: int) -> float:
    """Relative cost of one snapshot on an n^3 grid (FFT-bound: N log N)."""
    N = float(n) ** 3
    return N * math.log2(N)


def shard(costs, world: int, rank: int) -> list[int]:
    """Indices of the snapshots rank `rank` of `world` takes: longest first to
    the least-loaded rank (ties to the lower rank), so every index goes to
    exactly one rank and the loads differ by at most the largest cost.
    Deterministic: every rank computes the same assignment."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += float(costs[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank number over the default process group (the
    slowest rank sets the job's time); x itself without one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of a per-rank count over the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
