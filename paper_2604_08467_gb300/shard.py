"""Host-side sharding of the hot path over ranks (one process per GPU).

The work shards without any exchange on the data path: trajectories of one
circuit are independent samples (each rank draws its own error sets from its
own Philox seed), and the circuits of a mixed batch are independent problems
(each rank runs a subset).  The only collective is the timing reduction
(the slowest rank's step time) used to report whole-job throughput.
"""
from __future__ import annotations

import heapq


def rank_seed(base_seed: int, rank: int, step: int) -> int:
    """Philox seed of rank `rank` for step `step`: distinct for every
    (rank, step) pair below 1000 steps, so ranks draw independent error sets."""
    if step < 0 or step >= 1000 * 1000 or rank < 0:
        raise ValueError("step must be in [0, 1e6) and rank >= 0")
    return int(base_seed) + 7919 * (rank * 1_000_000 + step)


def shard_items(costs, world: int):
    """Longest-processing-time assignment of independent items (e.g. the
    circuits of a mixed batch, with modelled costs) to `world` ranks: items in
    decreasing cost, each to the currently least-loaded rank (ties: lowest
    rank).  Returns one sorted index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest value over all ranks (all_reduce MAX); `value` itself
    without a process group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device="cpu") -> float:
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
