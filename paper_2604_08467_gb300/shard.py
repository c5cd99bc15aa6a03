"""Host-side sharding of the hot path over ranks (one process per GPU).

Replica mode shards without any exchange on the data path: trajectories of one
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


# ------------------------------------------------ one job over many ranks ----
#
# The method parallelises over error sets (Sec. III; Fig. 1): one proportional
# NBS job of E trajectories and M shots is split by trajectory range, rank r
# taking [r E / G, (r + 1) E / G).  Every Philox counter carries the global
# trajectory index, so the ranks draw exactly the error sets and shots of the
# single-process run.  The exchange steps are: one allgather of the
# per-trajectory weights a_i = c_i w_i (w_i the block-1 total of trajectory i),
# after which every rank makes the same global multinomial allocation of M and
# keeps its slice, and one gather of the final (trajectory, bitstring, count)
# records, whose concatenation in rank order is the canonical order.


def traj_range(rank: int, world: int, n_traj: int):
    """[start, stop) of the trajectories of `rank` when n_traj are split over
    `world` ranks in contiguous, nearly equal ranges."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return rank * n_traj // world, (rank + 1) * n_traj // world


class LocalComm:
    """Collectives of a single process (world of one)."""

    rank, world = 0, 1

    def allgather(self, obj):
        return [obj]


class DistComm:
    """Collectives over an initialised torch.distributed process group (the
    exchanged objects are small host arrays: weights and final records)."""

    def __init__(self, dist):
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def allgather(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj)
        return out


class GpuBackend:
    """The library's calls for one rank's range: presampling with global
    counters, block contractions over the rank's trajectories, the global
    allocation and conditional sampling with global trajectory indices."""

    def __init__(self, plan, precision=0, circuit_id=0):
        from . import ptn
        self.ptn = ptn
        self.plan = plan
        self.precision = precision
        self.circuit_id = circuit_id
        self.traj = None

    def presample(self, seed, traj0, n):
        self.traj = self.ptn.ptn_presample_range(self.plan, seed, traj0, n, circuit_id=self.circuit_id)

    def contract(self, j, local, prefix):
        import numpy as np
        import torch
        b = self.plan.blocks[j][1]
        nt = torch.as_tensor(np.asarray(local, np.int32), device="cuda")
        npre = torch.as_tensor(np.asarray(prefix, np.uint64).astype(np.int64), device="cuda")
        marg = torch.empty((len(local), 1 << b), dtype=torch.float32, device="cuda")
        Z = torch.empty(len(local), dtype=torch.float64, device="cuda")
        if len(local):
            self.ptn.ptn_contract_batch(self.plan, self.traj, j, nt, npre, marg, Z, precision=self.precision)
        return marg, Z.cpu().numpy()

    def allocate(self, weights, total, seed):
        import numpy as np
        import torch
        w = torch.as_tensor(np.asarray(weights, np.float64), device="cuda")
        m = torch.empty(len(weights), dtype=torch.int64, device="cuda")
        self.ptn.ptn_allocate_shots(w, total, seed, self.circuit_id, m)
        return m.cpu().numpy()

    def sample(self, rows, gtraj, prefix, counts, seed, j):
        import numpy as np
        import torch
        start, b = self.plan.blocks[j]
        cap = int(np.minimum(counts, 1 << b).sum())
        if cap == 0:
            return gtraj[:0], prefix[:0], counts[:0]
        pt = torch.as_tensor(np.asarray(gtraj, np.int32), device="cuda")
        pp = torch.as_tensor(np.asarray(prefix, np.uint64).astype(np.int64), device="cuda")
        pc = torch.as_tensor(np.asarray(counts, np.int64), device="cuda")
        ct = torch.empty(cap, dtype=torch.int32, device="cuda")
        cp = torch.empty(cap, dtype=torch.int64, device="cuda")
        cc = torch.empty(cap, dtype=torch.int64, device="cuda")
        nc = self.ptn.ptn_sample_block(rows, b, start, pt, pp, pc, seed, self.circuit_id, j, ct, cp, cc)
        return (ct[:nc].cpu().numpy().astype(np.int64), cp[:nc].cpu().numpy().astype(np.uint64),
                cc[:nc].cpu().numpy())


def sharded_proportional(backend, comm, blocks, n_traj, total_shots, seed):
    """One proportional NBS job of n_traj trajectories and total_shots shots,
    this rank's part of it on `backend`, exchanged through `comm`.  Returns
    the job's final records (traj, bits, count) in canonical order on every
    rank, and this rank's number of networks per block."""
    import numpy as np
    r0, r1 = traj_range(comm.rank, comm.world, n_traj)
    n = r1 - r0
    backend.presample(seed, r0, n)
    local = np.arange(n, dtype=np.int64)
    rows0, Z = backend.contract(0, local, np.zeros(n, np.uint64))
    w_all = np.concatenate(comm.allgather(np.asarray(Z, np.float64)))       # global trajectory order
    m = backend.allocate(w_all, total_shots, seed)[r0:r1]
    keep = np.nonzero(m > 0)[0]
    gtraj = keep + r0
    prefix = np.zeros(len(keep), np.uint64)
    counts = m[keep]
    nets = []
    for j, (start, b) in enumerate(blocks):
        nets.append(n if j == 0 else len(gtraj))        # block 1 contracts every trajectory of the range
        rows = rows0[keep] if j == 0 else backend.contract(j, gtraj - r0, prefix)[0]
        gtraj, prefix, counts = backend.sample(rows, gtraj, prefix, counts, seed, j)
    parts = comm.allgather((gtraj, prefix, counts))
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(3)), nets
