"""The multi-rank path on CPU: two gloo ranks (no GPU) exercise the host
logic that shards the hot path over GPUs: per-rank Philox seeds give
independent error sets, the circuits of a mixed batch are shared out
without overlap, and the timing / throughput reductions."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_08467_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from oracle import pts
    cfg = W.config_c1()
    seeds = [shard.rank_seed(cfg["seed"], rank, k) for k in range(3)]
    kraus, _ = pts.presample(cfg["circuit"], 16, seeds[0])
    costs = [5.0, 1.0, 3.0, 3.0, 0.5, 8.0, 2.0]
    mine = shard.shard_items(costs, world)[rank]
    t = 1.0 + rank                         # this rank's step time
    res = dict(seeds=seeds, rows=kraus.tolist(), mine=mine,
               tmax=shard.max_over_ranks(t, dist), shots=shard.sum_over_ranks(1000 * (rank + 1), dist))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    # independent error sets: distinct seeds, different Kraus rows
    assert not set(r[0]["seeds"]) & set(r[1]["seeds"])
    assert r[0]["rows"] != r[1]["rows"]
    # the shards cover every item once
    assert sorted(r[0]["mine"] + r[1]["mine"]) == list(range(7))
    assert not set(r[0]["mine"]) & set(r[1]["mine"])
    # reductions: slowest rank's time, all ranks' shots
    assert r[0]["tmax"] == r[1]["tmax"] == 2.0
    assert r[0]["shots"] == r[1]["shots"] == 3000.0


def test_shard_items_balances_by_cost():
    costs = [5.0, 1.0, 3.0, 3.0, 0.5, 8.0, 2.0]
    parts = shard.shard_items(costs, 2)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(costs)
    assert shard.shard_items(costs, 1) == [list(range(7))]
    assert shard.shard_items([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard.shard_items(costs, 0)


def test_rank_seeds_distinct():
    seen = {shard.rank_seed(7, r, k) for r in range(8) for k in range(1000)}
    assert len(seen) == 8000
    with pytest.raises(ValueError):
        shard.rank_seed(7, 0, 10 ** 6)
    assert shard.max_over_ranks(3.5) == 3.5 and shard.sum_over_ranks(2.0) == 2.0
    np.testing.assert_equal(shard.rank_seed(0, 0, 0), 0)


# ------------------------------------------- one job split over two ranks ----

class OracleBackend:
    """The oracle standing in for the library inside the sharded pipeline:
    state-vector marginals of the rank's trajectories (drawn with their global
    counters), the oracle's allocation and its conditional sampling."""

    def __init__(self, circ, blocks):
        self.circ, self.blocks = circ, blocks

    def presample(self, seed, traj0, n):
        from oracle import pts, statevector as sv
        kraus, _ = pts.presample(self.circ, n, seed, traj0=traj0)
        self.probs = [np.abs(sv.trajectory_state(self.circ, kraus[i])) ** 2 for i in range(n)]

    def contract(self, j, local, prefix):
        from oracle import statevector as sv
        start, b = self.blocks[j]
        rows = np.array([sv.block_marginals(self.probs[int(i)], self.circ.n_qubits, start, b)[
            int(s) & ((1 << start) - 1)] for i, s in zip(local, prefix)]).reshape(len(local), 1 << b)
        return rows, rows.sum(axis=1)

    def allocate(self, weights, total, seed):
        from oracle import sampling
        return sampling.allocate_shots(weights, total, seed)

    def sample(self, rows, gtraj, prefix, counts, seed, j):
        from oracle import sampling
        start = self.blocks[j][0]
        par, xs, cs = sampling.sample_block(rows, gtraj, counts, sampling.rank_offsets(gtraj, counts), seed, j)
        return gtraj[par], prefix[par] | (xs.astype(np.uint64) << np.uint64(start)), cs


def _sharded_job(seed):
    import workloads as W
    rng = np.random.default_rng(808)
    circ = W.attach_noise(W.brickwork_1d(8, 5, rng), [W.depolarizing_kraus(0.05), W.amplitude_damping_kraus(0.1)])
    return circ, [(0, 3), (3, 3), (6, 2)], 13, 5000


def _sharded_rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    circ, blocks, E, M = _sharded_job(0)
    (t, b, c), nets = shard.sharded_proportional(OracleBackend(circ, blocks), shard.DistComm(dist), blocks, E, M,
                                                 seed=4242)
    np.savez(os.path.join(out_dir, f"job{rank}.npz"), t=t, b=b, c=c, nets=np.array(nets))
    dist.barrier()
    dist.destroy_process_group()


def test_one_job_split_over_two_gloo_ranks(tmp_path):
    """Two gloo ranks run one proportional NBS job by trajectory range (global
    Philox counters, allgathered weights, one global allocation, gathered
    records): with the oracle as the marginal source the gathered records equal
    the single-process run bit for bit, on both ranks."""
    from oracle import pts, sampling, statevector as sv
    world = 2
    mp.start_processes(_sharded_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    circ, blocks, E, M = _sharded_job(0)
    kraus, _ = pts.presample(circ, E, 4242)
    probs = [np.abs(sv.trajectory_state(circ, kraus[i])) ** 2 for i in range(E)]

    def marg(j, traj, prefix):
        start, b = blocks[j]
        return np.array([sv.block_marginals(probs[int(i)], 8, start, b)[int(s) & ((1 << start) - 1)]
                         for i, s in zip(traj, prefix)]).reshape(len(traj), 1 << b)

    rt, rb, rc, levels, m = sampling.nbs_proportional(marg, blocks, 4242, E, total_shots=M, mult=np.ones(E))
    for k in range(world):
        r = np.load(tmp_path / f"job{k}.npz")
        assert np.array_equal(r["t"], rt) and np.array_equal(r["b"], rb) and np.array_equal(r["c"], rc)
    n0, n1 = np.load(tmp_path / "job0.npz")["nets"], np.load(tmp_path / "job1.npz")["nets"]
    assert (n0 + n1)[0] == E and (n0 + n1)[1:].tolist() == levels[1:]
    assert rc.sum() == M


def test_traj_range_and_local_comm():
    assert [shard.traj_range(r, 3, 10) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert shard.traj_range(0, 1, 5) == (0, 5)
    with pytest.raises(ValueError):
        shard.traj_range(2, 2, 5)
    from oracle import pts
    circ, blocks, E, M = _sharded_job(0)
    full, _ = pts.presample(circ, E, 9)
    part, _ = pts.presample(circ, 5, 9, traj0=4)
    assert np.array_equal(part, full[4:9])
    (t, b, c), nets = shard.sharded_proportional(OracleBackend(circ, blocks), shard.LocalComm(), blocks, E, M, 4242)
    assert c.sum() == M and nets[0] <= E
