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
