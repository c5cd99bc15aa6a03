"""One proportional NBS job split by trajectory range over two ranks, each a
process on the same GPU with a gloo group on the host (the ranks exchange
only host data between launches, so none of their kernels waits on the
other): the gathered records equal the single-process ptn_sample_shots run
bit for bit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _job():
    import workloads as W
    rng = np.random.default_rng(3030)
    circ = W.attach_noise(W.brickwork_1d(20, 8, rng), [W.depolarizing_kraus(0.01), W.amplitude_damping_kraus(0.01)])
    return circ, [10, 10], 96, 200_000, 0x5EED


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2604_08467_gb300 import ptn, shard
    circ, bs, E, M, seed = _job()
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=E, est_shots=M)
    (t, b, c), nets = shard.sharded_proportional(shard.GpuBackend(plan), shard.DistComm(dist), plan.blocks, E, M,
                                                 seed)
    np.savez(os.path.join(out_dir, f"gpu_job{rank}.npz"), t=t, b=b, c=c, nets=np.array(nets))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_job_matches_single_process(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    from paper_2604_08467_gb300 import ptn
    circ, bs, E, M, seed = _job()
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=E, est_shots=M)
    tr = ptn.ptn_presample_trajectories(plan, seed, E)
    res = ptn.ptn_sample_shots(plan, tr, seed, total_shots=M)
    t, b, c = [x.cpu().numpy() for x in res.to_torch()]
    # the two ranks' ranges drawn with global counters are the rows of the full draw
    kr = tr.to_torch()[0].cpu().numpy()
    half = ptn.ptn_presample_range(plan, seed, E // 2, E - E // 2)
    assert np.array_equal(half.to_torch()[0].cpu().numpy(), kr[E // 2:])
    assert np.array_equal(half.to_torch()[3].cpu().numpy(), np.arange(E // 2, E))
    for k in range(world):
        r = np.load(tmp_path / f"gpu_job{k}.npz")
        assert np.array_equal(r["t"], t) and np.array_equal(r["b"].astype(np.int64), b) and np.array_equal(r["c"], c)
    nets = np.load(tmp_path / "gpu_job0.npz")["nets"] + np.load(tmp_path / "gpu_job1.npz")["nets"]
    assert nets.tolist() == res.nets_per_block
    assert c.sum() == M
