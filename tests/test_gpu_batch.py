"""GPU tests of the mixed-circuit batch executor (ptn_sample_shots_batch):
circuits of different qubit counts, depths, trajectory counts and shot
budgets from the mixed workload, run concurrently.  Every item must give
exactly the result of its own ptn_sample_shots call (same kernels, same
Philox counters, so bit-identical), over-budget circuits must come back as
PTN_ERR_TOO_LARGE without stopping the others (one item is replayed against
the oracle in test_gpu_replay.py)."""
import numpy as np
import pytest

import workloads as W


torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

TOO_LARGE = 3


def _c3(names):
    cfgs = {c["name"]: c for c in W.config_c3()}
    return [cfgs[n] for n in names]


def _prepare(cfg):
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=16, est_traj=cfg["n_traj"],
                             est_shots=cfg["total_shots"])
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"], dedup=True, circuit_id=cfg["circuit_id"])
    return plan, tr


def _host(shots):
    return [x.cpu().numpy() for x in shots.to_torch()]


SMALL_1D = ["c3_58_brickwork20q_d8", "c3_5_brickwork35q_d9", "c3_44_brickwork33q_d10", "c3_62_brickwork30q_d9",
            "c3_31_brickwork36q_d10", "c3_37_brickwork27q_d9"]


def test_batch_matches_individual_calls():
    cfgs = _c3(SMALL_1D)
    prepared = [_prepare(c) for c in cfgs]
    items = [dict(plan=p, traj=t, seed=c["seed"], total_shots=c["total_shots"], circuit_id=c["circuit_id"])
             for c, (p, t) in zip(cfgs, prepared)]
    out = ptn.ptn_sample_shots_batch(items, n_workers=3)
    torch.cuda.synchronize()
    assert [s for s, _ in out] == [0] * len(items)
    for c, (p, t), (_, shots) in zip(cfgs, prepared, out):
        ref = ptn.ptn_sample_shots(p, t, c["seed"], total_shots=c["total_shots"], circuit_id=c["circuit_id"])
        a, b = _host(shots), _host(ref)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), c["name"]
        assert a[2].sum() == c["total_shots"]


def test_batch_over_budget_items_fail_alone():
    """Grid circuits beyond the time budget (modelled 19.3 s and 98.9 s against
    15 s) or the memory cap come back as TOO_LARGE; the 1D circuits in the
    same batch still complete."""
    cfgs = _c3(["c3_3_grid6x5_d8", "c3_58_brickwork20q_d8", "c3_0_grid6x5_d10", "c3_62_brickwork30q_d9"])
    prepared = [_prepare(c) for c in cfgs]
    items = [dict(plan=p, traj=t, seed=c["seed"], total_shots=c["total_shots"], circuit_id=c["circuit_id"])
             for c, (p, t) in zip(cfgs, prepared)]
    out = ptn.ptn_sample_shots_batch(items, n_workers=2, max_est_seconds=15.0)
    st = [s for s, _ in out]
    assert st[0] == TOO_LARGE and st[2] == TOO_LARGE
    assert st[1] == 0 and st[3] == 0
    for k in (1, 3):
        assert _host(out[k][1])[2].sum() == cfgs[k]["total_shots"]
    # without the time guard the first grid (28 GB per trajectory) fails on the memory cap
    out2 = ptn.ptn_sample_shots_batch(items[:1], n_workers=4, mem_budget_bytes=8e9)
    assert out2[0][0] == TOO_LARGE


def test_batch_items_sharing_a_plan():
    cfg = _c3(["c3_44_brickwork33q_d10"])[0]
    plan, tr = _prepare(cfg)
    tr2 = ptn.ptn_presample_trajectories(plan, cfg["seed"] + 1, 50, dedup=False, circuit_id=cfg["circuit_id"])
    items = [dict(plan=plan, traj=tr, seed=11, total_shots=3000, circuit_id=cfg["circuit_id"]),
             dict(plan=plan, traj=tr2, seed=12, shots_per_traj=40, circuit_id=cfg["circuit_id"])]
    out = ptn.ptn_sample_shots_batch(items, n_workers=4)
    assert [s for s, _ in out] == [0, 0]
    r1 = ptn.ptn_sample_shots(plan, tr, 11, total_shots=3000, circuit_id=cfg["circuit_id"])
    r2 = ptn.ptn_sample_shots(plan, tr2, 12, shots_per_traj=40, circuit_id=cfg["circuit_id"])
    for (_, s), r in zip(out, (r1, r2)):
        for x, y in zip(_host(s), _host(r)):
            assert np.array_equal(x, y)


def test_batch_empty_and_bad_arguments():
    assert ptn.ptn_sample_shots_batch([]) == []
    cfg = _c3(["c3_58_brickwork20q_d8"])[0]
    p1, t1 = _prepare(cfg)
    p2, t2 = _prepare(cfg)
    with pytest.raises(ptn.PtnError):
        ptn.ptn_sample_shots_batch([dict(plan=p1, traj=t2, seed=1, total_shots=10)])
