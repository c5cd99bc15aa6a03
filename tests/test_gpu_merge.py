"""GPU tests of ptn_shots_merge (the emitted shots merged across
trajectories): against a NumPy aggregation of the same records, exact."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402


def _merged_ref(bits, cnt):
    u, inv = np.unique(bits, return_inverse=True)
    return u, np.bincount(inv, weights=cnt).astype(np.int64)


@pytest.mark.parametrize("mode", ["fixed", "total"])
def test_merge_matches_numpy(mode):
    cfg = W.config_c1()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=8, est_traj=64, est_shots=64000)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], 64)
    res = (ptn.ptn_sample_shots(plan, tr, cfg["seed"], shots_per_traj=1000) if mode == "fixed" else
           ptn.ptn_sample_shots(plan, tr, cfg["seed"], total_shots=50_000))
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    merged = ptn.ptn_shots_merge(res, len(plan.block_sizes))
    mt, mb, mc = [x.cpu().numpy() for x in merged.to_torch()]
    ub, uc = _merged_ref(bits.astype(np.uint64), cnt)
    assert np.array_equal(mb, ub) and np.array_equal(mc, uc)
    assert np.all(mt == -1) and mc.sum() == cnt.sum()
    assert merged.nets_per_block == res.nets_per_block


def test_merge_single_record_and_wide_bitstrings():
    """One trajectory, one shot (a single record); and a 30-qubit workload
    (four radix passes) on a few trajectories."""
    cfg = W.config_c1()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=4, est_traj=1, est_shots=1)
    tr = ptn.ptn_presample_trajectories(plan, 3, 1)
    res = ptn.ptn_sample_shots(plan, tr, 5, shots_per_traj=1)
    merged = ptn.ptn_shots_merge(res, 2)
    assert merged.n == 1
    mt, mb, mc = [x.cpu().numpy() for x in merged.to_torch()]
    assert mc.tolist() == [1]
    c2 = W.config_c2()
    plan2 = ptn.ptn_plan_path(c2["circuit"], c2["block_sizes"], hypersamples=4, est_traj=8, est_shots=4000)
    tr2 = ptn.ptn_presample_trajectories(plan2, 9, 8)
    res2 = ptn.ptn_sample_shots(plan2, tr2, 9, total_shots=4000)
    t, bits, cnt = [x.cpu().numpy() for x in res2.to_torch()]
    m2 = ptn.ptn_shots_merge(res2, 3)
    _, mb2, mc2 = [x.cpu().numpy() for x in m2.to_torch()]
    ub, uc = _merged_ref(bits.astype(np.uint64), cnt)
    assert np.array_equal(mb2, ub) and np.array_equal(mc2, uc) and mc2.sum() == 4000
