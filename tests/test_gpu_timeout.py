"""A bounded device wait that runs out: with the tensor-core kernel's wait
limit set to zero its pipeline waits give up, the kernel stops, drains its own
copies and MMAs, frees its tensor memory and the call returns PTN_ERR_TIMEOUT;
with the default limit restored the same contraction runs again on the same
context and gives exactly the result it gave before."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

TIMEOUT = 6


def test_wait_limit_zero_times_out_and_device_recovers():
    cfg = W.config_c2()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=100, est_traj=4096, est_shots=1e6)
    # a tensor-core step with a long contraction (the epilogue waits for many MMAs)
    assert max(s["n_sum"] for s in plan.describe(1)["blocks"][1]["steps"] if s["kind"]) >= 10
    tr = ptn.ptn_presample_trajectories(plan, 3, 8)
    traj = torch.tensor(np.repeat(np.arange(8), 4), dtype=torch.int32, device="cuda")
    prefix = torch.tensor(np.random.default_rng(1).integers(0, 1 << 10, size=32), dtype=torch.int64, device="cuda")

    def run():
        marg = torch.empty((32, 1024), dtype=torch.float32, device="cuda")
        Z = torch.empty(32, dtype=torch.float64, device="cuda")
        ptn.ptn_contract_batch(plan, tr, 1, traj, prefix, marg, Z)
        torch.cuda.synchronize()
        return marg.cpu().numpy()

    before = run()
    ptn.ptn_set_wait_limit(0.0)
    try:
        with pytest.raises(ptn.PtnError) as e:
            run()
        assert e.value.status == TIMEOUT and "timed out" in str(e.value)
    finally:
        ptn.ptn_set_wait_limit(2.0)
    torch.cuda.synchronize()
    after = run()
    assert np.array_equal(before, after)
    with pytest.raises(ptn.PtnError):
        ptn.ptn_set_wait_limit(-1.0)
