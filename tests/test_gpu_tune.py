"""Block-size autotuning on the GPU: every candidate block size is planned and
timed by a probe run; the chosen one is the fastest of the timed candidates,
and a candidate that cannot be planned is reported as +infinity."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402


def test_tune_picks_the_fastest_candidate():
    rng = np.random.default_rng(41)
    circ = W.attach_noise(W.brickwork_1d(16, 8, rng), [W.depolarizing_kraus(0.01)])
    cands = [2, 4, 8, 12]
    best, secs = ptn.ptn_tune_block_sizes(circ, cands, probe_traj=64, probe_shots=20_000, seed=3)
    assert best in cands and all(s > 0 and math.isfinite(s) for s in secs)
    assert secs[cands.index(best)] == min(secs)
    # the tuned plan samples correctly
    f = -(-16 // best)
    plan = ptn.ptn_plan_path(circ, [best] * (f - 1) + [16 - best * (f - 1)], hypersamples=16, est_traj=64)
    tr = ptn.ptn_presample_trajectories(plan, 5, 64)
    res = ptn.ptn_sample_shots(plan, tr, 5, total_shots=20_000)
    assert int(res.to_torch()[2].sum()) == 20_000


def test_tile_tuning_keeps_results_and_times_simt_steps():
    """Micro-tile autotuning of the SIMT steps of the 30-qubit benchmark plan:
    some steps are timed, and every block's marginals after tuning are
    bit-identical to those before (each output's multiply-add chain does not
    depend on the tile shape), as are the sampled records."""
    cfg = W.config_c2()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=100, est_traj=4096, est_shots=1e6)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], 32)
    prng = np.random.default_rng(8)

    def rows():
        out = []
        for j, (start, b) in enumerate(plan.blocks):
            traj = np.repeat(np.arange(32), 2)
            prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), np.int64)
            nt = torch.tensor(traj, dtype=torch.int32, device="cuda")
            npf = torch.tensor(prefix, dtype=torch.int64, device="cuda")
            marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device="cuda")
            Z = torch.empty(len(traj), dtype=torch.float64, device="cuda")
            ptn.ptn_contract_batch(plan, tr, j, nt, npf, marg, Z)
            out.append(marg.cpu().numpy())
        return out

    state = prng.bit_generator.state
    before = rows()
    rec0 = [x.cpu().numpy() for x in ptn.ptn_sample_shots(plan, tr, 3, total_shots=10_000).to_torch()]
    n_tuned, n_changed = ptn.ptn_tune_tiles(plan, tr, n_probe=32, reps=2)
    assert n_tuned > 10 and 0 <= n_changed <= n_tuned
    prng.bit_generator.state = state
    after = rows()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    rec1 = [x.cpu().numpy() for x in ptn.ptn_sample_shots(plan, tr, 3, total_shots=10_000).to_torch()]
    for a, b in zip(rec0, rec1):
        assert np.array_equal(a, b)
