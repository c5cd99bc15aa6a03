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
