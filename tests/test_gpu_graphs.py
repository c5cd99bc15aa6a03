"""CUDA-graph execution of the contraction (ptn_sample_opts.use_graphs): every
chunk's launches are recorded and launched as one graph whose executable is
updated in place from chunk to chunk and call to call.  The kernels and their
arguments are the same as without graphs, so every record must be identical:
proportional sampling at 12 and 30 qubits in FP32 and FP16x3, the plain
per-trajectory path (one chunk per trajectory, so the executable graph is
updated many times per block), repeated calls on one plan, and
non-proportional sampling."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402


def _host(res):
    return [x.cpu().numpy() for x in res.to_torch()]


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_graphs_c1_fixed_and_plain_path():
    cfg = W.config_c1()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=8, est_traj=64, est_shots=64000)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    ref = _host(ptn.ptn_sample_shots(plan, tr, 5, shots_per_traj=1000))
    for rep in range(2):   # the second call updates the kept executable graphs
        _same(_host(ptn.ptn_sample_shots(plan, tr, 5, shots_per_traj=1000, use_graphs=1)), ref)
    plain = _host(ptn.ptn_sample_shots(plan, tr, 5, shots_per_traj=1000, max_traj_per_chunk=1))
    _same(plain, ref)
    _same(_host(ptn.ptn_sample_shots(plan, tr, 5, shots_per_traj=1000, max_traj_per_chunk=1, use_graphs=1)), ref)


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3])
def test_graphs_c2_total_shots(prec):
    """The 30-qubit benchmark plan with 64 trajectories: tensor-core steps
    (TMA descriptors, stacked tile tables, pack kernels) and fused small-step
    runs inside the graphs."""
    cfg = W.config_c2()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=100, est_traj=4096, est_shots=1e6)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], 64)
    ref = _host(ptn.ptn_sample_shots(plan, tr, 9, total_shots=15616, precision=prec))
    got = _host(ptn.ptn_sample_shots(plan, tr, 9, total_shots=15616, precision=prec, use_graphs=1))
    _same(got, ref)
    assert ref[2].sum() == 15616


def test_graphs_nonproportional():
    rng = np.random.default_rng(2626)
    circ = W.attach_noise(W.brickwork_1d(20, 8, rng), [W.depolarizing_kraus(0.01)])
    plan = ptn.ptn_plan_path(circ, [6, 14], hypersamples=16, est_traj=8, est_shots=64)
    tr = ptn.ptn_presample_trajectories(plan, 5, 8)
    a = ptn.ptn_sample_nonprop(plan, tr, 31, mode="exhaustive", branch_shots=2, threshold=1e-4)
    b = ptn.ptn_sample_nonprop(plan, tr, 31, mode="exhaustive", branch_shots=2, threshold=1e-4, use_graphs=1)
    _same(_host(a), _host(b))
    assert np.array_equal(a.probs().cpu().numpy(), b.probs().cpu().numpy())


def test_graphs_flag_checked():
    cfg = W.config_c1()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=2, est_traj=4, est_shots=40)
    tr = ptn.ptn_presample_trajectories(plan, 1, 4)
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_sample_shots(plan, tr, 1, shots_per_traj=10, use_graphs=2)
    assert e.value.status == 1
