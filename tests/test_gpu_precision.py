"""Precision study (GPU): tensor-core contractions in the three precision
modes against the complex128 oracle on the 16-qubit (4x4 grid, depth 10)
slice of the grid family: per-network marginal error and the sampled
distribution's TVD.  The measured errors are printed (pytest -s) and bounded
by what each mode's arithmetic allows:
  FP32 (TF32 hi/lo split, ~2^-24 per product):   2e-5 (as every FP32 test)
  FP16X3 (FP16 hi/lo, 22 bits, scaled):           2e-5
  BF16X3 (BF16 hi/lo, 16 bits):                   1e-4
"""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

BOUND = {ptn.PTN_PREC_FP32: 2e-5, ptn.PTN_PREC_FP16X3: 2e-5, ptn.PTN_PREC_BF16X3: 1e-4}
NAME = {ptn.PTN_PREC_FP32: "fp32", ptn.PTN_PREC_FP16X3: "fp16x3", ptn.PTN_PREC_BF16X3: "bf16x3"}


@pytest.fixture(scope="module")
def slice16():
    cfg = W.config_c4_slice()
    circ = cfg["circuit"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=2048, est_shots=2 ** 20)
    assert sum(b["n_gemm"] for b in plan.describe()["blocks"]) > 0
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], 24)
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(24)]
    return cfg, plan, tr, probs


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3, ptn.PTN_PREC_BF16X3])
def test_marginal_error_by_precision(slice16, prec):
    cfg, plan, tr, probs = slice16
    prng = np.random.default_rng(1)
    worst = 0.0
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(24), 3)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        nt = torch.tensor(traj, dtype=torch.int32, device="cuda")
        npf = torch.tensor(prefix, dtype=torch.int64, device="cuda")
        marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device="cuda")
        Z = torch.empty(len(traj), dtype=torch.float64, device="cuda")
        ptn.ptn_contract_batch(plan, tr, j, nt, npf, marg, Z, precision=prec)
        got = marg.cpu().numpy().astype(np.float64)
        want = np.array([sv.block_marginals(probs[t], 16, start, b)[int(s)] for t, s in zip(traj, prefix)])
        assert np.all(np.isfinite(got))
        err = np.linalg.norm(got - want, axis=1) / np.maximum(np.linalg.norm(want, axis=1), 1e-12)
        worst = max(worst, float(err.max()))
    print(f"\n[precision] {NAME[prec]}: max norm-wise marginal error {worst:.3e}")
    assert worst < BOUND[prec]


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_BF16X3])
def test_sampled_tvd_by_precision(slice16, prec):
    cfg, plan, tr, probs = slice16
    shots = 4000
    res = ptn.ptn_sample_shots(plan, tr, 77, shots_per_traj=shots, precision=prec)
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    assert cnt.sum() == 24 * shots
    mix = np.mean([p / p.sum() for p in probs], axis=0)
    emp = np.zeros(1 << 16)
    np.add.at(emp, bits.astype(np.int64), cnt)
    emp /= emp.sum()
    N = 24 * shots
    idx = np.arange(1 << 16)
    for qs in ([0, 1, 2, 3], [5, 6, 9, 10], [12, 13, 14, 15]):
        key = sum(((idx >> q) & 1) << k for k, q in enumerate(qs))
        pe = np.bincount(key, weights=emp, minlength=16)
        pq = np.bincount(key, weights=mix, minlength=16)
        tvd = 0.5 * np.abs(pe - pq).sum()
        print(f"\n[precision] {NAME[prec]}: TVD on qubits {qs} = {tvd:.4f} (bound {3 / np.sqrt(N):.4f})")
        assert tvd < 3 / np.sqrt(N)


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3, ptn.PTN_PREC_BF16X3])
def test_c2_marginal_error_by_precision(prec):
    """The 30-qubit brickwork workload (4096 trajectories, launched as in the
    benchmark) in each precision mode: sampled networks of every block against
    the exact-MPS oracle, within the mode's bound."""
    from oracle import mps
    cfg = W.config_c2()
    circ = cfg["circuit"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=100, est_traj=cfg["n_traj"],
                             est_shots=cfg["total_shots"])
    # the benchmark's plan: its middle block packs rows of 2^14 complex slots
    # (FP16: one row over a cluster of four CTAs)
    assert max(s["n_sum"] for s in plan.describe(1)["blocks"][1]["steps"] if s["kind"]) >= 13
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    kraus = tr.to_torch()[0].cpu().numpy()
    pick = [0, 2049, 4095]
    states = {t: mps.trajectory_mps(circ, kraus[t]) for t in pick}
    prng = np.random.default_rng(6)
    worst = 0.0
    for j in range(3):
        start = 10 * j
        traj = np.arange(4096) if j == 0 else np.repeat(pick, 3)
        prefix = np.zeros(len(traj), int) if j == 0 else prng.integers(0, 1 << start, size=len(traj))
        nt = torch.tensor(traj, dtype=torch.int32, device="cuda")
        npf = torch.tensor(prefix, dtype=torch.int64, device="cuda")
        marg = torch.empty((len(traj), 1024), dtype=torch.float32, device="cuda")
        Z = torch.empty(len(traj), dtype=torch.float64, device="cuda")
        ptn.ptn_contract_batch(plan, tr, j, nt, npf, marg, Z, precision=prec)
        got = marg.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        rows = range(len(traj)) if j else pick
        for n in rows:
            t, s = int(traj[n]), int(prefix[n])
            want = states[t].block_marginal(start, 10, s)
            worst = max(worst, float(np.linalg.norm(got[n] - want) / max(np.linalg.norm(want), 1e-12)))
    print(f"\n[precision c2] {NAME[prec]}: max norm-wise marginal error {worst:.3e}")
    assert worst < BOUND[prec]
