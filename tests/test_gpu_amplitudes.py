"""Amplitude-level GPU parity: the trajectory states psi_i contracted by the
library's kernels (ptn_trajectory_amplitudes: the ket network of the whole
circuit with the sampled Kraus operators merged into their gates, one path for
every error set) against complex128 state vectors of the oracle.

Tolerance: norm-wise ||a_gpu - a_ref|| / ||a_ref|| <= 1e-5 per trajectory in
the FP32 modes (complex64 storage, FP32 or FP16 hi/lo tensor-core operands);
the BF16 hi/lo split keeps 16 significand bits per product, so its bound is
1e-4 (its measured error is stated by the test's assertion message)."""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"
BOUND = {ptn.PTN_PREC_FP32: 1e-5, ptn.PTN_PREC_FP16X3: 1e-5, ptn.PTN_PREC_BF16X3: 1e-4}


def _amps(plan, tr, t0, n, prec=ptn.PTN_PREC_FP32):
    a = torch.empty((n, 1 << plan.n_qubits), dtype=torch.complex64, device=DEV)
    ptn.ptn_trajectory_amplitudes(plan, tr, t0, n, a, precision=prec)
    torch.cuda.synchronize()
    return a.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    # a zero-norm trajectory (amplitude damping can annihilate a state) is
    # compared absolutely: its amplitudes must vanish
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-12)


CIRCUITS = [
    ("brick6_dep_ad", lambda r: W.attach_noise(W.brickwork_1d(6, 5, r), [W.depolarizing_kraus(0.2),
                                                                      W.amplitude_damping_kraus(0.3)]), 16),
    ("grid3x4", lambda r: W.attach_noise(W.grid_4colour(3, 4, 6, r), [W.depolarizing_kraus(0.1)]), 16),
    ("c1_brick12_d8", lambda r: W.config_c1()["circuit"], 64),
    ("brick20_d10", lambda r: W.attach_noise(W.brickwork_1d(20, 10, r), [W.depolarizing_kraus(0.01),
                                                                      W.amplitude_damping_kraus(0.01)]), 6),
    ("c5_hea16_l6", lambda r: W.config_c5()["circuit"], 5),
]


@pytest.mark.parametrize("name,make,n_traj", CIRCUITS, ids=[c[0] for c in CIRCUITS])
def test_amplitudes_match_statevector(name, make, n_traj):
    circ = make(np.random.default_rng(4242))
    plan = ptn.ptn_plan_path(circ, None, hypersamples=8, est_traj=n_traj)
    tr = ptn.ptn_presample_trajectories(plan, 17, n_traj)
    kraus = tr.to_torch()[0].cpu().numpy()
    got = _amps(plan, tr, 0, n_traj)
    want = np.array([sv.trajectory_state(circ, kraus[t]) for t in range(n_traj)])
    err = _rel(got, want)
    assert np.max(err) <= 1e-5, (name, float(np.max(err)))
    # the norm is the trajectory weight w_i (1 for unitary insertions)
    np.testing.assert_allclose(np.sum(np.abs(got) ** 2, axis=1), np.sum(np.abs(want) ** 2, axis=1), rtol=2e-5)


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3, ptn.PTN_PREC_BF16X3],
                         ids=["fp32", "fp16x3", "bf16x3"])
def test_amplitude_error_by_precision(prec):
    """16-qubit ansatz and 20-qubit brickwork: the tensor-core steps of the
    state's path run in each operand split; the error stays within the
    mode's bound."""
    rng = np.random.default_rng(99)
    for circ, n_traj in [(W.config_c5()["circuit"], 4),
                         (W.attach_noise(W.brickwork_1d(20, 10, rng), [W.depolarizing_kraus(0.01)]), 3)]:
        plan = ptn.ptn_plan_path(circ, None, hypersamples=8, est_traj=1024)
        d = plan.describe(detail=2)
        tr = ptn.ptn_presample_trajectories(plan, 5, n_traj)
        kraus = tr.to_torch()[0].cpu().numpy()
        got = _amps(plan, tr, 0, n_traj, prec)
        want = np.array([sv.trajectory_state(circ, kraus[t]) for t in range(n_traj)])
        err = float(np.max(_rel(got, want)))
        assert err <= BOUND[prec], (prec, circ.n_qubits, err)
        assert sum(1 for st in d["expval"]["steps"] if st["kind"] != 0) > 0


def test_amplitude_ranges_and_edges():
    rng = np.random.default_rng(5)
    circ = W.attach_noise(W.brickwork_1d(8, 4, rng), [W.depolarizing_kraus(0.1)])
    plan = ptn.ptn_plan_path(circ, None, hypersamples=4, est_traj=32)
    tr = ptn.ptn_presample_trajectories(plan, 3, 32)
    full = _amps(plan, tr, 0, 32)
    part = _amps(plan, tr, 29, 3)
    np.testing.assert_allclose(part, full[29:32], rtol=0, atol=1e-6 * np.abs(full).max())
    empty = torch.empty((0, 256), dtype=torch.complex64, device=DEV)
    ptn.ptn_trajectory_amplitudes(plan, tr, 32, 0, empty)
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_trajectory_amplitudes(plan, tr, 30, 3, torch.empty((3, 256), dtype=torch.complex64, device=DEV))
    assert e.value.status == 1
