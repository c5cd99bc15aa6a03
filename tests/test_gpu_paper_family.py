"""The paper's own benchmark circuit family on the GPU (random circuits of
{H, X, Y, Z, T, Rx} and nearest-neighbour {CX, CY, CZ, CH, CRx} at 20%, a
single Pauli error channel after every one-qubit gate and a two-qubit
depolarizing channel after every two-qubit gate, p ~ U[0.02, 0.2]): Kraus
draws of the 16-operator two-qubit channel bit-exact, block marginals against
complex128 state vectors and exact-MPS contractions, and the paper's sampling
regime (blocks of 10, one shot per non-final block, exhaustive final block)
replayed exactly by the oracle on the GPU's marginals."""
import numpy as np
import pytest

import workloads as W
from oracle import mps, pts, sampling, statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _contract(plan, tr, j, traj, prefix, b):
    nt = torch.tensor(np.asarray(traj, np.int64), dtype=torch.int32, device=DEV)
    npre = torch.tensor(np.asarray(prefix, np.uint64).astype(np.int64), dtype=torch.int64, device=DEV)
    marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device=DEV)
    Z = torch.empty(len(traj), dtype=torch.float64, device=DEV)
    ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z)
    torch.cuda.synchronize()
    return marg.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-12)


@pytest.mark.parametrize("split", [1, 0])
def test_paper_family_small_vs_statevector(split):
    rng = np.random.default_rng(1616)
    circ = W.paper_random_circuit(16, 90, rng)
    assert any(s.qubit < 0 for s in circ.sites)
    plan = ptn.ptn_plan_path(circ, [10, 6], hypersamples=16, split_gates=split, est_traj=32, est_shots=1e4)
    tr = ptn.ptn_presample_trajectories(plan, 77, 32)
    kraus = tr.to_torch()[0].cpu().numpy()
    k_ref, _ = pts.presample(circ, 32, 77)
    assert np.array_equal(kraus, k_ref) and kraus.max() >= 4       # two-qubit channels draw up to 15
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(32)]
    prng = np.random.default_rng(2)
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(32), 3)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        got = _contract(plan, tr, j, traj, prefix, b)
        want = np.array([sv.block_marginals(probs[t], 16, start, b)[int(s)] for t, s in zip(traj, prefix)])
        assert np.max(_rel(got, want)) < 2e-5, j


def test_paper_family_50q_vs_mps_and_nonprop_replay():
    """50 qubits, 200 gates (the paper's smallest configuration), blocks of 10
    and a final block of 20: sampled networks against exact MPS, then one
    shot per non-final block and an exhaustive final harvest replayed by the
    oracle on the GPU's marginals."""
    cfg = W.config_paper(50, 200)
    circ = cfg["circuit"]
    bs = [10, 10, 10, 20]
    E = 12
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=16, est_traj=E, est_shots=E)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], E)
    kraus = tr.to_torch()[0].cpu().numpy()
    pick = [0, 7]
    states = {t: mps.trajectory_mps(circ, kraus[t]) for t in pick}
    prng = np.random.default_rng(6)
    for j, (start, b) in enumerate(plan.blocks[:3]):
        traj = np.repeat(pick, 2)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        got = _contract(plan, tr, j, traj, prefix, b)
        for n, (t, s) in enumerate(zip(traj, prefix)):
            assert _rel(got[n], states[t].block_marginal(start, b, int(s))) < 2e-5, (j, t)
    res = ptn.ptn_sample_nonprop(plan, tr, 31, mode="exhaustive", threshold=1e-5)
    t, b, c = [x.cpu().numpy() for x in res.to_torch()]
    p = res.probs().cpu().numpy()

    def rows(j, traj, prefix):
        return _contract(plan, tr, j, traj, prefix, plan.blocks[j][1])

    (rt, rb, rp), nets = sampling.nbs_nonproportional(rows, plan.blocks, 31, E, mode="exhaustive", tau=1e-5)
    assert res.nets_per_block == nets
    assert np.array_equal(t, rt) and np.array_equal(b.astype(np.uint64), rb) and np.array_equal(p, rp)
    assert len(t) >= E
