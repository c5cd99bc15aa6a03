"""GPU parity of the ket-only network form (plan option network_form): a block
lowered as the ket network of the block and later qubits (prefix projected)
plus a closing step that sums |a|^2 over the later qubits must give the same
marginals as the double layer, within the same norm-wise 2e-5 bound against
the complex128 oracle.  Form 0 (AUTO) picks per block the cheaper of the two
forms by the cost model, form 2 takes the ket-only form wherever it has a
path."""
import numpy as np
import pytest

import workloads as W
from oracle import mps, statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _contract(plan, tr, j, traj, prefix, b):
    nt = torch.tensor(traj, dtype=torch.int32, device=DEV)
    npre = torch.tensor(np.asarray(prefix, dtype=np.int64), dtype=torch.int64, device=DEV)
    marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device=DEV)
    Z = torch.empty(len(traj), dtype=torch.float64, device=DEV)
    ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z)
    torch.cuda.synchronize()
    return marg.cpu().numpy().astype(np.float64), Z.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-12)


def _ket_blocks(plan):
    return [b["ket_only"] for b in plan.describe()["blocks"]]


SMALL = [
    ("brick6", lambda r: W.attach_noise(W.brickwork_1d(6, 5, r), [W.depolarizing_kraus(0.2),
                                                               W.amplitude_damping_kraus(0.3)]), [2, 3, 1]),
    ("grid3x4", lambda r: W.attach_noise(W.grid_4colour(3, 4, 6, r), [W.depolarizing_kraus(0.1)]), [5, 7]),
    ("hea6", lambda r: W.attach_noise(W.hea_ring(6, 3, r.standard_normal(36)), [W.depolarizing_kraus(0.05)]),
     [3, 2, 1]),
]


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("name,make,bs", SMALL, ids=[c[0] for c in SMALL])
def test_forms_small_circuits(name, make, bs, form):
    rng = np.random.default_rng(len(name) * 7919)
    circ = make(rng)
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=16, est_shots=256, network_form=form)
    if form == 2:
        assert all(_ket_blocks(plan)), name
    tr = ptn.ptn_presample_trajectories(plan, 11, 16)
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(16)]
    prng = np.random.default_rng(3)
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(16), 5)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        marg, Z = _contract(plan, tr, j, traj, prefix, b)
        want = np.array([sv.block_marginals(probs[t], circ.n_qubits, start, b)[int(s)]
                         for t, s in zip(traj, prefix)])
        assert np.max(_rel(marg, want)) < 2e-5, (name, j)
        np.testing.assert_allclose(Z, want.sum(axis=1), rtol=2e-5, atol=1e-12)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_forms_c1_all_blocks(form):
    """12-qubit brickwork (depth 8, 64 trajectories): block 1 for every
    trajectory, block 2 for ragged prefix sets, in the ket-only forms."""
    cfg = W.config_c1()
    circ = cfg["circuit"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=64, est_shots=64000,
                             network_form=form)
    if form == 2:
        assert all(_ket_blocks(plan))
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(64)]
    marg, Z = _contract(plan, tr, 0, np.arange(64), np.zeros(64, int), 10)
    want = np.array([sv.block_marginals(p, 12, 0, 10)[0] for p in probs])
    assert np.max(_rel(marg, want)) < 2e-5
    traj, prefix = [], []
    prng = np.random.default_rng(9)
    for t in range(64):
        for _ in range(t % 7):
            traj.append(t)
            prefix.append(int(prng.integers(0, 1024)))
    marg2, Z2 = _contract(plan, tr, 1, np.array(traj), np.array(prefix), 2)
    want2 = np.array([sv.block_marginals(probs[t], 12, 10, 2)[s] for t, s in zip(traj, prefix)])
    assert np.max(_rel(marg2, want2)) < 2e-5
    np.testing.assert_allclose(Z2, [want[t][s] for t, s in zip(traj, prefix)], rtol=2e-5, atol=1e-12)


def test_form1_c2_sampled_networks_vs_mps():
    """30-qubit brickwork (depth 12, 4096 trajectories) planned with form AUTO,
    whose last block takes the ket-only form; sampled networks of every block
    against the exact-MPS oracle, launched over the full trajectory set."""
    cfg = W.config_c2()
    circ = cfg["circuit"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=cfg["n_traj"],
                             est_shots=cfg["total_shots"], network_form=0)
    kb = _ket_blocks(plan)
    assert kb[-1] == 1
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    kraus = tr.to_torch()[0].cpu().numpy()
    pick = [0, 5, 2048, 4095]
    states = {t: mps.trajectory_mps(circ, kraus[t]) for t in pick}
    marg, _ = _contract(plan, tr, 0, np.arange(4096), np.zeros(4096, int), 10)
    for t in pick:
        assert _rel(marg[t], states[t].block_marginal(0, 10, 0)) < 2e-5
    prng = np.random.default_rng(14)
    for j in (1, 2):
        start = 10 * j
        # every trajectory has networks here, so the launch spans the full batch
        traj = np.repeat(np.arange(4096), 2)
        prefix = prng.integers(0, 1 << start, size=len(traj))
        m, Z = _contract(plan, tr, j, traj, prefix, 10)
        assert np.all(np.isfinite(m)) and np.allclose(Z, m.sum(axis=1), rtol=1e-9)
        for t in pick:
            for n in np.nonzero(traj == t)[0]:
                want = states[t].block_marginal(start, 10, int(prefix[n]))
                assert _rel(m[n], want) < 2e-5, (j, t)


def test_form2_tensor_core_plan_vs_statevector():
    """20-qubit brickwork with every block in the ket-only form and tensor-core
    (tcgen05) steps in its paths, every block against c128 state vectors."""
    rng = np.random.default_rng(2020)
    circ = W.attach_noise(W.brickwork_1d(20, 10, rng), [W.depolarizing_kraus(0.01),
                                                         W.amplitude_damping_kraus(0.01)])
    plan = ptn.ptn_plan_path(circ, [10, 6, 4], hypersamples=16, est_traj=512, est_shots=1e5, network_form=2)
    d = plan.describe()
    assert sum(b["n_gemm"] for b in d["blocks"]) > 0
    assert any(b["ket_only"] for b in d["blocks"])
    tr = ptn.ptn_presample_trajectories(plan, 31, 6)
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(6)]
    prng = np.random.default_rng(8)
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(6), 7)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        marg, _ = _contract(plan, tr, j, traj, prefix, b)
        want = np.array([sv.block_marginals(probs[t], 20, start, b)[int(s)] for t, s in zip(traj, prefix)])
        assert np.max(_rel(marg, want)) < 2e-5, j


def test_form1_end_to_end_distribution():
    """Proportional NBS through ptn_sample_shots with the ket-only form: every
    shot accounted for and 4-qubit marginals within TVD 3/sqrt(shots) of the
    exact trajectory mixture."""
    cfg = W.config_c1()
    circ = cfg["circuit"]
    plan = ptn.ptn_plan_path(circ, [4, 4, 4], hypersamples=16, est_traj=64, est_shots=64000, network_form=2)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    res = ptn.ptn_sample_shots(plan, tr, cfg["seed"], shots_per_traj=1000)
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    assert cnt.sum() == 64_000
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = np.mean([np.abs(sv.trajectory_state(circ, kraus[i])) ** 2 for i in range(64)], axis=0)
    emp = np.zeros(1 << 12)
    np.add.at(emp, bits.astype(np.int64), cnt)
    emp /= emp.sum()
    idx = np.arange(1 << 12)
    for qs in ([0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 10, 11], [1, 4, 7, 10]):
        key = sum(((idx >> q) & 1) << k for k, q in enumerate(qs))
        pe = np.bincount(key, weights=emp, minlength=16)
        pq = np.bincount(key, weights=probs, minlength=16)
        assert 0.5 * np.abs(pe - pq).sum() < 3 / np.sqrt(64_000)
