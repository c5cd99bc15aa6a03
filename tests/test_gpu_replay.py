"""End-to-end replay of proportional NBS against the oracle.

Two checks per workload (the tie/boundary reading in tests/replay_check.py):
  1. the GPU's shot list equals, record for record, the oracle's NBS procedure
     run on the marginals the GPU itself contracts for the same networks
     (ptn_contract_batch): allocation, Philox draws, CDF search, prefix
     dedup and canonical order are then bit-exact;
  2. on every level's parents, the draws made from the GPU's complex64
     marginals and from the oracle's complex128 marginals differ only for
     draws that lie within delta of the boundary between the two bins
     (delta = L1 distance of the normalised rows), and rarely.
Together these pin every shot of the end-to-end run to the complex128
oracle up to near-boundary events."""
import numpy as np
import pytest

import workloads as W
from oracle import philox, sampling, statevector as sv

from replay_check import boundary_mismatches, nbs_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _gpu_rows(plan, tr):
    def rows(j, traj, prefix):
        start, b = plan.blocks[j]
        nt = torch.tensor(np.asarray(traj, np.int64), dtype=torch.int32, device=DEV)
        npre = torch.tensor(np.asarray(prefix, np.uint64).astype(np.int64), dtype=torch.int64, device=DEV)
        marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device=DEV)
        Z = torch.empty(len(traj), dtype=torch.float64, device=DEV)
        ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z)
        torch.cuda.synchronize()
        rows.Z = Z.cpu().numpy()
        return marg.cpu().numpy().astype(np.float64)
    return rows


def _sv_rows(circ, kraus, blocks):
    n = circ.n_qubits
    probs = [np.abs(sv.trajectory_state(circ, kraus[i])) ** 2 for i in range(len(kraus))]
    tables = {}

    def rows(j, traj, prefix):
        start, b = blocks[j]
        out = []
        for i, s in zip(traj, prefix):
            key = (int(i), j)
            if key not in tables:
                tables[key] = sv.block_marginals(probs[int(i)], n, start, b)
            out.append(tables[key][int(s) & ((1 << start) - 1)])
        return np.array(out)
    return rows


def _check(res, plan, tr, circ, seed, m, circuit=0, max_rate=1e-3):
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    (rt, rb, rc), levels = nbs_levels(_gpu_rows(plan, tr), plan.blocks, seed, m, circuit)
    assert np.array_equal(t, rt) and np.array_equal(bits.astype(np.uint64), rb) and np.array_equal(cnt, rc)
    assert res.nets_per_block == [len(lv[0]) for lv in levels]
    kraus = tr.to_torch()[0].cpu().numpy()
    ref = _sv_rows(circ, kraus, plan.blocks)
    tot_d = tot_m = 0
    for j, (lt, lp, lc, rows_gpu) in enumerate(levels):
        d, mm, worst = boundary_mismatches(rows_gpu, ref(j, lt, lp), lt, lc, seed, j, circuit)
        assert worst <= 1.0, (j, worst)
        tot_d += d
        tot_m += mm
    assert tot_m <= max_rate * tot_d, (tot_m, tot_d)
    return tot_d, tot_m


def test_replay_small_fixed_shots():
    rng = np.random.default_rng(77)
    circ = W.attach_noise(W.brickwork_1d(8, 5, rng), [W.depolarizing_kraus(0.05)])
    plan = ptn.ptn_plan_path(circ, [3, 3, 2], hypersamples=8, est_traj=8, est_shots=4000)
    tr = ptn.ptn_presample_trajectories(plan, 21, 8)
    res = ptn.ptn_sample_shots(plan, tr, 99, shots_per_traj=500)
    _check(res, plan, tr, circ, 99, [500] * 8)


def test_replay_c1_brickwork12():
    """12-qubit brickwork, depth 8, 64 trajectories x 1000 shots, blocks 10/2."""
    cfg = W.config_c1()
    circ = cfg["circuit"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=64, est_shots=64000)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    res = ptn.ptn_sample_shots(plan, tr, cfg["seed"], shots_per_traj=1000)
    d, _ = _check(res, plan, tr, circ, cfg["seed"], [1000] * 64)
    assert d == 2 * 64_000


def test_replay_mixed_batch_item_proportional_total():
    """The 20-qubit item of the mixed workload run through the batch executor
    with proportional allocation of its 13817 shots: allocation and sampling
    replayed exactly on the GPU's own weights and marginals, and allocation
    draws from GPU vs complex128 trajectory weights differ only near
    boundaries."""
    cfg = {c["name"]: c for c in W.config_c3()}["c3_58_brickwork20q_d8"]
    circ, E, M, cid = cfg["circuit"], cfg["n_traj"], cfg["total_shots"], cfg["circuit_id"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=E)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], E, dedup=False, circuit_id=cid)
    (st, shots), = ptn.ptn_sample_shots_batch([dict(plan=plan, traj=tr, seed=cfg["seed"], total_shots=M,
                                                    circuit_id=cid)])
    assert st == 0
    rows = _gpu_rows(plan, tr)
    rows(0, np.arange(E), np.zeros(E, np.uint64))
    w_gpu = rows.Z.copy()
    m = sampling.allocate_shots(w_gpu, M, cfg["seed"], cid)
    _check(shots, plan, tr, circ, cfg["seed"], m, circuit=cid)
    kraus = tr.to_torch()[0].cpu().numpy()
    w_ref = np.array([np.sum(np.abs(sv.trajectory_state(circ, kraus[i])) ** 2) for i in range(E)])
    d, mm, worst = boundary_mismatches(w_gpu[None, :], w_ref[None, :], np.zeros(1, np.int64), np.array([M]),
                                       cfg["seed"], 0, cid, stream=philox.STREAM_ALLOC)
    assert d == M and worst <= 1.0 and mm <= 1e-3 * M
