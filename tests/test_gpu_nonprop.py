"""GPU parity of non-proportional NBS (ptn_sample_shots in the NONPROP modes):
branching non-final blocks and the direct / exhaustive harvest of the final
block's population vector, against the oracle (oracle.sampling.
nbs_nonproportional).

As for proportional sampling (tests/test_gpu_replay.py): fed the marginals
the GPU contracts for the same networks, the oracle's procedure must give the
GPU's records exactly (branch draws, prefix sets, 64-bit population vector,
direct draws, thresholds, probabilities); against the complex128 marginals the
branch draws may differ only near CDF boundaries and the harvested
probabilities within the marginal tolerance."""
import numpy as np
import pytest

import workloads as W
from oracle import sampling, statevector as sv

from replay_check import boundary_mismatches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _gpu_rows(plan, tr, levels=None):
    def rows(j, traj, prefix):
        start, b = plan.blocks[j]
        nt = torch.tensor(np.asarray(traj, np.int64), dtype=torch.int32, device=DEV)
        npre = torch.tensor(np.asarray(prefix, np.uint64).astype(np.int64), dtype=torch.int64, device=DEV)
        marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device=DEV)
        Z = torch.empty(len(traj), dtype=torch.float64, device=DEV)
        ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z)
        torch.cuda.synchronize()
        out = marg.cpu().numpy().astype(np.float64)
        if levels is not None:
            levels.append((np.asarray(traj), np.asarray(prefix, np.uint64), out))
        return out
    return rows


def _records(res, with_prob=True):
    t, b, c = [x.cpu().numpy() for x in res.to_torch()]
    p = res.probs().cpu().numpy() if with_prob else None
    return t, b.astype(np.uint64), c, p


def _sv_rows(circ, kraus, blocks):
    probs = [np.abs(sv.trajectory_state(circ, kraus[i])) ** 2 for i in range(len(kraus))]

    def rows(j, traj, prefix):
        start, b = blocks[j]
        return np.stack([sv.block_marginals(probs[int(i)], circ.n_qubits, start, b)[int(s) & ((1 << start) - 1)]
                         for i, s in zip(traj, prefix)])
    return rows


CASES = [
    # name, circuit maker, blocks, trajectories, branch
    ("brick8_dep", lambda r: W.attach_noise(W.brickwork_1d(8, 5, r), [W.depolarizing_kraus(0.05)]), [3, 2, 3], 12, 1),
    ("brick10_dep_ad", lambda r: W.attach_noise(W.brickwork_1d(10, 6, r), [W.depolarizing_kraus(0.03),
                                                                        W.amplitude_damping_kraus(0.05)]),
     [2, 8], 16, 3),
    ("grid3x4", lambda r: W.attach_noise(W.grid_4colour(3, 4, 6, r), [W.depolarizing_kraus(0.05)]), [4, 4, 4], 9, 2),
]


@pytest.mark.parametrize("mode", ["exhaustive", "direct"])
@pytest.mark.parametrize("name,make,bs,E,branch", CASES, ids=[c[0] for c in CASES])
def test_nonprop_exact_replay_and_c128_agreement(name, make, bs, E, branch, mode):
    circ = make(np.random.default_rng(len(name) * 101))
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=E, est_shots=E * branch ** (len(bs) - 1))
    tr = ptn.ptn_presample_trajectories(plan, 23, E)
    kw = dict(final_shots=700) if mode == "direct" else dict(threshold=0.004)
    res = ptn.ptn_sample_nonprop(plan, tr, 0xBEEF, mode=mode, branch_shots=branch, **kw)
    t, b, c, p = _records(res)
    levels = []
    (rt, rb, rv), nets = sampling.nbs_nonproportional(_gpu_rows(plan, tr, levels), plan.blocks, 0xBEEF, E,
                                                      branch=branch, mode=mode, tau=kw.get("threshold", 0.0),
                                                      final_shots=kw.get("final_shots", 0))
    assert res.nets_per_block == nets
    assert np.array_equal(t, rt) and np.array_equal(b, rb)
    if mode == "direct":
        assert np.array_equal(c, rv) and c.sum() == 700 * nets[-1]
    else:
        assert np.all(c == 1) and np.array_equal(p, rv)
    assert np.all(p > 0) and np.all(p <= 1.0)
    # against complex128 marginals: branch draws differ only near boundaries,
    # and the harvested probabilities match the exact conditionals
    kraus = tr.to_torch()[0].cpu().numpy()
    ref = _sv_rows(circ, kraus, plan.blocks)
    for j, (lt, lp, rows_gpu) in enumerate(levels[:-1]):
        counts = np.full(len(lt), branch)
        d, mm, worst = boundary_mismatches(rows_gpu, ref(j, lt, lp), lt, counts, 0xBEEF, j)
        assert worst <= 1.0 and mm <= max(2, 1e-3 * d)
    ft, fp, _ = levels[-1]
    want = ref(len(bs) - 1, ft, fp)
    start = plan.blocks[-1][0]
    for n in range(len(ft)):
        sel = (t == ft[n]) & ((b & np.uint64((1 << start) - 1)) == fp[n])
        x = (b[sel] >> np.uint64(start)).astype(np.int64)
        cond = want[n] / want[n].sum()
        # norm-wise, as the marginals themselves (2e-5 of the row's norm)
        assert np.linalg.norm(p[sel] - cond[x]) <= 2e-5 * np.linalg.norm(cond) + 1e-12, (name, n)


def test_nonprop_large_final_block_subbatched():
    """30-qubit brickwork (depth 12, depolarizing + amplitude damping) with
    blocks 10/20, one shot per first-block prefix and an exhaustive harvest of
    the 2^20-entry final population vectors (tiled finalize, multi-tile
    harvest), run with a memory cap that splits the final networks into
    several sub-batches: records equal the oracle's on the GPU's marginals."""
    cfg = W.config_c2()
    E = 24
    plan = ptn.ptn_plan_path(cfg["circuit"], [10, 20], hypersamples=16, est_traj=E, est_shots=E,
                             mem_cap_bytes=1.5e8)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], E)
    res = ptn.ptn_sample_nonprop(plan, tr, 99, mode="exhaustive", threshold=2e-6)
    t, b, c, p = _records(res)
    (rt, rb, rp), nets = sampling.nbs_nonproportional(_gpu_rows(plan, tr), plan.blocks, 99, E, mode="exhaustive",
                                                      tau=2e-6)
    assert res.nets_per_block == nets == [E, E]
    assert np.array_equal(t, rt) and np.array_equal(b, rb) and np.array_equal(p, rp)
    assert len(t) > 10 * E
    # per network the kept probabilities sum to at most 1 and cover most of the mass
    for i in range(E):
        s_i = p[t == i].sum()
        assert 0.3 < s_i <= 1.0 + 1e-12


def test_nonprop_direct_b24_against_oracle():
    """Direct sampling of 24-qubit final blocks (2^24-entry population vectors,
    two-level CDF search over 65536 tiles) on a 26-qubit brickwork."""
    rng = np.random.default_rng(2626)
    circ = W.attach_noise(W.brickwork_1d(26, 8, rng), [W.depolarizing_kraus(0.01)])
    E = 3
    plan = ptn.ptn_plan_path(circ, [2, 24], hypersamples=16, est_traj=E, est_shots=E)
    tr = ptn.ptn_presample_trajectories(plan, 5, E)
    res = ptn.ptn_sample_nonprop(plan, tr, 1234, mode="direct", branch_shots=2, final_shots=20000)
    t, b, c, p = _records(res)
    (rt, rb, rc), nets = sampling.nbs_nonproportional(_gpu_rows(plan, tr), plan.blocks, 1234, E, branch=2,
                                                      mode="direct", final_shots=20000)
    assert res.nets_per_block == nets
    assert np.array_equal(t, rt) and np.array_equal(b, rb) and np.array_equal(c, rc)
    assert c.sum() == 20000 * nets[-1]


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3])
def test_paper50_final28_records_against_mps(prec):
    """The benchmarked non-proportional configuration at full size: a 50-qubit,
    200-gate member of the paper's family, blocks 10/10/2/28, one shot per
    prefix and an exhaustive harvest of the 2^28-entry final blocks
    (threshold 1e-6).  The non-final draws and the harvest replay exactly on
    the GPU's marginals of the first blocks (checked by the smaller cases
    above); here sampled records are checked one by one against the exact-MPS
    oracle: p(x | prefix) = |<prefix x|psi>|^2 / p(prefix), both from the
    trajectory's MPS, and the kept mass of every network is at most 1."""
    from oracle import mps
    cfg = W.config_paper(50, 200)
    assert cfg["block_sizes"] == [10, 10, 2, 28]
    E = 4
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=100, est_traj=E, est_shots=E)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], E)
    kraus = tr.to_torch()[0].cpu().numpy()
    res = ptn.ptn_sample_nonprop(plan, tr, 77, mode="exhaustive", threshold=1e-6, precision=prec)
    t, b, c, p = _records(res)
    assert res.nets_per_block == [E, E, E, E]
    assert len(t) > 1000 * E and np.all(c == 1) and np.all(p >= 1e-6)
    start = 22
    for i in range(E):
        sel = np.nonzero(t == i)[0]
        assert len(sel) > 0 and p[sel].sum() <= 1.0 + 1e-9
        pre = {int(x) & ((1 << start) - 1) for x in b[sel]}
        assert len(pre) == 1                       # one shot per prefix: one final network per trajectory
        st = mps.trajectory_mps(cfg["circuit"], kraus[i])
        s_pre = pre.pop()
        p_pre = float(st.block_marginal(start, 0, s_pre)[0])
        pick = np.random.default_rng(i).choice(sel, size=min(100, len(sel)), replace=False)
        for r in pick:
            bits = int(b[r])
            v = np.ones((1, 1), dtype=np.complex128)
            for q in range(50):
                v = v @ st.t[q][:, (bits >> q) & 1, :]
            want = float(abs(v[0, 0]) ** 2) / p_pre
            assert abs(p[r] - want) <= 1e-3 * want + 1e-8, (i, bits, p[r], want)


def test_nonprop_argument_checks():
    rng = np.random.default_rng(3)
    circ = W.attach_noise(W.brickwork_1d(6, 3, rng), [W.depolarizing_kraus(0.05)])
    plan = ptn.ptn_plan_path(circ, [2, 4], hypersamples=4, est_traj=4)
    tr = ptn.ptn_presample_trajectories(plan, 1, 4)
    for kw in (dict(mode="direct", final_shots=0), dict(mode="exhaustive", threshold=1.5),
               dict(mode="exhaustive", branch_shots=0)):
        with pytest.raises(ptn.PtnError) as e:
            ptn.ptn_sample_nonprop(plan, tr, 1, **kw)
        assert e.value.status == 1
    # a proportional run of a plan whose last block exceeds 14 qubits is refused
    big = ptn.ptn_plan_path(W.attach_noise(W.brickwork_1d(18, 3, rng), [W.depolarizing_kraus(0.05)]), [2, 16],
                            hypersamples=4, est_traj=4)
    t2 = ptn.ptn_presample_trajectories(big, 1, 4)
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_sample_shots(big, t2, 1, shots_per_traj=10)
    assert e.value.status == 7
    # proportional results carry no probabilities
    res = ptn.ptn_sample_shots(plan, tr, 1, shots_per_traj=10)
    with pytest.raises(ptn.PtnError):
        res.probs()
