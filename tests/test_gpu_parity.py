"""GPU parity tests: the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs."""
import numpy as np
import pytest

import workloads as W
from oracle import mps, pts, sampling, statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _plan(cfg, hyper=16):
    shots = cfg.get("total_shots") or cfg["n_traj"] * (cfg.get("shots_per_traj") or 1)
    return ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=hyper,
                             est_traj=cfg["n_traj"], est_shots=shots)


# ---------------------------------------------------------- pre-sampling ----

@pytest.mark.parametrize("cfg_fn", [W.config_c1, W.config_c2], ids=["c1", "c2"])
def test_presample_bit_exact(cfg_fn):
    cfg = cfg_fn()
    plan = _plan(cfg, hyper=2)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"], dedup=False)
    kr, lq, mu, fi = [x.cpu().numpy() for x in tr.to_torch()]
    k_ref, lq_ref = pts.presample(cfg["circuit"], cfg["n_traj"], cfg["seed"])
    assert np.array_equal(kr, k_ref)
    np.testing.assert_allclose(lq, lq_ref, rtol=1e-12, atol=1e-12)
    assert np.all(mu == 1) and np.array_equal(fi, np.arange(cfg["n_traj"]))


def test_presample_dedup_matches_oracle():
    cfg = W.config_c1()
    plan = _plan(cfg, hyper=2)
    for seed in (cfg["seed"], 7, 8):
        tr = ptn.ptn_presample_trajectories(plan, seed, 300, dedup=True)
        kr, lq, mu, fi = [x.cpu().numpy() for x in tr.to_torch()]
        k_ref, lq_ref = pts.presample(cfg["circuit"], 300, seed)
        ku, lu, mult, first = pts.dedup(k_ref, lq_ref)
        assert np.array_equal(kr, ku) and np.array_equal(mu, mult) and np.array_equal(fi, first)
        assert mu.sum() == 300 and len(mu) < 300


def test_presample_dedup_large_against_oracle():
    """Dedup by hash sort at 200,000 trajectories (past what a pairwise search
    handles): the 12-qubit brickwork at p = 0.01 over 184 sites leaves about
    16% of the rows error-free, so one run of equal rows holds ~31k entries.
    The deduplicated rows, multiplicities and first indices equal the oracle's
    dedup of the same draw (the undeduplicated rows, which are bit-exact with
    the oracle's pre-sampling in the tests above)."""
    cfg = W.config_c1()
    plan = _plan(cfg, hyper=2)
    N = 200_000
    full = ptn.ptn_presample_trajectories(plan, 4242, N, dedup=False)
    rows, lq_all = [x.cpu().numpy() for x in full.to_torch()[:2]]
    tr = ptn.ptn_presample_trajectories(plan, 4242, N, dedup=True)
    kr, lq, mu, fi = [x.cpu().numpy() for x in tr.to_torch()]
    ku, lu, mult, first = pts.dedup(rows, lq_all)
    assert np.array_equal(kr, ku) and np.array_equal(mu, mult) and np.array_equal(fi, first)
    assert np.array_equal(lq, lu)
    assert mu.sum() == N and mu.max() > 20_000 and len(mu) < N


def test_presample_edge_single_trajectory_and_circuit_id():
    cfg = W.config_c1()
    plan = _plan(cfg, hyper=2)
    tr = ptn.ptn_presample_trajectories(plan, 5, 1, circuit_id=3)
    kr = tr.to_torch()[0].cpu().numpy()
    k_ref, _ = pts.presample(cfg["circuit"], 1, 5, circuit_id=3)
    assert np.array_equal(kr, k_ref)


# ----------------------------------------------------------- contraction ----

def _contract(plan, tr, j, traj, prefix, b):
    nt = torch.tensor(traj, dtype=torch.int32, device=DEV)
    npre = torch.tensor(np.asarray(prefix, dtype=np.int64), dtype=torch.int64, device=DEV)
    marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device=DEV)
    Z = torch.empty(len(traj), dtype=torch.float64, device=DEV)
    ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z)
    torch.cuda.synchronize()
    return marg.cpu().numpy().astype(np.float64), Z.cpu().numpy()


def _rel(a, b):
    # norm-wise relative error; a zero row (zero-norm trajectory) is compared absolutely
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-12)


SMALL = [
    ("brick6", lambda r: W.attach_noise(W.brickwork_1d(6, 5, r), [W.depolarizing_kraus(0.2),
                                                               W.amplitude_damping_kraus(0.3)]), [2, 3, 1]),
    ("grid3x4", lambda r: W.attach_noise(W.grid_4colour(3, 4, 6, r), [W.depolarizing_kraus(0.1)]), [5, 7]),
    ("hea6", lambda r: W.attach_noise(W.hea_ring(6, 3, r.standard_normal(36)), [W.depolarizing_kraus(0.05)]),
     [3, 2, 1]),
]


@pytest.mark.parametrize("name,make,bs", SMALL, ids=[c[0] for c in SMALL])
def test_contract_small_circuits(name, make, bs):
    rng = np.random.default_rng(len(name) * 7919)
    circ = make(rng)
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=16, est_shots=256)
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
        assert np.max(_rel(marg, want)) < 2e-5, name
        np.testing.assert_allclose(Z, marg.sum(axis=1), rtol=1e-12)
        np.testing.assert_allclose(Z, want.sum(axis=1), rtol=2e-5, atol=1e-12)


def test_contract_c1_all_blocks():
    """Config C1 (12-qubit brickwork, depth 8): block 1 for all 64
    trajectories, block 2 for ragged prefix sets, against the c128 oracle."""
    cfg = W.config_c1()
    circ = cfg["circuit"]
    plan = _plan(cfg)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(64)]
    marg, Z = _contract(plan, tr, 0, np.arange(64), np.zeros(64, int), 10)
    want = np.array([sv.block_marginals(p, 12, 0, 10)[0] for p in probs])
    assert np.max(_rel(marg, want)) < 2e-5
    np.testing.assert_allclose(Z, 1.0, rtol=1e-5)     # depolarizing: unit-norm trajectories
    # ragged: trajectory t has t % 7 networks (some have none)
    traj, prefix = [], []
    prng = np.random.default_rng(9)
    for t in range(64):
        for _ in range(t % 7):
            traj.append(t)
            prefix.append(int(prng.integers(0, 1024)))
    marg2, Z2 = _contract(plan, tr, 1, np.array(traj), np.array(prefix), 2)
    want2 = np.array([sv.block_marginals(probs[t], 12, 10, 2)[s] for t, s in zip(traj, prefix)])
    assert np.max(_rel(marg2, want2)) < 2e-5
    # parent-child identity: Z of a block-2 network equals the parent's marginal entry
    np.testing.assert_allclose(Z2, [want[t][s] for t, s in zip(traj, prefix)], rtol=2e-5, atol=1e-12)


def test_contract_empty_batch():
    cfg = W.config_c1()
    plan = _plan(cfg, hyper=2)
    tr = ptn.ptn_presample_trajectories(plan, 1, 4)
    marg, Z = _contract(plan, tr, 1, np.zeros(0, int), np.zeros(0, int), 2)
    assert marg.shape == (0, 4)


def test_contract_rejects_unsorted_networks():
    cfg = W.config_c1()
    plan = _plan(cfg, hyper=2)
    tr = ptn.ptn_presample_trajectories(plan, 1, 4)
    with pytest.raises(ptn.PtnError) as e:
        _contract(plan, tr, 0, np.array([1, 0]), np.zeros(2, int), 10)
    assert e.value.status == 1


def test_contract_c2_sampled_networks_vs_mps():
    """Config C2 at full size (30 qubits, depth 12, 4096 trajectories), launched
    as in the benchmark; sampled networks of every block checked one by one
    against the exact-MPS oracle."""
    cfg = W.config_c2()
    circ = cfg["circuit"]
    plan = _plan(cfg, hyper=16)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    kraus = tr.to_torch()[0].cpu().numpy()
    pick = [0, 1, 1777, 4095]
    states = {t: mps.trajectory_mps(circ, kraus[t]) for t in pick}
    marg, Z = _contract(plan, tr, 0, np.arange(4096), np.zeros(4096, int), 10)
    for t in pick:
        want = states[t].block_marginal(0, 10, 0)
        assert _rel(marg[t], want) < 2e-5
    prng = np.random.default_rng(4)
    for j in (1, 2):
        start = 10 * j
        traj = np.repeat(pick, 3)
        prefix = prng.integers(0, 1 << start, size=len(traj))
        m, _ = _contract(plan, tr, j, traj, prefix, 10)
        for n, (t, s) in enumerate(zip(traj, prefix)):
            want = states[t].block_marginal(start, 10, int(s))
            assert _rel(m[n], want) < 2e-5, (j, t)


# --------------------------------------------------------------- sampling ----

def _sample_gpu(p_rows, traj, prefix, counts, b, start, seed, block, circuit=0):
    n = len(traj)
    marg = torch.tensor(p_rows, dtype=torch.float32, device=DEV)
    pt = torch.tensor(traj, dtype=torch.int32, device=DEV)
    pp = torch.tensor(np.asarray(prefix, np.int64), dtype=torch.int64, device=DEV)
    pc = torch.tensor(counts, dtype=torch.int64, device=DEV)
    cap = int(np.minimum(np.asarray(counts), 1 << b).sum()) + 1
    ct = torch.empty(cap, dtype=torch.int32, device=DEV)
    cp = torch.empty(cap, dtype=torch.int64, device=DEV)
    cc = torch.empty(cap, dtype=torch.int64, device=DEV)
    nc = ptn.ptn_sample_block(marg, b, start, pt, pp, pc, seed, circuit, block, ct, cp, cc)
    torch.cuda.synchronize()
    return ct[:nc].cpu().numpy(), cp[:nc].cpu().numpy().astype(np.uint64), cc[:nc].cpu().numpy()


@pytest.mark.parametrize("b,start,n,circuit", [(10, 0, 300, 0), (2, 10, 500, 5), (7, 3, 64, 1), (1, 40, 17, 0),
                                               (12, 20, 9, 2)])
def test_sample_block_bit_exact(b, start, n, circuit):
    rows = W.synthetic_marginals(n, b, seed=b * 100 + n)
    rng = np.random.default_rng(n)
    traj = np.sort(rng.integers(0, max(n // 3, 1), size=n))
    prefix = rng.integers(0, 1 << start, size=n) if start else np.zeros(n, int)
    counts = rng.integers(0, 2000, size=n)
    counts[::7] = 0                                  # parents with no shots
    counts[1::11] = rng.integers(5000, 20000, size=len(counts[1::11]))   # heavy parents
    ct, cp, cc = _sample_gpu(rows, traj, prefix, counts, b, start, seed=0xABCDEF, block=3, circuit=circuit)
    r0 = sampling.rank_offsets(traj, counts)
    par, xs, cs = sampling.sample_block(rows, traj, counts, r0, 0xABCDEF, 3, circuit)
    assert np.array_equal(ct, traj[par])
    assert np.array_equal(cp, (prefix[par].astype(np.uint64) | (xs.astype(np.uint64) << np.uint64(start))))
    assert np.array_equal(cc, cs)
    assert cc.sum() == counts.sum()


def test_sample_block_degenerate_rows():
    """One-hot rows always return their nonzero bin; uniform rows spread."""
    b = 4
    rows = np.zeros((3, 16), np.float32)
    rows[0, 9] = 1e-30
    rows[1, :] = 1.0
    rows[2, 15] = 7.0
    ct, cp, cc = _sample_gpu(rows, [0, 1, 2], [0, 0, 0], [100, 16000, 5], b, 0, seed=1, block=0)
    assert cp[ct == 0].tolist() == [9] and cc[ct == 0].tolist() == [100]
    assert len(cp[ct == 1]) == 16
    assert cp[ct == 2].tolist() == [15]


def test_sample_block_rejects_short_child_capacity():
    """A child capacity below sum_n min(count_n, 2^b) is an error (nothing is
    written past the caller's buffers); a capacity equal to it succeeds."""
    b, n = 6, 40
    rows = W.synthetic_marginals(n, b, seed=5)
    counts = np.full(n, 100)
    need = int(np.minimum(counts, 1 << b).sum())
    dev = DEV
    args = (torch.tensor(rows, dtype=torch.float32, device=dev), b, 0,
            torch.arange(n, dtype=torch.int32, device=dev), torch.zeros(n, dtype=torch.int64, device=dev),
            torch.tensor(counts, dtype=torch.int64, device=dev), 3, 0, 0)
    for fn in (ptn.ptn_sample_block, ptn.ptn_sample_block_noalloc):
        guard = 4096
        ct = torch.full((need - 1 + guard,), -7, dtype=torch.int32, device=dev)
        cp = torch.full((need - 1 + guard,), -7, dtype=torch.int64, device=dev)
        cc = torch.full((need - 1 + guard,), -7, dtype=torch.int64, device=dev)
        with pytest.raises(ptn.PtnError) as e:
            fn(*args, ct[:need - 1], cp[:need - 1], cc[:need - 1])
        assert e.value.status == 1 and "capacity" in str(e.value)
        torch.cuda.synchronize()
        assert bool((ct[need - 1:] == -7).all()) and bool((cc[need - 1:] == -7).all())
        ct2 = torch.empty(need, dtype=torch.int32, device=dev)
        cp2 = torch.empty(need, dtype=torch.int64, device=dev)
        cc2 = torch.empty(need, dtype=torch.int64, device=dev)
        nc = fn(*args, ct2, cp2, cc2)
        assert int(cc2[:nc].sum()) == counts.sum()


def test_allocate_shots_bit_exact():
    rng = np.random.default_rng(12)
    for n, total in [(4096, 1_000_000), (1, 10), (37, 12345)]:
        w = rng.exponential(1.0, size=n) * np.exp(rng.uniform(-5, 0, size=n))
        if n > 10:
            w[::9] = 0.0
        wt = torch.tensor(w, dtype=torch.float64, device=DEV)
        m = torch.empty(n, dtype=torch.int64, device=DEV)
        ptn.ptn_allocate_shots(wt, total, 0x5EED, 2, m)
        got = m.cpu().numpy()
        want = sampling.allocate_shots(w, total, 0x5EED, 2)
        assert np.array_equal(got, want)
        assert got.sum() == total


# ---------------------------------------------------------- end to end ----

def _tvd(p, q):
    return 0.5 * np.abs(p - q).sum()


def test_sample_shots_c1_end_to_end():
    """C1: 64 trajectories x 1000 shots.  Every shot accounted for, canonical
    order, and 4-qubit marginals (16 outcomes, so the expected sampling TVD is
    well below the bound) within TVD 3/sqrt(shots) of the exact trajectory
    mixture (oracle state vectors)."""
    cfg = W.config_c1()
    circ = cfg["circuit"]
    plan = _plan(cfg)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    res = ptn.ptn_sample_shots(plan, tr, cfg["seed"], shots_per_traj=1000)
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    assert cnt.sum() == 64_000
    for i in range(64):
        assert cnt[t == i].sum() == 1000
    keys = list(zip(t.tolist(), bits.tolist()))
    assert keys == sorted(keys, key=lambda k: (k[0], k[1] & 1023, k[1] >> 10))
    assert res.nets_per_block[0] == 64
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = np.mean([np.abs(sv.trajectory_state(circ, kraus[i])) ** 2 for i in range(64)], axis=0)
    emp = np.zeros(1 << 12)
    np.add.at(emp, bits.astype(np.int64), cnt)
    emp /= emp.sum()
    N = 64_000
    for qs in ([0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 10, 11], [0, 5, 10, 11]):
        idx = np.arange(1 << 12)
        key = sum(((idx >> q) & 1) << k for k, q in enumerate(qs))
        pe = np.bincount(key, weights=emp, minlength=1 << len(qs))
        pq = np.bincount(key, weights=probs, minlength=1 << len(qs))
        assert _tvd(pe, pq) < 3 / np.sqrt(N)


def test_sample_shots_c2_proportional_total():
    """C2 at full size: 1e6 shots over 4096 trajectories (allocation by
    multiplicity x norm), blocks of 10."""
    cfg = W.config_c2()
    plan = _plan(cfg, hyper=16)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"])
    res = ptn.ptn_sample_shots(plan, tr, cfg["seed"], total_shots=cfg["total_shots"])
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    assert cnt.sum() == 1_000_000
    assert res.nets_per_block[0] == 4096
    assert res.nets_per_block[1] <= 1_000_000 and res.nets_per_block[2] >= res.nets_per_block[1]
    assert np.all(np.diff(t) >= 0)
    assert len(set(zip(t.tolist(), bits.tolist()))) == len(t)


def test_sample_shots_c2_distribution_vs_mps_mixture():
    """30-qubit brickwork (depth 12, depolarizing + amplitude damping) on a
    16-trajectory subset with 10^6 shots allocated in proportion to the
    trajectory weights: each shot is an i.i.d. draw from the mixture
    sum_i w_i p_i / sum_i w_i, so 4-qubit window marginals of the shots must lie
    within TVD 3/sqrt(shots) of the exact-MPS mixture (16 outcomes: expected
    TVD about 1.5/sqrt(shots))."""
    cfg = W.config_c2()
    circ = cfg["circuit"]
    plan = _plan(cfg, hyper=16)
    E, N = 16, 1_000_000
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"] + 17, E)
    res = ptn.ptn_sample_shots(plan, tr, cfg["seed"] + 17, total_shots=N)
    t, bits, cnt = [x.cpu().numpy() for x in res.to_torch()]
    assert cnt.sum() == N
    kraus = tr.to_torch()[0].cpu().numpy()
    states = [mps.trajectory_mps(circ, kraus[i]) for i in range(E)]
    bits = bits.astype(np.uint64)
    for start in (0, 8, 18, 26):
        key = ((bits >> np.uint64(start)) & np.uint64(15)).astype(np.int64)
        pe = np.bincount(key, weights=cnt, minlength=16) / N
        pq = sum(st.window_marginal(start, 4) for st in states)   # sum_i w_i p_i (unnormalised)
        pq = pq / pq.sum()
        assert _tvd(pe, pq) < 3 / np.sqrt(N), (start, _tvd(pe, pq))


def test_contract_tensor_core_steps_vs_statevector():
    """A 20-qubit brickwork whose block paths contain tensor-core (tcgen05)
    GEMM steps, every block against c128 state vectors."""
    rng = np.random.default_rng(2020)
    circ = W.attach_noise(W.brickwork_1d(20, 10, rng), [W.depolarizing_kraus(0.01),
                                                         W.amplitude_damping_kraus(0.01)])
    plan = ptn.ptn_plan_path(circ, [10, 6, 4], hypersamples=16, est_traj=512, est_shots=1e5)
    d = plan.describe()
    assert sum(b["n_gemm"] for b in d["blocks"]) > 0
    tr = ptn.ptn_presample_trajectories(plan, 31, 6)
    kraus = tr.to_torch()[0].cpu().numpy()
    probs = [np.abs(sv.trajectory_state(circ, kraus[t])) ** 2 for t in range(6)]
    prng = np.random.default_rng(8)
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(6), 7)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        marg, Z = _contract(plan, tr, j, traj, prefix, b)
        want = np.array([sv.block_marginals(probs[t], 20, start, b)[int(s)] for t, s in zip(traj, prefix)])
        assert np.max(_rel(marg, want)) < 2e-5, j
