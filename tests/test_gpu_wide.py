"""Plans of more than 64 qubits (the paper's circuit family at 100 and more
qubits, Sec. IV-B): prefixes and bitstrings are W = ceil(n / 64) words.
Sampled networks whose projected prefixes reach past bit 64 against the
exact-MPS oracle; proportional and non-proportional sampling replayed exactly
by the oracle on the GPU's own marginals (bitstrings compared as integers);
the merge of a wide result against a host aggregation."""
import numpy as np
import pytest

import workloads as W
from oracle import mps, sampling

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _rows_fn(plan, tr):
    """marginal_fn for the oracle: GPU marginals of the given networks
    (prefixes as Python integers or uint64, passed as W-word rows)."""
    nw = ptn.words_of(plan.n_qubits)

    def rows(j, traj, prefix):
        start, b = plan.blocks[j]
        nt = torch.tensor(np.asarray(traj, np.int64), dtype=torch.int32, device=DEV)
        npre = torch.from_numpy(ptn.int_to_words([int(p) for p in prefix], nw).copy()).to(DEV)
        marg = torch.empty((len(traj), 1 << b), dtype=torch.float32, device=DEV)
        Z = torch.empty(len(traj), dtype=torch.float64, device=DEV)
        ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z)
        torch.cuda.synchronize()
        return marg.cpu().numpy().astype(np.float64)
    return rows


def _ints(bits):
    b = bits.cpu().numpy() if hasattr(bits, "cpu") else np.asarray(bits)
    return [ptn.bits_to_int(r) for r in b]


def _plan(n, g, bs, seed=7, E=8):
    rng = np.random.default_rng(seed)
    circ = W.paper_random_circuit(n, g, rng)
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=16, est_traj=E, est_shots=E * 8)
    return circ, plan


def test_wide_networks_vs_mps():
    """100 qubits, 300 gates, blocks of 10: networks of the blocks starting at
    qubits 70, 80 and 90 with random prefixes (bits up to 89) against exact
    MPS block marginals."""
    circ, plan = _plan(100, 300, [10] * 10)
    assert ptn.words_of(plan.n_qubits) == 2
    E = 4
    tr = ptn.ptn_presample_trajectories(plan, 3, E)
    kraus = tr.to_torch()[0].cpu().numpy()
    states = [mps.trajectory_mps(circ, kraus[t]) for t in range(E)]
    rows = _rows_fn(plan, tr)
    rng = np.random.default_rng(11)
    for j in (6, 7, 8, 9):
        start, b = plan.blocks[j]
        traj = np.repeat(np.arange(E), 2)
        prefix = [int.from_bytes(rng.bytes(12), "little") & ((1 << start) - 1) for _ in traj]
        got = rows(j, traj, prefix)
        for n, (t, s) in enumerate(zip(traj, prefix)):
            want = states[t].block_marginal(start, b, s)
            err = np.linalg.norm(got[n] - want) / max(np.linalg.norm(want), 1e-12)
            assert err < 2e-5, (j, t, err)


@pytest.mark.parametrize("prec", [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3])
def test_wide_proportional_replay_and_merge(prec):
    """80 qubits, blocks of 10, 8 trajectories, 4000 shots: the GPU's records
    equal the oracle's proportional NBS on the GPU's marginals; merging
    across trajectories equals a host aggregation of the same records."""
    circ, plan = _plan(80, 260, [10] * 8)
    E = 8
    tr = ptn.ptn_presample_trajectories(plan, 5, E)
    res = ptn.ptn_sample_shots(plan, tr, 21, total_shots=4000, precision=prec)
    t, b, c = res.to_torch()
    assert b.shape == (res.n, 2)
    rt, rb, rc, levels, _ = sampling.nbs_proportional(_rows_fn(plan, tr), plan.blocks, 21, E, total_shots=4000)
    assert res.nets_per_block == levels
    assert np.array_equal(t.cpu().numpy(), rt) and np.array_equal(c.cpu().numpy(), rc)
    assert _ints(b) == [int(x) for x in rb]
    assert any(x >> 64 for x in _ints(b))
    merged = ptn.ptn_shots_merge(res, len(plan.blocks))
    mt, mb, mc = merged.to_torch()
    agg = {}
    for x, k in zip(_ints(b), c.cpu().numpy()):
        agg[x] = agg.get(x, 0) + int(k)
    keys = sorted(agg)
    assert _ints(mb) == keys and [int(k) for k in mc.cpu().numpy()] == [agg[k] for k in keys]
    assert np.all(mt.cpu().numpy() == -1)


def test_wide_nonproportional_exhaustive_replay():
    """100 qubits: eight blocks of 10 with one shot per prefix, then an
    exhaustive harvest of a 20-qubit final block (records reach bit 99)."""
    circ, plan = _plan(100, 300, [10] * 8 + [20], seed=9)
    E = 6
    tr = ptn.ptn_presample_trajectories(plan, 8, E)
    res = ptn.ptn_sample_nonprop(plan, tr, 31, mode="exhaustive", threshold=1e-5)
    t, b, c = res.to_torch()
    p = res.probs().cpu().numpy()
    (rt, rb, rp), nets = sampling.nbs_nonproportional(_rows_fn(plan, tr), plan.blocks, 31, E, mode="exhaustive",
                                                      tau=1e-5)
    assert res.nets_per_block == nets
    assert np.array_equal(t.cpu().numpy(), rt) and np.array_equal(p, rp)
    assert _ints(b) == [int(x) for x in rb]
    assert len(rt) > E and max(_ints(b)) >> 80
