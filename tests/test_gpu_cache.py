"""Intermediate caching across error sets (Sec. VI) on the GPU: a plan with
cache_intermediates gives bit-identical marginals and sampled records to the
same plan without it, and every cached step runs over exactly as many
instances as the chunk has distinct variant keys on the step's columns
(counted on the host from the trajectories' Kraus rows and the planner's
column lists, compared through the per-step flop counts of the library's
statistics)."""
import numpy as np
import pytest

import workloads as W
from plan_replay import var_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _plans(circ, bs, **kw):
    base = dict(hypersamples=8, est_traj=256, est_shots=4096)
    base.update(kw)
    return (ptn.ptn_plan_path(circ, bs, cache_intermediates=True, **base),
            ptn.ptn_plan_path(circ, bs, cache_intermediates=False, **base))


def _contract(plan, tr, j, nt, npre, prec):
    b = plan.block_sizes[j]
    marg = torch.empty((nt.numel(), 1 << b), dtype=torch.float32, device=DEV)
    Z = torch.empty(nt.numel(), dtype=torch.float64, device=DEV)
    ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z, precision=prec)
    torch.cuda.synchronize()
    return marg, Z


def _step_flops():
    out = {}
    for blk, st, _k, _l, _ms, _by, fl in ptn.ptn_stats_read_steps():
        out[(blk, st)] = out.get((blk, st), 0.0) + fl
    return out


def _check(circ, bs, E, precisions, seed=5, **kw):
    pc, pp = _plans(circ, bs, **kw)
    desc = pc.describe(detail=1)
    assert sum(b["n_cache"] for b in desc["blocks"]) > 0
    trc = ptn.ptn_presample_trajectories(pc, seed, E)
    trp = ptn.ptn_presample_trajectories(pp, seed, E)
    kraus = trc.to_torch()[0].cpu().numpy()
    assert np.array_equal(kraus, trp.to_torch()[0].cpu().numpy())
    vids = var_ids(desc, kraus)
    rng = np.random.default_rng(seed)
    shared = 0
    for prec in precisions:
        for j, (start, b) in enumerate(pc.blocks):
            nt = torch.arange(E, dtype=torch.int32, device=DEV)
            pre = rng.integers(0, 1 << start, size=E, dtype=np.int64) if start else np.zeros(E, np.int64)
            npre = torch.from_numpy(pre).to(DEV)
            ptn.ptn_stats_enable(True)
            ptn.ptn_stats_reset()
            mc, zc = _contract(pc, trc, j, nt, npre, prec)
            fc = _step_flops()
            ptn.ptn_stats_reset()
            mp, zp = _contract(pp, trp, j, nt, npre, prec)
            fp = _step_flops()
            ptn.ptn_stats_enable(False)
            assert torch.equal(mc, mp) and torch.equal(zc, zp), (prec, j)
            for i, st in enumerate(desc["blocks"][j]["steps"]):
                if not st["cache"]:
                    continue
                cols = desc["blocks"][j]["cache_cols"][st["cache"] - 1]
                n_rep = len({tuple(r) for r in vids[:, cols]})
                assert fp[(j, i)] > 0
                assert fc[(j, i)] * E == pytest.approx(fp[(j, i)] * n_rep, rel=1e-12), (j, i, n_rep)
                shared += E - n_rep
    assert shared > 0
    return pc, pp


def test_cache_gate_level_steps_c1():
    """12-qubit brickwork with every step launched on its own (fuse_max = 1):
    the gate-level SIMT steps (direct and register-tiled kernels) cached."""
    c1 = W.config_c1()
    _check(c1["circuit"], [10, 2], 256, [ptn.PTN_PREC_FP32], fuse_max=1)
    _check(c1["circuit"], [10, 2], 256, [ptn.PTN_PREC_FP32], fuse_max=1, network_form=2)


def test_cache_c2_tensor_core_steps():
    """The 30-qubit brickwork plan as benchmarked (fused runs, tensor-core
    trajectory steps among the cached ones), 64 trajectories, FP32 (TF32
    hi/lo) and FP16x3."""
    c2 = W.config_c2()
    pc, _ = _check(c2["circuit"], c2["block_sizes"], 64, [ptn.PTN_PREC_FP32, ptn.PTN_PREC_FP16X3],
                   est_traj=4096, est_shots=1e6, hypersamples=100)
    desc = pc.describe(detail=1)
    assert any(st["cache"] and st["kind"] == 1 for b in desc["blocks"] for st in b["steps"])


@pytest.mark.parametrize("graphs", [0, 1])
def test_cache_c2_sampling_records_identical(graphs):
    """ptn_sample_shots on the 30-qubit plan, 64 trajectories, 15,616 shots:
    the same records with and without caching (stream and graph execution)."""
    c2 = W.config_c2()
    pc, pp = _plans(c2["circuit"], c2["block_sizes"], hypersamples=100, est_traj=4096, est_shots=1e6)
    out = []
    for p in (pc, pp):
        tr = ptn.ptn_presample_trajectories(p, 77, 64)
        res = ptn.ptn_sample_shots(p, tr, 9, total_shots=15616, precision=ptn.PTN_PREC_FP16X3, use_graphs=graphs)
        out.append([x.cpu().numpy() for x in res.to_torch()])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_cache_nonprop_identical():
    """Non-proportional sampling (one shot per prefix, exhaustive harvest of
    the last 10-qubit block) on the 30-qubit plan with caching: the same
    records and probabilities as without."""
    c2 = W.config_c2()
    pc, pp = _plans(c2["circuit"], c2["block_sizes"], hypersamples=100, est_traj=4096, est_shots=1e6)
    out = []
    for p in (pc, pp):
        tr = ptn.ptn_presample_trajectories(p, 3, 64)
        res = ptn.ptn_sample_nonprop(p, tr, 5, mode="exhaustive", threshold=1e-5, precision=ptn.PTN_PREC_FP16X3)
        out.append([x.cpu().numpy() for x in res.to_torch()] + [res.probs().cpu().numpy()])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
