"""Outer products formed in the operand pack on the GPU: a plan whose marked
outer-product steps are formed by their tensor-core consumer's pack gives the
same marginals, bit for bit, as the plan with every step materialised
(keep_products = 1), in every precision mode, and the same sampled records."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"
PRECS = [ptn.PTN_PREC_FP32, ptn.PTN_PREC_BF16X3, ptn.PTN_PREC_FP16X3]


def _pair(circ, bs, **kw):
    fused = ptn.ptn_plan_path(circ, bs, **kw)
    keep = ptn.ptn_plan_path(circ, bs, keep_products=True, **kw)
    d = fused.describe(detail=1)
    blocks = [j for j, b in enumerate(d["blocks"]) if any(st["prod"] for st in b["steps"])]
    assert blocks
    return fused, keep, blocks


def _marg(plan, tr, j, nt, npre, prec):
    b = plan.block_sizes[j]
    m = torch.empty((nt.numel(), 1 << b), dtype=torch.float32, device=DEV)
    Z = torch.empty(nt.numel(), dtype=torch.float64, device=DEV)
    ptn.ptn_contract_batch(plan, tr, j, nt, npre, m, Z, precision=prec)
    torch.cuda.synchronize()
    return m, Z


@pytest.mark.parametrize("which", ["brick20", "c2"])
def test_products_bit_identical(which):
    if which == "c2":
        c2 = W.config_c2()
        circ, bs, kw, E = c2["circuit"], c2["block_sizes"], dict(hypersamples=100, est_traj=4096, est_shots=1e6), 64
    else:
        rng = np.random.default_rng(0)
        circ = W.attach_noise(W.brickwork_1d(20, 8, rng), [W.depolarizing_kraus(0.01)])
        bs, kw, E = [10, 10], dict(hypersamples=8, est_traj=64, est_shots=4096, network_form=1), 32
    fused, keep, blocks = _pair(circ, bs, **kw)
    trf = ptn.ptn_presample_trajectories(fused, 11, E)
    trk = ptn.ptn_presample_trajectories(keep, 11, E)
    rng = np.random.default_rng(3)
    for j in blocks:
        start = fused.blocks[j][0]
        nt = torch.repeat_interleave(torch.arange(E, dtype=torch.int32, device=DEV), 3)
        npre = torch.from_numpy(rng.integers(0, 1 << start, size=3 * E, dtype=np.int64)).to(DEV)
        for prec in PRECS:
            mf, zf = _marg(fused, trf, j, nt, npre, prec)
            mk, zk = _marg(keep, trk, j, nt, npre, prec)
            assert torch.equal(mf, mk) and torch.equal(zf, zk), (j, prec)


def test_products_c2_sampling_identical():
    c2 = W.config_c2()
    fused, keep, _ = _pair(c2["circuit"], c2["block_sizes"], hypersamples=100, est_traj=4096, est_shots=1e6)
    out = []
    for p in (fused, keep):
        tr = ptn.ptn_presample_trajectories(p, 21, 64)
        res = ptn.ptn_sample_shots(p, tr, 4, total_shots=15616, precision=ptn.PTN_PREC_FP16X3)
        out.append([x.cpu().numpy() for x in res.to_torch()])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
