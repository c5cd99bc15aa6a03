"""GPU test of ptn_sample_block_noalloc, the sampling entry point for callers
that cannot allocate device memory while it runs (its scratch is a fixed
static device array).  It must return exactly what the allocating
ptn_sample_block returns, on consecutive calls that share the array, and
refuse work that does not fit the array.  Kept in a file of its own, collected
last."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402


def _call(fn, rows, traj, prefix, counts, b, start, seed, block, circuit, cap=None):
    dev = "cuda"
    marg = torch.tensor(rows, dtype=torch.float32, device=dev)
    pt = torch.tensor(traj, dtype=torch.int32, device=dev)
    pp = torch.tensor(np.asarray(prefix, np.int64), dtype=torch.int64, device=dev)
    pc = torch.tensor(counts, dtype=torch.int64, device=dev)
    if cap is None:
        cap = int(np.minimum(np.asarray(counts), 1 << b).sum()) + 1
    ct = torch.empty(cap, dtype=torch.int32, device=dev)
    cp = torch.empty(cap, dtype=torch.int64, device=dev)
    cc = torch.empty(cap, dtype=torch.int64, device=dev)
    nc = fn(marg, b, start, pt, pp, pc, seed, circuit, block, ct, cp, cc)
    torch.cuda.synchronize()
    return ct[:nc].cpu().numpy(), cp[:nc].cpu().numpy(), cc[:nc].cpu().numpy()


def _inputs(n, b, start, seed):
    rows = W.synthetic_marginals(n, b, seed=seed)
    rng = np.random.default_rng(seed)
    traj = np.sort(rng.integers(0, max(n // 4, 1), size=n))
    prefix = rng.integers(0, 1 << start, size=n) if start else np.zeros(n, int)
    counts = rng.integers(0, 3000, size=n)
    counts[::5] = 0
    return rows, traj, prefix, counts


def test_noalloc_matches_allocating_sampler_on_consecutive_calls():
    # a large call, then a smaller one that reads the array after the first left it dirty
    for n, b, start, seed in [(2000, 10, 10, 11), (37, 6, 3, 12)]:
        rows, traj, prefix, counts = _inputs(n, b, start, seed)
        got = _call(ptn.ptn_sample_block_noalloc, rows, traj, prefix, counts, b, start, 0xC0FFEE, 1, 4)
        want = _call(ptn.ptn_sample_block, rows, traj, prefix, counts, b, start, 0xC0FFEE, 1, 4)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
        assert got[2].sum() == counts.sum()


def test_noalloc_rejects_work_beyond_its_scratch():
    rows, traj, prefix, counts = _inputs(64, 8, 0, 13)
    with pytest.raises(ptn.PtnError) as e:
        _call(ptn.ptn_sample_block_noalloc, rows, traj, prefix, counts, 8, 0, 1, 0, 0, cap=4_000_000)
    assert e.value.status == 3 and "scratch" in str(e.value)
