"""Path search with per-restart random streams (ptn_plan_opts.search_threads):
the plan does not depend on the number of host threads, the plans it finds
replay to the statevector oracle, and a negative count is rejected.  No GPU."""
import zlib

import numpy as np
import pytest

import workloads as W
from oracle import pts
from paper_2604_08467_gb300 import ptn
from plan_replay import run_block
from test_plan_host import CASES, _oracle_rows


def _desc(circ, bs, **kw):
    d = ptn.ptn_plan_path(circ, bs, **kw).describe(detail=1)
    d.pop("plan_seconds")
    return d


def test_plan_independent_of_thread_count():
    c2 = W.config_c2()
    kw = dict(hypersamples=48, est_traj=4096, est_shots=1e6)
    ref = _desc(c2["circuit"], c2["block_sizes"], search_threads=1, **kw)
    for n in (2, 5, 16):
        assert _desc(c2["circuit"], c2["block_sizes"], search_threads=n, **kw) == ref, n


@pytest.mark.parametrize("name,make,bs", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_threaded_search_plans_replay_to_oracle(name, make, bs):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    circ = make(rng)
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=24, est_traj=4, est_shots=64, search_threads=4)
    desc = plan.describe(detail=1)
    kraus, _ = pts.presample(circ, 4, seed=17)
    prng = np.random.default_rng(5)
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(4), 3)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        got = run_block(desc, j, kraus, traj, prefix)
        want = _oracle_rows(circ, kraus, plan.blocks, j, traj, prefix)
        assert np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30) < 2e-5, (name, j)


def test_negative_thread_count_rejected():
    c1 = W.config_c1()
    with pytest.raises(ptn.PtnError):
        ptn.ptn_plan_path(c1["circuit"], c1["block_sizes"], hypersamples=4, search_threads=-1)


def test_search_keeps_only_lowerable_paths():
    """Paths with a step summing more bits than a step may (24) are skipped by
    the search rather than chosen and rejected at lowering: the ket-only form of
    a 6x5-grid block whose cheapest ket-only path exceeds the limit still plans,
    and every lowered step stays within it."""
    c = {x["name"]: x for x in W.config_c3()}["c3_55_grid6x5_d13"]
    plan = ptn.ptn_plan_path(c["circuit"], c["block_sizes"], hypersamples=100, est_traj=c["n_traj"],
                             est_shots=c["total_shots"], network_form=2)
    d = plan.describe(detail=1)
    assert all(st["n_sum"] <= 24 and st["n_out"] <= 40 for b in d["blocks"] for st in b["steps"])
