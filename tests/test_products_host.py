"""Outer products formed in the operand pack (ptn_plan_opts.keep_products = 0),
host side: the planner's marks checked against the step graph (a marked step
has no summed bits, is read only by the tensor-core operand it is marked for,
and no step in between writes into its factors' arena ranges), the plan is
otherwise the same as with keep_products = 1, and a host replay that skips the
marked steps (their outputs poisoned with NaN) and forms the operand from the
factors at the consumer equals the materialised replay and the statevector
oracle.  No GPU."""
import numpy as np
import pytest

import workloads as W
from oracle import pts
from oracle import statevector as sv
from paper_2604_08467_gb300 import ptn
from plan_replay import run_block
from test_cache_host import _subtree_columns


def _strip(obj):
    if isinstance(obj, dict):
        return {k: _strip(v) for k, v in obj.items() if k not in ("virt", "prod", "prod_src", "plan_seconds")}
    if isinstance(obj, list):
        return [_strip(v) for v in obj]
    return obj


def _check_marks(desc):
    n_marks = 0
    for blk in desc["blocks"]:
        steps = blk["steps"]
        _, producer, _ = _subtree_columns(steps)
        consumers = {}
        for g, st in enumerate(steps):
            for x, k in enumerate(producer[g]):
                if k is not None:
                    consumers.setdefault(k, []).append((g, x))
        for g, G in enumerate(steps):
            if not G["prod"]:
                continue
            n_marks += 1
            x, k = G["prod"] - 1, G["prod_src"]
            P = steps[k]
            assert G["kind"] in (1, 2) and P["virt"] == 1 and P["kind"] == 0 and P["n_sum"] == 0
            assert producer[g][x] == k and consumers[k] == [(g, x)]
            assert not G["ops"][x]["slices"]
            assert all(op["inst_size"] <= 1 << 31 for op in P["ops"])
            for s in range(k + 1, g):
                S = steps[s]
                for f in P["ops"]:
                    if f["mode"] == 1 and f["arena"] == S["out_arena"]:
                        assert (f["arena_off"] >= S["out_off"] + (1 << S["n_out"])
                                or S["out_off"] >= f["arena_off"] + f["inst_size"]), (k, g, s)
        virt = [i for i, st in enumerate(steps) if st["virt"]]
        assert sorted(virt) == sorted(st["prod_src"] for st in steps if st["prod"])
    return n_marks


def _circuit20():
    rng = np.random.default_rng(0)
    return W.attach_noise(W.brickwork_1d(20, 8, rng), [W.depolarizing_kraus(0.01)])


def test_product_marks_c2_and_20_qubits():
    """The benchmarked 30-qubit plan and a 20-qubit brickwork: every mark is
    valid, there is at least one, and keep_products = 1 gives the same plan
    without them."""
    c2 = W.config_c2()
    cases = [(c2["circuit"], c2["block_sizes"], dict(hypersamples=100, est_traj=4096, est_shots=1e6)),
             (_circuit20(), [10, 10], dict(hypersamples=8, est_traj=64, est_shots=4096, network_form=1))]
    for circ, bs, kw in cases:
        desc = ptn.ptn_plan_path(circ, bs, **kw).describe(detail=1)
        assert _check_marks(desc) >= 1
        keep = ptn.ptn_plan_path(circ, bs, keep_products=True, **kw).describe(detail=1)
        assert _check_marks(keep) == 0
        assert _strip(keep) == _strip(desc)


def test_product_replay_equals_materialised_and_oracle():
    circ = _circuit20()
    kw = dict(hypersamples=8, est_traj=64, est_shots=4096, network_form=1)
    desc = ptn.ptn_plan_path(circ, [10, 10], **kw).describe(detail=1)
    keep = ptn.ptn_plan_path(circ, [10, 10], keep_products=True, **kw).describe(detail=1)
    assert any(st["prod"] for st in desc["blocks"][1]["steps"])
    kraus, _ = pts.presample(circ, 3, seed=4)
    traj = np.repeat(np.arange(3), 2)
    prefix = np.random.default_rng(2).integers(0, 1 << 10, size=len(traj))
    got = run_block(desc, 1, kraus, traj, prefix)
    assert not np.isnan(got).any()
    assert np.array_equal(got, run_block(keep, 1, kraus, traj, prefix))
    want = []
    for t, s in zip(traj, prefix):
        p = np.abs(sv.trajectory_state(circ, kraus[t])) ** 2
        want.append(sv.block_marginals(p, 20, 10, 10)[int(s)])
    want = np.array(want)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5
