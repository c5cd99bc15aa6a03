"""Intermediate caching across error sets (Sec. VI), host side: the planner's
cache marks checked against column sets recomputed here from the lowered step
graph, and a host replay that computes cached steps for representative
trajectories only (the other instances poisoned with NaN) against the plain
replay and the statevector oracle.  No GPU."""
import zlib

import numpy as np
import pytest

import workloads as W
from oracle import pts
from oracle import statevector as sv
from paper_2604_08467_gb300 import ptn
from plan_replay import run_block, var_ids

CACHE_MIN_WORK = 4096
CACHE_MIN_OUT_BITS = 7
SMALL_OUT, SMALL_SUM, SMALL_OP = 12, 8, 14


def _small(st):
    return (st["kind"] == 0 and st["out_cls"] == 1 and st["n_out"] <= SMALL_OUT and st["n_sum"] <= SMALL_SUM
            and all(op["inst_size"] <= 1 << SMALL_OP for op in st["ops"]))


def _subtree_columns(steps):
    """Per step, the variant columns of its subtree's leaves, by following every
    buffer operand back to the last step that wrote its arena address."""
    written, cols, producer = {}, [], []
    for i, st in enumerate(steps):
        acc, prod = set(), []
        for op in st["ops"]:
            if op["mode"] == 0:
                if op["leaf_col"] >= 0:
                    acc.add(op["leaf_col"])
                prod.append(None)
            else:
                k = written.get((op["arena"], op["arena_off"]))
                prod.append(k)
                if k is not None:
                    acc |= cols[k]
        cols.append(acc)
        producer.append(prod)
        written[(st["out_arena"], st["out_off"])] = i
    return cols, producer, written


def _eligible(steps, i, cols, fuse_max):
    st = steps[i]
    fused = fuse_max != 1 and _small(st) and (st["fuse_prev"] or (i + 1 < len(steps) and steps[i + 1]["fuse_prev"]))
    return (st["out_cls"] == 1 and st["kind"] != 2 and not fused and bool(cols[i])
            and st["n_out"] >= CACHE_MIN_OUT_BITS and 2 ** (st["n_out"] + st["n_sum"]) >= CACHE_MIN_WORK)


def _strip_cache(obj):
    if isinstance(obj, dict):
        return {k: _strip_cache(v) for k, v in obj.items() if k not in ("cache", "n_cache", "cache_cols",
                                                                         "plan_seconds")}
    if isinstance(obj, list):
        return [_strip_cache(v) for v in obj]
    return obj


@pytest.mark.parametrize("form", [0, 1, 2])
def test_cache_marks_match_subtree_columns(form):
    """On the 30-qubit brickwork plan: every step the rules admit (trajectory
    class, not stacked, not in a fused run, >= 2^7 outputs, >= 4096 MACs, some
    variant column) is cached and no other; slot k lists exactly the columns of
    its subtree; every read of a cached buffer (the root's too) carries its
    producer's slot; with caching off the plan is the same apart from the
    marks."""
    c2 = W.config_c2()
    kw = dict(hypersamples=8, est_traj=4096, est_shots=1e6, network_form=form)
    plan = ptn.ptn_plan_path(c2["circuit"], c2["block_sizes"], cache_intermediates=True, **kw)
    desc = plan.describe(detail=1)
    total = 0
    for blk in desc["blocks"]:
        steps = blk["steps"]
        cols, producer, written = _subtree_columns(steps)
        slot = 0
        for i, st in enumerate(steps):
            want = _eligible(steps, i, cols, 1024)
            assert bool(st["cache"]) == want, (i, st["cache"])
            if want:
                slot += 1
                assert st["cache"] == slot
                assert blk["cache_cols"][slot - 1] == sorted(cols[i])
            for op, k in zip(st["ops"], producer[i]):
                exp = steps[k]["cache"] if (k is not None and op["cls"] == 1) else 0
                assert op["cache"] == exp, (i, op["cache"], exp)
        assert blk["n_cache"] == slot == len(blk["cache_cols"])
        total += slot
        r = blk["root"]["op"]
        if r["mode"] == 1:
            k = written[(r["arena"], r["arena_off"])]
            assert r["cache"] == (steps[k]["cache"] if r["cls"] == 1 else 0)
    assert total > 0
    plain = ptn.ptn_plan_path(c2["circuit"], c2["block_sizes"], cache_intermediates=False, **kw).describe(detail=1)
    assert all(b["n_cache"] == 0 for b in plain["blocks"])
    assert _strip_cache(plain) == _strip_cache(desc)


def _cases():
    out = [("c1", W.config_c1()["circuit"], [10, 2])]
    rng = np.random.default_rng(zlib.crc32(b"brick14"))
    out.append(("brick14", W.attach_noise(W.brickwork_1d(14, 6, rng), [W.depolarizing_kraus(0.01)]), [8, 6]))
    return out


def _near_copies(circ, seed):
    """Eight Kraus index rows: four drawn by pre-sampling and, for each, a copy
    that differs from it at one site only, index 0 <-> 1 (every site of these
    circuits has at least two Kraus operators); a copy shares every
    intermediate whose subtree misses that site."""
    kraus, _ = pts.presample(circ, 4, seed=seed)
    rng = np.random.default_rng(seed)
    rows = [r.copy() for r in kraus]
    for r in kraus:
        c = r.copy()
        s = int(rng.integers(0, len(c)))
        c[s] = 1 if c[s] == 0 else 0
        rows.append(c)
    return np.array(rows)


def _oracle_rows(circ, kraus, start, b, traj, prefix):
    cache, out = {}, []
    for t, s in zip(traj, prefix):
        if t not in cache:
            cache[t] = np.abs(sv.trajectory_state(circ, kraus[t])) ** 2
        out.append(sv.block_marginals(cache[t], circ.n_qubits, start, b)[int(s)])
    return np.array(out)


@pytest.mark.parametrize("name,circ,bs", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("form", [1, 2])
def test_cached_replay_equals_plain_replay_and_oracle(name, circ, bs, form):
    """Every step launched on its own (fuse_max = 1), so the gate-level steps
    are cached too: the replay that computes cached steps for representatives
    only gives the same marginals bit for bit as the plain replay (no poisoned
    instance is read) and matches the statevector oracle."""
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=8, est_shots=64, network_form=form,
                             cache_intermediates=True, fuse_max=1)
    desc = plan.describe(detail=1)
    assert desc["blocks"][0]["n_cache"] > 0
    kraus = _near_copies(circ, 3)
    vids = var_ids(desc, kraus)
    prng = np.random.default_rng(11)
    shared = 0
    for j, (start, b) in enumerate(plan.blocks):
        traj = np.repeat(np.arange(8), 2)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        got = run_block(desc, j, kraus, traj, prefix, cache=True)
        assert np.array_equal(got, run_block(desc, j, kraus, traj, prefix)), j
        want = _oracle_rows(circ, kraus, start, b, traj, prefix)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5
        for cols in desc["blocks"][j]["cache_cols"]:
            shared += 8 - len({tuple(r) for r in vids[:, cols]})
    assert shared > 0   # some cached step is really shared between trajectories


def test_dropped_cache_column_is_caught():
    """Planted mistake: removing from a slot's list a column on which two
    trajectories differ while agreeing on the rest makes them share a wrong
    intermediate, and the cached replay no longer equals the plain one."""
    name, circ, bs = _cases()[0]
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, est_traj=8, est_shots=64, network_form=1,
                             cache_intermediates=True, fuse_max=1)
    desc = plan.describe(detail=1)
    kraus, _ = pts.presample(circ, 32, seed=5)
    vids = var_ids(desc, kraus)
    blk = desc["blocks"][0]
    for k, cols in enumerate(blk["cache_cols"]):
        for c in cols:
            rest = [x for x in cols if x != c]
            seen = {}
            for t in range(len(kraus)):
                key = tuple(vids[t, rest])
                if key in seen and vids[seen[key], c] != vids[t, c]:
                    blk["cache_cols"][k] = rest
                    traj = np.arange(len(kraus))
                    prefix = np.zeros(len(traj), int)
                    bad = run_block(desc, 0, kraus, traj, prefix, cache=True)
                    blk["cache_cols"][k] = cols
                    good = run_block(desc, 0, kraus, traj, prefix, cache=True)
                    assert np.array_equal(good, run_block(desc, 0, kraus, traj, prefix))
                    assert not np.array_equal(bad, good)
                    return
                seen.setdefault(key, t)
    pytest.fail("no column separates two otherwise equal trajectories")
