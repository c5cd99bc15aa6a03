"""CPU tests of the host side of libptn: the library loads and exports every
symbol of include/ptn.h, planning validates its inputs, and every lowered
plan, replayed on the host by tests/plan_replay.py, reproduces the oracle's
block marginals.  No GPU calls."""
import os
import re
import zlib

import numpy as np
import pytest

import workloads as W
from oracle import pts, statevector as sv
from paper_2604_08467_gb300 import ptn

from plan_replay import run_block

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_header_symbol():
    header = open(os.path.join(ROOT, "include", "ptn.h")).read()
    declared = sorted(set(re.findall(r"^(?:ptn_status|void|const char\*)\s+(ptn_\w+)\s*\(", header, re.M)))
    lib = ptn.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(ptn.exported_symbols())
    assert lib.ptn_version().decode().startswith("ptn")
    assert lib.ptn_status_string(3).decode() == "PTN_ERR_TOO_LARGE"


def test_plan_rejects_non_cptp_channel():
    rng = np.random.default_rng(0)
    circ = W.brickwork_1d(4, 2, rng)
    bad = W.depolarizing_kraus(0.1)
    bad.kraus[0] = bad.kraus[0] * 1.01
    W.attach_noise(circ, [bad])
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_plan_path(circ, [4], hypersamples=2)
    assert e.value.status == 2


@pytest.mark.parametrize("blocks", [[3], [2, 2], [5, 1]])
def test_plan_rejects_bad_blocks(blocks):
    rng = np.random.default_rng(0)
    circ = W.attach_noise(W.brickwork_1d(4, 2, rng), [W.depolarizing_kraus(0.1)])
    if sum(blocks) == 4:
        ptn.ptn_plan_path(circ, blocks, hypersamples=2)
    else:
        with pytest.raises(ptn.PtnError) as e:
            ptn.ptn_plan_path(circ, blocks, hypersamples=2)
        assert e.value.status == 1


def _oracle_rows(circ, kraus, blocks, j, traj, prefix):
    start, b = blocks[j]
    out = []
    cache = {}
    for t, s in zip(traj, prefix):
        if t not in cache:
            cache[t] = np.abs(sv.trajectory_state(circ, kraus[t])) ** 2
        out.append(sv.block_marginals(cache[t], circ.n_qubits, start, b)[int(s) & ((1 << start) - 1)])
    return np.array(out)


CASES = [
    ("brick6", lambda r: W.attach_noise(W.brickwork_1d(6, 5, r), [W.depolarizing_kraus(0.2),
                                                               W.amplitude_damping_kraus(0.3)]), [2, 3, 1]),
    ("brick8", lambda r: W.attach_noise(W.brickwork_1d(8, 6, r), [W.depolarizing_kraus(0.1)]), [3, 3, 2]),
    ("grid3x3", lambda r: W.attach_noise(W.grid_4colour(3, 3, 5, r), [W.depolarizing_kraus(0.1)]), [4, 5]),
    ("hea5", lambda r: W.attach_noise(W.hea_ring(5, 2, r.standard_normal(20)), [W.depolarizing_kraus(0.1)]),
     [2, 2, 1]),
    ("idle_qubit", lambda r: W.attach_noise(W.Circuit(3, [W.Gate((0,), W.haar_u2(r)),
                                                          W.Gate((0, 1), W.CZ.copy())]),
                                            [W.amplitude_damping_kraus(0.4)]), [1, 2]),
    # the paper's random family: Pauli errors and two-qubit depolarizing channels
    ("paper8", lambda r: W.paper_random_circuit(8, 40, r, frac_2q=0.3), [3, 5]),
]


@pytest.mark.parametrize("name,make,bs", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("split,form", [(1, 1), (0, 1), (1, 2), (0, 0)])
def test_lowered_plan_reproduces_oracle_marginals(name, make, bs, split, form):
    """form 1 (DOUBLE_LAYER): double-layer networks; 2 (KET_ONLY): ket-only
    networks (amplitudes of the block and later qubits, then the closing |.|^2
    step); 0 (AUTO): the cheaper of the two per block."""
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    circ = make(rng)
    n = circ.n_qubits
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, split_gates=split, est_traj=4, est_shots=64,
                             network_form=form)
    desc = plan.describe(detail=1)
    kraus, _ = pts.presample(circ, 4, seed=17)
    blocks = plan.blocks
    prng = np.random.default_rng(5)
    for j, (start, b) in enumerate(blocks):
        traj = np.repeat(np.arange(4), 3)
        prefix = prng.integers(0, 1 << start, size=len(traj)) if start else np.zeros(len(traj), int)
        got = run_block(desc, j, kraus, traj, prefix)
        for sched in ("asc", "desc"):   # fused runs: one CTA per trajectory, any interleaving
            assert np.array_equal(run_block(desc, j, kraus, traj, prefix, schedule=sched), got), (j, sched)
        want = _oracle_rows(circ, kraus, blocks, j, traj, prefix)
        err = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
        assert err < 2e-5, (name, j, err)


def test_plan_c1_c2_sizes():
    c1 = W.config_c1()
    p1 = ptn.ptn_plan_path(c1["circuit"], c1["block_sizes"], hypersamples=4, est_traj=64, est_shots=64000)
    d1 = p1.describe()
    assert [b["b"] for b in d1["blocks"]] == [10, 2]
    assert d1["n_sites"] == 184
    c2 = W.config_c2()
    p2 = ptn.ptn_plan_path(c2["circuit"], c2["block_sizes"], hypersamples=4, est_traj=4096, est_shots=1e6)
    d2 = p2.describe()
    assert [b["start"] for b in d2["blocks"]] == [0, 10, 20]
    assert d2["n_sites"] == 1416
    for b in d2["blocks"]:
        assert b["max_out_bits"] <= 40


# ------------------------------------------------ expectation-value plan ----

def _shared_param_circuit(r):
    """Rotations that share angles (parameter 0 on three gates) between CZs."""
    th = r.standard_normal(3)
    g = [W.Gate((0,), W.RY(th[0]), W.PARAM_RY, 0), W.Gate((1,), W.RY(th[0]), W.PARAM_RY, 0),
         W.Gate((0, 1), W.CZ.copy()), W.Gate((2,), W.haar_u2(r)), W.Gate((1, 2), W.CZ.copy()),
         W.Gate((2,), W.RZ(th[1]), W.PARAM_RZ, 1), W.Gate((1,), W.RY(th[2]), W.PARAM_RY, 2),
         W.Gate((0,), W.RY(th[0]), W.PARAM_RY, 0), W.Gate((0, 2), W.CZ.copy())]
    return W.Circuit(3, g)


EV_CASES = [
    ("hea5_dep_ad", lambda r: W.attach_noise(W.hea_ring(5, 2, r.standard_normal(20)),
                                             [W.depolarizing_kraus(0.1), W.amplitude_damping_kraus(0.2)]), [3, 2]),
    ("hea4_noiseless", lambda r: W.hea_ring(4, 3, r.standard_normal(24)), [4]),
    ("shared3", lambda r: W.attach_noise(_shared_param_circuit(r), [W.depolarizing_kraus(0.2)]), [3]),
    ("brick6_hea", lambda r: W.attach_noise(W.Circuit(6, W.brickwork_1d(6, 3, r).gates +
                                                      W.hea_ring(6, 1, r.standard_normal(12)).gates),
                                            [W.amplitude_damping_kraus(0.3)]), [6]),
]


@pytest.mark.parametrize("name,make,bs", EV_CASES, ids=[c[0] for c in EV_CASES])
@pytest.mark.parametrize("split,ckpt", [(1, 0), (0, 0), (1, 1)])
def test_expval_plan_replay(name, make, bs, split, ckpt):
    """The lowered ket network reproduces the oracle's trajectory states and
    expectation values, and every parametrised leaf's adjoint G is the exact
    derivative: sum_e G[e] L'[e] = sum_x w(x) conj(psi(x)) psi'(x), psi' the
    state with that leaf replaced by an arbitrary tensor L' (psi is linear in
    each leaf and F holomorphic in psi with conj(psi) held fixed)."""
    from oracle import gradient as G
    from plan_replay import run_expval
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    circ = make(rng)
    n = circ.n_qubits
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=8, split_gates=split, est_traj=4, est_shots=64,
                             grad_checkpoint=bool(ckpt))
    desc = plan.describe(detail=2)
    ev = desc["expval"]
    if ckpt:   # recomputation steps make the reversed list longer than the adjoint steps alone
        plain = ptn.ptn_plan_path(circ, bs, hypersamples=8, split_gates=split, est_traj=4, est_shots=64)
        ev0 = plain.describe(detail=2)["expval"]
        assert len(ev["bwd"]) >= len(ev0["bwd"])
    assert ev["n_params"] == circ.n_params()
    assert len(ev["pleaves"]) == len(G.rotation_occurrences(circ))
    kraus, _ = pts.presample(circ, 4, seed=23)
    terms = [(0.7, 0b11), (-0.4, (1 << (n - 1)) | 1), (0.25, 0)]
    w = G.pauli_weights(n, terms)
    psi, F, grads = run_expval(desc, kraus, w)
    for sched in ("asc", "desc"):   # fused runs: one CTA per trajectory, any interleaving
        p2, F2, g2 = run_expval(desc, kraus, w, schedule=sched)
        assert np.array_equal(p2, psi) and np.array_equal(F2, F), sched
        assert all(np.array_equal(g2[k], grads[k]) for k in grads), sched
    for t in range(4):
        want = sv.trajectory_state(circ, kraus[t])
        err = np.linalg.norm(psi[t] - want)
        assert err <= 2e-5 * np.linalg.norm(want) + 1e-12, (t, err)   # zero-norm trajectories stay zero
        f = G.trajectory_expval(circ, kraus[t], w)
        assert abs(F[t] - f) < 2e-5 * max(1.0, abs(f)), (t, F[t], f)
    vt0 = np.array(desc["var_table"], dtype=np.float32)
    for p in ev["pleaves"]:
        vt = vt0.copy()
        m = p["n_var"] * p["size"]
        vt[2 * p["var_base"]: 2 * (p["var_base"] + m)] = rng.standard_normal(2 * m).astype(np.float32)
        psi2, _, _ = run_expval(desc, kraus, w, var_table=vt)
        lp = vt[2 * p["var_base"]: 2 * (p["var_base"] + m)].view(np.complex64).reshape(p["n_var"], p["size"])
        from plan_replay import var_ids
        vids = var_ids(desc, kraus)
        for t in range(4):
            var = vids[t, p["var_col"]] if p["var_col"] >= 0 else 0
            lhs = np.sum(grads[p["leaf"]][t].astype(np.complex128) * lp[var])
            rhs = np.sum(w * np.conj(psi[t].astype(np.complex128)) * psi2[t])
            assert abs(lhs - rhs) < 1e-4 * max(1.0, abs(rhs)), (p["leaf"], t, lhs, rhs)


def _fused_runs(steps):
    runs, cur = [], []
    for st in steps:
        if st["fuse_prev"]:
            cur.append(st)
        else:
            if len(cur) > 1:
                runs.append(cur)
            cur = [st]
    if len(cur) > 1:
        runs.append(cur)
    return runs


def test_fused_runs_share_no_addresses_across_trajectories():
    """Instances of a buffer sit one after another in its arena (offset x
    instances + instance x size), so two buffers of one fused run whose
    per-instance ranges overlap without coinciding would share addresses
    between different trajectories' CTAs.  Every pair of ranges of one run, at
    least one of them written, is disjoint or identical; the runs of the
    100-qubit workload stay long (the gate-level start of each block is one
    launch); and a run starts only at a small direct trajectory-class step."""
    c2 = W.config_c2()
    plan = ptn.ptn_plan_path(c2["circuit"], c2["block_sizes"], hypersamples=8, est_traj=4096, est_shots=1e6)
    d = plan.describe(1)
    for blk in d["blocks"]:
        runs = _fused_runs(blk["steps"])
        assert max(len(r) for r in runs) >= 100
        for run in runs:
            rng = []
            for st in run:
                assert st["kind"] == 0 and st["out_cls"] == 1 and st["n_out"] <= 12 and st["n_sum"] <= 8
                rng += [(o["arena"], o["arena_off"], o["inst_size"], False) for o in st["ops"] if o["mode"] == 1]
                rng.append((st["out_arena"], st["out_off"], 1 << st["n_out"], True))
            rng.sort()
            for a in range(len(rng)):
                for b in range(a + 1, len(rng)):
                    x, y = rng[a], rng[b]
                    if y[0] != x[0] or y[1] >= x[1] + x[2]:
                        break
                    if (x[3] or y[3]) and (x[1], x[2]) != (y[1], y[2]):
                        raise AssertionError(f"fused run shares addresses: {x} {y}")


def test_gemm_operands_have_contiguous_summed_bits():
    """Producers lay out their outputs with the consumer's summed bits
    innermost, so tensor-core steps read the summed axis of their intermediate
    operands contiguously (the packing's coalesced path).  An operand reached
    through a slice view or shared by a mirrored pair can keep another order,
    so the bound is on the fraction."""
    c2 = W.config_c2()
    plan = ptn.ptn_plan_path(c2["circuit"], c2["block_sizes"], hypersamples=8, est_traj=4096, est_shots=1e6)
    d = plan.describe(1)
    n = ok = 0
    for blk in d["blocks"]:
        for st in blk["steps"]:
            if st["kind"] == 0:
                continue
            for o in range(2):
                if st["ops"][o]["mode"] != 1:      # intermediate (arena) operand
                    continue
                n += 1
                ok += st["sum_stride"][o] == [1 << q for q in range(st["n_sum"])]
    assert n > 20 and ok >= 0.9 * n, (ok, n)
