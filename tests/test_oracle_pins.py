"""Pins of the CPU oracle to facts fixed outside the oracle itself: published
known-answer vectors, closed forms, brute force on tiny inputs, invariants and
special cases.  CPU only."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import densmat, mps, philox, pts, sampling, statevector as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[0:4], *v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_mulhi64_exact():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**63, size=2000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=2000, dtype=np.uint64)
    t = rng.integers(1, 2**53, size=2000, dtype=np.uint64)
    got = philox.mulhi64(a, t)
    want = [(int(x) * int(y)) >> 64 for x, y in zip(a, t)]
    assert [int(g) for g in got] == want
    assert int(philox.mulhi64(np.uint64(2**64 - 1), np.uint64(2**53))) == 2**53 - 1


def test_uniform53_range():
    u = philox.uniform53(np.array([0, 0xFFFFFFFF], np.uint64), np.array([0, 0xFFFFFFFF], np.uint64))
    assert u[0] == 0.0 and u[1] < 1.0 and u[1] == 1.0 - 2.0**-53


# ------------------------------------------------------- Kraus channels ----

@pytest.mark.parametrize("p", [0.0, 0.003, 0.01, 0.2, 0.75])
def test_depolarizing_completeness_and_action(p):
    ch = W.depolarizing_kraus(p)
    assert pts.completeness_error(ch.kraus) < 1e-14
    q = pts.kraus_probs(ch.kraus)
    assert abs(q.sum() - 1) < 1e-15
    np.testing.assert_allclose(q, [1 - p, p / 3, p / 3, p / 3], atol=1e-15)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    rho = a @ a.conj().T
    rho /= np.trace(rho)
    x = np.array([[0, 1], [1, 0]]); y = np.array([[0, -1j], [1j, 0]]); z = np.diag([1, -1])
    closed = (1 - p) * rho + p / 3 * (x @ rho @ x + y @ rho @ y + z @ rho @ z)
    got = sum(k @ rho @ k.conj().T for k in ch.kraus)
    np.testing.assert_allclose(got, closed, atol=1e-14)
    if p == 0.75:   # fully depolarising: maps every state to I/2
        np.testing.assert_allclose(got, np.eye(2) / 2, atol=1e-14)


@pytest.mark.parametrize("g", [0.0, 0.002, 0.3, 1.0])
def test_amplitude_damping_closed_form(g):
    ch = W.amplitude_damping_kraus(g)
    assert pts.completeness_error(ch.kraus) < 1e-14
    one = np.diag([0.0, 1.0]).astype(complex)
    got = sum(k @ one @ k.conj().T for k in ch.kraus)
    np.testing.assert_allclose(got, np.diag([g, 1 - g]), atol=1e-15)
    plus = np.full((2, 2), 0.5, dtype=complex)
    got = sum(k @ plus @ k.conj().T for k in ch.kraus)
    want = np.array([[0.5 + 0.5 * g, 0.5 * math.sqrt(1 - g)], [0.5 * math.sqrt(1 - g), 0.5 - 0.5 * g]])
    np.testing.assert_allclose(got, want, atol=1e-15)
    np.testing.assert_allclose(pts.kraus_probs(ch.kraus), [1 - g / 2, g / 2], atol=1e-15)


def test_cdf_last_entry_is_one():
    for ch in (W.depolarizing_kraus(0.01), W.amplitude_damping_kraus(0.002)):
        c = pts.kraus_cdf(ch.kraus)
        assert c[-1] == 1.0 and np.all(np.diff(c) >= 0)


def test_haar_u2_unitary():
    rng = np.random.default_rng(0)
    for _ in range(20):
        u = W.haar_u2(rng)
        np.testing.assert_allclose(u @ u.conj().T, np.eye(2), atol=1e-14)


# ---------------------------------------------------------- pre-sampling ----

def test_presample_frequencies_match_q():
    rng = np.random.default_rng(5)
    circ = W.attach_noise(W.brickwork_1d(4, 2, rng), [W.depolarizing_kraus(0.2)])
    k, logq = pts.presample(circ, 4000, seed=123)
    counts = np.bincount(k.reshape(-1), minlength=4)
    n = k.size
    exp = n * np.array([0.8, 0.2 / 3, 0.2 / 3, 0.2 / 3])
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    assert chi2 < 16.3            # chi2(3) at p = 1e-3
    q = pts.kraus_probs(circ.channels[0].kraus)
    np.testing.assert_allclose(logq, np.log(q)[k].sum(axis=1), rtol=1e-13)


def test_presample_counter_addressing():
    """Draws depend only on (seed, site, trajectory): a subset reproduces."""
    circ = W.config_c1()["circuit"]
    k_all, _ = pts.presample(circ, 16, seed=99)
    k_few, _ = pts.presample(circ, 4, seed=99)
    assert np.array_equal(k_all[:4], k_few)
    k_other, _ = pts.presample(circ, 4, seed=100)
    assert not np.array_equal(k_other, k_few)


def test_dedup_first_occurrence():
    k = np.array([[0, 1], [0, 0], [0, 1], [2, 0], [0, 0]], dtype=np.uint8)
    lq = np.arange(5, dtype=float)
    ku, lu, mult, first = pts.dedup(k, lq)
    assert first.tolist() == [0, 1, 3]
    assert mult.tolist() == [2, 2, 1]
    assert np.array_equal(ku, k[[0, 1, 3]])


# ---------------------------------------------------------- state vector ----

def _full_operator(n, qubits, m):
    """Brute force: the 2^n x 2^n matrix of a gate, built element by element."""
    d = 1 << n
    out = np.zeros((d, d), dtype=np.complex128)
    for col in range(d):
        for row in range(d):
            rest_ok = all(((row >> q) & 1) == ((col >> q) & 1) for q in range(n) if q not in qubits)
            if not rest_ok:
                continue
            if len(qubits) == 1:
                q = qubits[0]
                out[row, col] = m[(row >> q) & 1, (col >> q) & 1]
            else:
                a, b = qubits
                r = (((row >> a) & 1) << 1) | ((row >> b) & 1)
                c = (((col >> a) & 1) << 1) | ((col >> b) & 1)
                out[row, col] = m[r, c]
    return out


@pytest.mark.parametrize("qubits", [(0,), (2,), (0, 1), (1, 0), (3, 1), (0, 3)])
def test_apply_gate_brute_force(qubits):
    n = 4
    rng = np.random.default_rng(7)
    d = 1 << len(qubits)
    m = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    got = sv.apply_gate(psi, n, qubits, m)
    np.testing.assert_allclose(got, _full_operator(n, qubits, m) @ psi, atol=1e-12)


def test_bell_state_distribution():
    h = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    circ = W.Circuit(2, [W.Gate((0,), h.astype(complex)), W.Gate((1,), h.astype(complex)),
                         W.Gate((0, 1), W.CZ.copy()), W.Gate((1,), h.astype(complex))])
    p = np.abs(sv.pure_state(circ)) ** 2
    np.testing.assert_allclose(p, [0.5, 0, 0, 0.5], atol=1e-15)   # H(0) then CNOT(0->1)


def test_hadamard_layer_uniform_marginals():
    h = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
    n = 6
    circ = W.Circuit(n, [W.Gate((q,), h) for q in range(n)])
    p = np.abs(sv.pure_state(circ)) ** 2
    for start, b in [(0, 4), (4, 2)]:
        m = sv.block_marginals(p, n, start, b)
        np.testing.assert_allclose(m, np.full(m.shape, 1.0 / (1 << n) * (1 << (n - start - b))), atol=1e-15)


def test_zero_noise_is_pure_circuit():
    rng = np.random.default_rng(11)
    circ = W.attach_noise(W.brickwork_1d(6, 4, rng),
                          [W.depolarizing_kraus(0.0), W.amplitude_damping_kraus(0.0)])
    k, logq = pts.presample(circ, 3, seed=5)
    assert np.all(k == 0) and np.all(logq == 0.0)
    np.testing.assert_allclose(sv.trajectory_state(circ, k[0]), sv.pure_state(circ), atol=1e-14)


def test_depolarizing_trajectories_unit_norm():
    circ = W.config_c1()["circuit"]
    k, _ = pts.presample(circ, 4, seed=7)
    for i in range(4):
        assert abs(np.linalg.norm(sv.trajectory_state(circ, k[i])) - 1) < 1e-12


def test_trajectory_average_converges_to_density_matrix():
    """mean_i |psi_i><psi_i| -> rho at rate O(1/sqrt(E)) (unbiased estimator)."""
    rng = np.random.default_rng(13)
    circ = W.attach_noise(W.brickwork_1d(3, 3, rng),
                          [W.depolarizing_kraus(0.15), W.amplitude_damping_kraus(0.3)])
    rho = densmat.density_matrix(circ)
    assert abs(np.trace(rho) - 1) < 1e-12
    errs = []
    for e in (250, 4000):
        k, _ = pts.presample(circ, e, seed=77)
        acc = np.zeros_like(rho)
        for i in range(e):
            psi = sv.trajectory_state(circ, k[i])
            acc += np.outer(psi, psi.conj())
        errs.append(np.linalg.norm(acc / e - rho))
    assert errs[1] < 3.0 / math.sqrt(4000)
    assert errs[1] < errs[0]


def test_dropped_kraus_scale_breaks_convergence():
    """Planted mistake: inserting K_k without the 1/sqrt(q_k) factor biases the
    average away from rho, which the convergence pin detects."""
    rng = np.random.default_rng(13)
    circ = W.attach_noise(W.brickwork_1d(3, 3, rng), [W.depolarizing_kraus(0.15)])
    rho = densmat.density_matrix(circ)
    k, _ = pts.presample(circ, 2000, seed=77)
    acc = np.zeros_like(rho)
    for i in range(2000):
        psi = np.zeros(8, complex); psi[0] = 1
        for l, g in enumerate(circ.gates):
            m = g.matrix
            for s, site in enumerate(circ.sites):
                if site.gate == l:
                    kk = circ.channels[site.channel].kraus[k[i, s]]     # unscaled
                    m = (np.kron(kk, np.eye(2)) if g.arity == 2 and site.qubit == g.qubits[0]
                         else np.kron(np.eye(2), kk) if g.arity == 2 else kk) @ m
            psi = sv.apply_gate(psi, 3, g.qubits, m)
        acc += np.outer(psi, psi.conj())
    assert np.linalg.norm(acc / 2000 - rho) > 3 * 3.0 / math.sqrt(2000)


def test_block_marginals_parent_child_identity():
    circ = W.config_c1()["circuit"]
    k, _ = pts.presample(circ, 2, seed=3)
    psi = sv.trajectory_state(circ, k[1])
    p = np.abs(psi) ** 2
    m1 = sv.block_marginals(p, 12, 0, 10)      # [1, 1024]
    m2 = sv.block_marginals(p, 12, 10, 2)      # [1024, 4]
    np.testing.assert_allclose(m2.sum(axis=1), m1[0], rtol=1e-12, atol=1e-18)
    assert abs(m1.sum() - np.linalg.norm(psi) ** 2) < 1e-12


# ------------------------------------------------------------------- MPS ----

def test_mps_matches_statevector():
    cfg = W.config_c2(n_traj=4)
    rng = np.random.default_rng(21)
    circ = W.attach_noise(W.brickwork_1d(12, 12, rng), cfg["circuit"].channels)
    k, _ = pts.presample(circ, 3, seed=cfg["seed"])
    for i in range(3):
        psi = sv.trajectory_state(circ, k[i])
        p = np.abs(psi) ** 2
        m = mps.trajectory_mps(circ, k[i])
        for start, b in [(0, 4), (4, 4), (8, 4)]:
            ref = sv.block_marginals(p, 12, start, b)
            for prefix in (0, 5, (1 << start) - 1):
                if prefix >= (1 << start) and start > 0:
                    continue
                got = m.block_marginal(start, b, prefix if start else 0)
                np.testing.assert_allclose(got, ref[prefix if start else 0], rtol=1e-10, atol=1e-15)


# -------------------------------------------------------------- sampling ----

def test_quantise_is_exact_integer_cdf():
    rows = W.synthetic_marginals(20, 10, seed=4)
    for r in rows:
        P, C = sampling.quantise(r)
        assert np.all(P == np.floor(P)) and C[-1] <= 2.0**52
        assert C[-1] == float(sum(int(x) for x in P))
        assert np.all((P == 0) == (r <= 0))   # scale keeps every nonzero entry


def test_inverse_cdf_never_picks_zero_bins_and_matches_law():
    p = np.array([0.0, 1.0, 0.0, 2.0, 5.0, 0.0, 0.0, 2.0])
    _, C = sampling.quantise(p)
    a = sampling.draw_words(np.arange(200000, dtype=np.uint64), np.uint64(0), 77, seed=1)
    x = sampling.inverse_cdf(C, a)
    cnt = np.bincount(x, minlength=8)
    assert cnt[[0, 2, 5, 6]].sum() == 0
    exp = 200000 * p / p.sum()
    nz = exp > 0
    assert float(np.sum((cnt[nz] - exp[nz]) ** 2 / exp[nz])) < 16.3


def test_inverse_cdf_boundaries():
    """r = 0 picks the first positive bin; the largest word picks the last positive bin."""
    C = np.array([0.0, 3.0, 3.0, 10.0])
    a = np.array([0, 2**64 - 1], dtype=np.uint64)
    assert sampling.inverse_cdf(C, a).tolist() == [1, 3]


def test_single_block_is_plain_sampling():
    """One block covering all qubits reduces NBS to plain sampling of |psi|^2."""
    rng = np.random.default_rng(31)
    circ = W.attach_noise(W.brickwork_1d(5, 4, rng), [W.depolarizing_kraus(0.05)])
    k, _ = pts.presample(circ, 2, seed=9)
    probs = [np.abs(sv.trajectory_state(circ, k[i])) ** 2 for i in range(2)]

    def marg(j, traj, prefix):
        return np.stack([probs[t] for t in traj])

    traj, bits, cnt, levels, m = sampling.nbs_proportional(marg, [(0, 5)], seed=3, n_traj=2,
                                                           shots=[50000, 50000])
    for t in range(2):
        h = np.zeros(32)
        h[bits[traj == t].astype(int)] = cnt[traj == t]
        exp = 50000 * probs[t] / probs[t].sum()
        nz = exp > 5
        assert float(np.sum((h[nz] - exp[nz]) ** 2 / exp[nz])) < 2 * nz.sum() + 30


def test_nbs_law_equals_joint_distribution():
    """Block-by-block conditional sampling draws from the joint |psi|^2 law, and
    carries every shot (sum of counts = m_i) in canonical order."""
    rng = np.random.default_rng(41)
    circ = W.attach_noise(W.brickwork_1d(6, 5, rng), [W.depolarizing_kraus(0.05)])
    k, _ = pts.presample(circ, 3, seed=2)
    probs = [np.abs(sv.trajectory_state(circ, k[i])) ** 2 for i in range(3)]
    blocks = [(0, 2), (2, 3), (5, 1)]

    def marg(j, traj, prefix):
        start, b = blocks[j]
        return np.stack([sv.block_marginals(probs[t], 6, start, b)[int(s)]
                         for t, s in zip(traj, prefix)])

    shots = [40000, 1, 30000]
    traj, bits, cnt, levels, m = sampling.nbs_proportional(marg, blocks, seed=5, n_traj=3,
                                                           shots=shots)
    for t in range(3):
        assert cnt[traj == t].sum() == shots[t]
    keys = list(zip(traj.tolist(), bits.tolist()))
    assert len(set(keys)) == len(keys)
    # canonical: per trajectory, sorted by (x1, x2, x3) with block 1 most significant
    def lex(bt):
        return tuple(((bt >> s) & ((1 << b) - 1)) for s, b in blocks)
    for t in range(3):
        bt = bits[traj == t].tolist()
        assert bt == sorted(bt, key=lex)
    for t in (0, 2):
        h = np.zeros(64)
        h[bits[traj == t].astype(int)] = cnt[traj == t]
        exp = shots[t] * probs[t] / probs[t].sum()
        nz = exp > 5
        assert float(np.sum((h[nz] - exp[nz]) ** 2 / exp[nz])) < 2 * nz.sum() + 30


def test_allocation_sums_and_proportionality():
    w = np.array([1.0, 3.0, 0.0, 6.0])
    m = sampling.allocate_shots(w, 100000, seed=8)
    assert m.sum() == 100000 and m[2] == 0
    exp = 100000 * w / w.sum()
    nz = exp > 0
    assert float(np.sum((m[nz] - exp[nz]) ** 2 / exp[nz])) < 13.8


def test_rank_offsets():
    assert sampling.rank_offsets([0, 0, 1, 1, 1], [3, 2, 1, 4, 2]).tolist() == [0, 3, 0, 1, 5]


def test_zero_norm_parent_drops_its_shots():
    rows = np.array([[0.0, 0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 3.0]])
    par, xs, cs = sampling.sample_block(rows, [0, 1], [5, 7], [0, 0], seed=1, block=0)
    assert set(par.tolist()) == {1} and cs.sum() == 7
    assert sampling.allocate_shots(np.zeros(3), 10, seed=1).tolist() == [0, 0, 0]


# ------------------------------------------------ gradients (oracle.gradient) ----

def test_rotation_is_matrix_exponential():
    from scipy.linalg import expm
    from oracle import gradient as G
    y = np.array([[0, -1j], [1j, 0]]); z = np.diag([1.0, -1.0])
    for t in (-2.3, 0.0, 0.7, 3.9):
        np.testing.assert_allclose(G.rotation(G.PARAM_RY, t), expm(-0.5j * t * y), atol=1e-14)
        np.testing.assert_allclose(G.rotation(G.PARAM_RZ, t), expm(-0.5j * t * z), atol=1e-14)


def test_expval_grad_closed_form_two_qubits():
    """RY(a) (x) RY(b) then CZ on |00>: <Z0 Z1> = cos a cos b (CZ commutes with
    Z Z), <Z0> = cos a, and RZ angles do not enter."""
    from oracle import gradient as G
    a, b, c = 0.9, -1.7, 0.4
    circ = W.Circuit(2, [W.Gate((0,), W.RY(0), W.PARAM_RY, 0), W.Gate((1,), W.RY(0), W.PARAM_RY, 1),
                         W.Gate((1,), W.RZ(0), W.PARAM_RZ, 2), W.Gate((0, 1), W.CZ.copy())])
    rows, mult = np.zeros((1, 0), np.uint8), [1]
    th = [a, b, c]
    assert abs(G.expval(circ, rows, mult, [(1.0, 0b11)], th) - np.cos(a) * np.cos(b)) < 1e-14
    g = G.expval_grad_shift(circ, rows, mult, [(1.0, 0b11), (0.5, 0b01)], th)
    want = [-np.sin(a) * np.cos(b) - 0.5 * np.sin(a), -np.cos(a) * np.sin(b), 0.0]
    np.testing.assert_allclose(g, want, atol=1e-14)


def test_expval_grad_shift_matches_finite_differences():
    """Parameter shift (exact) against central differences (O(h^2)) on sampled
    noisy trajectories, shared angles included."""
    from oracle import gradient as G
    rng = np.random.default_rng(11)
    th = rng.standard_normal(12)
    circ = W.attach_noise(W.hea_ring(3, 2, th), [W.depolarizing_kraus(0.1), W.amplitude_damping_kraus(0.2)])
    circ.gates[6].param_index = 0          # a second occurrence of angle 0
    kraus, _ = pts.presample(circ, 12, seed=4)
    terms = [(0.5, 0b011), (0.5, 0b110), (-0.2, 0b100)]
    g1 = G.expval_grad_shift(circ, kraus, np.arange(1, 13), terms, th)
    g2 = G.expval_grad_fd(circ, kraus, np.arange(1, 13), terms, th, h=1e-5)
    np.testing.assert_allclose(g1, g2, atol=1e-9)
    assert np.abs(g1).max() > 1e-2


def test_expval_enumeration_equals_density_matrix():
    """Averaging the unnormalised trajectory expectations over every Kraus
    combination with weight prod q_k gives Tr(O rho) exactly, and so does its
    gradient: the trajectory form is checked against the FP64 density-matrix
    gradient (parameter shift on the exact channel evolution)."""
    import itertools
    from oracle import gradient as G
    rng = np.random.default_rng(2)
    th = rng.standard_normal(4)
    circ = W.attach_noise(W.hea_ring(2, 1, th), [W.depolarizing_kraus(0.15)])
    circ.sites = [s for s in circ.sites if s.gate in (0, 3, 4)]     # 4 sites: 256 combinations
    q = pts.kraus_probs(circ.channels[0].kraus)
    rows = np.array(list(itertools.product(range(4), repeat=len(circ.sites))), dtype=np.uint8)
    weight = np.prod(q[rows], axis=1)
    terms = [(1.0, 0b11), (0.3, 0b01)]
    f_traj = G.expval(circ, rows, weight, terms, th)
    f_dm = G.density_expval(circ, terms, th)
    assert abs(f_traj - f_dm) < 1e-12
    g_traj = G.expval_grad_shift(circ, rows, weight, terms, th)
    g_dm = G.density_grad_shift(circ, terms, th)
    np.testing.assert_allclose(g_traj, g_dm, atol=1e-12)
    assert np.abs(g_dm).max() > 1e-2


def test_density_row_application_equals_column_loop():
    """The density-matrix left action (one 2n-qubit gate application) equals
    applying the gate to each column of rho separately."""
    from oracle import densmat
    rng = np.random.default_rng(8)
    n = 4
    rho = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    for qubits in [(0,), (3,), (1, 2), (3, 0)]:
        m = W.haar_u2(rng) if len(qubits) == 1 else np.kron(W.haar_u2(rng), W.haar_u2(rng)) @ W.CZ
        loop = np.stack([sv.apply_gate(rho[:, c], n, qubits, m) for c in range(16)], axis=1)
        np.testing.assert_allclose(densmat._apply_left(rho, n, qubits, m), loop, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2])
def test_adjoint_gradients_match_parameter_shift(seed):
    """Reverse-mode gradients (state vector per trajectory, and the density
    matrix) equal the parameter-shift rule, which is exact for rotations, on
    small noisy ansatz circuits with shared angles and amplitude damping."""
    from oracle import gradient as G, pts as P
    r = np.random.default_rng(seed)
    th = r.standard_normal(5 * 2 * 2)
    circ = W.attach_noise(W.hea_ring(5, 2, th), [W.depolarizing_kraus(0.1), W.amplitude_damping_kraus(0.2)])
    # a shared angle: parameter 3 also drives gate 0's rotation
    circ.gates[0].param_index = 3
    terms = [(0.3, 0b00011), (-0.7, 0b10100), (0.25, 0b00001)]
    rows, _ = P.presample(circ, 6, 40 + seed)
    mult = np.arange(1, 7)
    v_adj, g_adj = G.expval_grad_adjoint(circ, rows, mult, terms, th)
    g_sh = G.expval_grad_shift(circ, rows, mult, terms, th)
    assert abs(v_adj - G.expval(circ, rows, mult, terms, th)) < 1e-12
    np.testing.assert_allclose(g_adj, g_sh, rtol=0, atol=1e-11)
    vd, gd = G.density_grad_adjoint(circ, terms, th)
    assert abs(vd - G.density_expval(circ, terms, th)) < 1e-12
    np.testing.assert_allclose(gd, G.density_grad_shift(circ, terms, th), rtol=0, atol=1e-11)


def test_mps_window_marginal_brute_force():
    """Marginal of a window of qubits with every other qubit traced equals the
    brute-force sum of |psi|^2 over the other qubits' outcomes."""
    rng = np.random.default_rng(31)
    circ = W.attach_noise(W.brickwork_1d(8, 6, rng), [W.depolarizing_kraus(0.1), W.amplitude_damping_kraus(0.2)])
    kraus, _ = pts.presample(circ, 3, 9)
    for t in range(3):
        probs = np.abs(sv.trajectory_state(circ, kraus[t])) ** 2
        m = mps.trajectory_mps(circ, kraus[t])
        idx = np.arange(256)
        for start, b in [(0, 3), (2, 4), (5, 3), (0, 8), (7, 1)]:
            key = (idx >> start) & ((1 << b) - 1)
            want = np.bincount(key, weights=probs, minlength=1 << b)
            np.testing.assert_allclose(m.window_marginal(start, b), want, rtol=1e-10, atol=1e-14)


# ------------------------------------------------ non-proportional NBS ----

def test_quantise64_exact_and_close_to_the_row():
    rng = np.random.default_rng(61)
    for n_bins in (1, 2, 7, 1024, 1 << 16):
        p = rng.exponential(size=n_bins) * np.exp(rng.uniform(-30, 0))
        p[rng.random(n_bins) < 0.1] = 0.0
        if not np.any(p > 0):
            p[0] = 1.0
        P, C = sampling.quantise64(p)
        tot = sum(int(v) for v in P)
        assert int(C[-1]) == tot < 2 ** 62 and int(P.max()) >= 2 ** 60 >> max(0, math.ceil(math.log2(n_bins)))
        bits = math.ceil(math.log2(n_bins)) if n_bins > 1 else 0
        err = np.abs(P.astype(np.float64) / tot - p / p.sum())
        assert err.max() <= 2.0 ** (bits - 59) * (p.max() / p.sum()) + 1e-300


def test_inverse_cdf64_brute_force():
    rng = np.random.default_rng(62)
    for _ in range(20):
        p = rng.random(rng.integers(1, 40))
        p[rng.random(len(p)) < 0.3] = 0.0
        if not np.any(p > 0):
            p[-1] = 0.5
        P, C = sampling.quantise64(p)
        T = int(C[-1])
        a = rng.integers(0, 2 ** 63, size=200, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=200,
                                                                                              dtype=np.uint64)
        got = sampling.inverse_cdf64(C, a)
        for ai, x in zip(a.tolist(), got.tolist()):
            r = (int(ai) * T) >> 64
            want = next(k for k in range(len(C)) if r < int(C[k]))
            assert x == want and P[x] > 0


def test_harvest_exhaustive_threshold_and_probabilities():
    p = np.array([0.5, 0.0, 0.25, 0.125, 0.0625, 0.0625, 0.0, 0.0])
    t, b, pr = sampling.harvest_exhaustive(p[None, :] * 3.0, np.array([4]), np.array([5], np.uint64), 3, 0.0)
    assert t.tolist() == [4] * 5 and b.tolist() == [5 | (x << 3) for x in (0, 2, 3, 4, 5)]
    np.testing.assert_allclose(pr, [0.5, 0.25, 0.125, 0.0625, 0.0625], rtol=1e-15)
    t, b, pr = sampling.harvest_exhaustive(p[None, :], np.array([0]), np.array([0], np.uint64), 0, 0.1)
    assert b.tolist() == [0, 2, 3]
    onehot = np.zeros((1, 64))
    onehot[0, 37] = 1e-20
    t, b, pr = sampling.harvest_exhaustive(onehot, np.array([1]), np.array([0], np.uint64), 6, 0.5)
    assert b.tolist() == [37 << 6] and pr.tolist() == [1.0]
    # zero-norm network: no records
    t, b, pr = sampling.harvest_exhaustive(np.zeros((1, 8)), np.array([0]), np.array([0], np.uint64), 0, 0.0)
    assert len(t) == 0


def test_harvest_direct_law_and_counts():
    p = np.array([0.1, 0.4, 0.0, 0.2, 0.3])
    rows = np.stack([p, p[::-1]])
    t, b, c = sampling.harvest_direct(rows, np.array([0, 0]), np.array([1, 0], np.uint64), 1, 200_000, 5, 2)
    assert c.sum() == 400_000 and np.all(np.diff(t) >= 0)
    for n, row in enumerate(rows):
        sel = (b & np.uint64(1)) == np.uint64(1 - n)
        freq = np.zeros(5)
        freq[(b[sel] >> np.uint64(1)).astype(np.int64)] = c[sel]
        freq /= freq.sum()
        assert np.abs(freq - row).max() < 0.005
        assert freq[np.nonzero(row == 0)[0]].sum() == 0


def test_nbs_nonproportional_branching_and_final_law():
    """One shot per non-final block: every trajectory keeps exactly one prefix
    per block, and the first block's outcomes follow its marginal; the
    exhaustive final harvest of each network equals the exact conditional
    distribution of the final block given that prefix."""
    rng = np.random.default_rng(63)
    circ = W.brickwork_1d(6, 4, rng)           # noiseless: every trajectory is the same state
    psi = sv.pure_state(circ)
    probs = np.abs(psi) ** 2
    blocks = [(0, 2), (2, 2), (4, 2)]

    def marg(j, traj, prefix):
        start, b = blocks[j]
        return np.stack([sv.block_marginals(probs, 6, start, b)[int(s) & ((1 << start) - 1)] for s in prefix])

    E = 4000
    (t, bits, pr), nets = sampling.nbs_nonproportional(marg, blocks, 77, E, branch=1, mode="exhaustive", tau=0.0)
    assert nets == [E, E, E]
    assert sorted(set(t.tolist())) == list(range(E))
    first = (bits[np.r_[0, np.nonzero(np.diff(t))[0] + 1]] & np.uint64(3)).astype(np.int64)
    freq = np.bincount(first, minlength=4) / E
    assert np.abs(freq - sv.block_marginals(probs, 6, 0, 2)[0] / probs.sum()).max() < 0.03
    for i in (0, 17, 3999):
        sel = t == i
        pre = int(bits[sel][0]) & 15
        cond = sv.block_marginals(probs, 6, 4, 2)[pre]
        cond = cond / cond.sum()
        got = np.zeros(4)
        got[(bits[sel] >> np.uint64(4)).astype(np.int64)] = pr[sel]
        np.testing.assert_allclose(got, cond, rtol=1e-12, atol=1e-15)
    # branch > 1 grows the prefix set; direct mode returns counts
    (t2, b2, c2), nets2 = sampling.nbs_nonproportional(marg, blocks, 78, 10, branch=3, mode="direct", final_shots=50)
    assert nets2[0] == 10 and nets2[1] >= 10 and nets2[2] >= nets2[1] and c2.sum() == 50 * nets2[2]


# ------------------------------------------- the paper's circuit family ----

def test_two_qubit_depolarizing_closed_form():
    """Completeness, nominal probabilities (1 - p, p/15 x 15) and the channel's
    action on a random two-qubit state: (1 - p) rho + p/15 sum_{PQ != II}."""
    p = 0.13
    ch = W.depolarizing2_kraus(p)
    assert pts.completeness_error(ch.kraus) < 1e-14
    q = pts.kraus_probs(ch.kraus)
    np.testing.assert_allclose(q, [1 - p] + [p / 15] * 15, rtol=1e-14)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    rho = a @ a.conj().T
    rho /= np.trace(rho)
    out = sum(k @ rho @ k.conj().T for k in ch.kraus)
    # the fully depolarizing part of a unit-trace state is I / 4: (1 - 16 p / 15) rho + 16 p / 15 * I / 4
    want = (1 - 16 * p / 15) * rho + (16 * p / 15) * np.eye(4) / 4
    np.testing.assert_allclose(out, want, atol=1e-14)


def test_paper_family_trajectories_match_density_matrix():
    """A 4-qubit member of the paper's random family (Pauli and two-qubit
    depolarizing noise): the exact average over every Kraus assignment,
    weighted by the nominal probabilities, of the merged-gate trajectory
    states equals the density matrix of the channel evolution."""
    import itertools
    rng = np.random.default_rng(17)
    circ = W.paper_random_circuit(4, 40, rng, frac_2q=0.5)
    # a short prefix of the draw with two two-qubit and three one-qubit gates
    keep = [l for l, g in enumerate(circ.gates) if g.arity == 2][:2] + \
           [l for l, g in enumerate(circ.gates) if g.arity == 1][:3]
    keep.sort()
    gates = [circ.gates[l] for l in keep]
    sites = [W.Site(i, s.qubit, s.channel) for i, l in enumerate(keep) for s in circ.sites if s.gate == l]
    circ = W.Circuit(4, gates, circ.channels, sites)
    assert sum(s.qubit < 0 for s in circ.sites) == 2 and sum(s.qubit >= 0 for s in circ.sites) == 3
    rho = densmat.density_matrix(circ)
    qs = [pts.kraus_probs(circ.channels[s.channel].kraus) for s in circ.sites]
    acc = np.zeros((16, 16), dtype=np.complex128)
    for choice in itertools.product(*[range(len(q)) for q in qs]):
        w = np.prod([q[k] for q, k in zip(qs, choice)])
        if w == 0:
            continue
        psi = sv.trajectory_state(circ, np.array(choice))
        acc += w * np.outer(psi, psi.conj())
    np.testing.assert_allclose(acc, rho, atol=1e-12)


def test_merged_two_qubit_pauli_product():
    """The merge of a two-qubit depolarizing Kraus choice 4a + b into its gate is
    (P_a (x) P_b) G on the gate's (first, second) qubits."""
    g = W.Gate((3, 2), np.kron(W.haar_u2(np.random.default_rng(1)), W.haar_u2(np.random.default_rng(2))) @ W.CZ)
    ch = W.depolarizing2_kraus(0.2)
    circ = W.Circuit(4, [g], [ch], [W.Site(0, -1, 0)])
    P = [W.PAULI[c] for c in "IXYZ"]
    for k in (0, 6, 15):
        # K_k / sqrt(q_k) is the bare Pauli product (K_k = sqrt(q_k) P (x) Q)
        m = pts.merged_gate(circ, 0, np.array([k]))
        np.testing.assert_allclose(m, np.kron(P[k // 4], P[k % 4]) @ g.matrix, atol=1e-13)


def test_wide_bitstrings_shift_block_outcomes():
    """Bitstrings past bit 63 (circuits of more than 64 qubits) are Python
    integers.  With marginals that do not depend on the prefix, moving blocks
    2 and 3 from bits 4 and 8 to bits 64 and 130 moves their outcomes there
    and changes nothing else: the draws depend on trajectory, shot rank and
    block index only, and the canonical order is by block outcomes."""
    from oracle import sampling
    rng = np.random.default_rng(5)
    rows = [rng.random((1, 16)) + 0.05 for _ in range(3)]

    def mf(j, traj, prefix):
        return np.repeat(rows[j], len(traj), axis=0)

    narrow, wide = [(0, 4), (4, 4), (8, 4)], [(0, 4), (64, 4), (130, 4)]

    def widen(bits):
        b = int(bits)
        return (b & 15) | (((b >> 4) & 15) << 64) | (((b >> 8) & 15) << 130)

    tn, bn, cn, ln, _ = sampling.nbs_proportional(mf, narrow, 77, 6, shots=[40, 0, 13, 7, 25, 3])
    tw, bw, cw, lw, _ = sampling.nbs_proportional(mf, wide, 77, 6, shots=[40, 0, 13, 7, 25, 3])
    assert bw.dtype == object and any(int(x) >> 64 for x in bw)
    assert np.array_equal(tn, tw) and np.array_equal(cn, cw) and ln == lw
    assert [widen(x) for x in bn] == [int(x) for x in bw]
    for mode, kw in (("exhaustive", dict(tau=0.02)), ("direct", dict(final_shots=50))):
        (rt, rb, rv), nn = sampling.nbs_nonproportional(mf, narrow, 9, 5, branch=2, mode=mode, **kw)
        (wt, wb, wv), nw = sampling.nbs_nonproportional(mf, wide, 9, 5, branch=2, mode=mode, **kw)
        assert nn == nw and np.array_equal(rt, wt) and np.array_equal(rv, wv)
        assert [widen(x) for x in rb] == [int(x) for x in wb]
