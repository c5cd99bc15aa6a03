"""GPU tests of ptn_expval_grad (trajectory-averaged Pauli expectations and
their adjoint gradients) against the oracle's parameter-shift gradient, and at
the 16-qubit / 6-layer / 1024-trajectory ansatz size against central finite
differences of the GPU values.

Tolerance: the contraction runs in complex64 with FP64 reductions, so each
amplitude carries a relative error of order 1e-6; an expectation value and
every gradient entry are sums of such products weighted by the observable, so
both are compared with an absolute bound 1e-4 * S, S = sum_t |a_t| times the
mean squared trajectory norm (the largest value |F| can take)."""
import numpy as np
import pytest

import workloads as W
from oracle import gradient as G, pts, statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_08467_gb300 import ptn  # noqa: E402

DEV = "cuda"


def _gpu(plan, tr, terms, theta):
    v = torch.empty(1, dtype=torch.float64, device=DEV)
    g = torch.empty(max(len(theta), 1), dtype=torch.float64, device=DEV)
    ptn.ptn_expval_grad(plan, tr, terms, np.asarray(theta, np.float64), v, g)
    torch.cuda.synchronize()
    return float(v.item()), g.cpu().numpy()[: len(theta)]


def _traj_rows(tr):
    kr, _, mu, _ = [x.cpu().numpy() for x in tr.to_torch()]
    return kr, mu


def _scale(circ, rows, mult, terms):
    nrm = np.array([np.sum(np.abs(sv.trajectory_state(circ, r)) ** 2) for r in rows])
    return sum(abs(a) for a, _ in terms) * float(np.sum(mult * nrm) / np.sum(mult))


def _shared(r):
    th = r.standard_normal(3)
    g = [W.Gate((0,), W.RY(th[0]), W.PARAM_RY, 0), W.Gate((1,), W.RY(th[0]), W.PARAM_RY, 0),
         W.Gate((0, 1), W.CZ.copy()), W.Gate((2,), W.haar_u2(r)), W.Gate((1, 2), W.CZ.copy()),
         W.Gate((2,), W.RZ(th[1]), W.PARAM_RZ, 1), W.Gate((1,), W.RY(th[2]), W.PARAM_RY, 2),
         W.Gate((0,), W.RY(th[0]), W.PARAM_RY, 0), W.Gate((0, 2), W.CZ.copy()),
         W.Gate((3,), W.haar_u2(r)), W.Gate((2, 3), W.CZ.copy()), W.Gate((3,), W.RY(th[1]), W.PARAM_RY, 1)]
    return W.Circuit(4, g), th


def _hea(n, layers, noise, seed):
    r = np.random.default_rng(seed)
    th = r.standard_normal(n * layers * 2)
    c = W.hea_ring(n, layers, th)
    if noise:
        W.attach_noise(c, noise)
    return c, th


CASES = [
    ("hea6_dep", lambda: _hea(6, 3, [W.depolarizing_kraus(0.05)], 1), [3, 3], 48),
    ("hea5_dep_ad", lambda: _hea(5, 2, [W.depolarizing_kraus(0.1), W.amplitude_damping_kraus(0.2)], 2), [5], 32),
    ("hea4_noiseless", lambda: _hea(4, 3, None, 3), [4], 4),
    ("shared4", lambda: (lambda c_th: (W.attach_noise(c_th[0], [W.depolarizing_kraus(0.2)]), c_th[1]))(
        _shared(np.random.default_rng(4))), [4], 40),
    ("hea10_dep", lambda: _hea(10, 2, [W.depolarizing_kraus(0.02)], 5), [10], 16),
]


@pytest.mark.parametrize("name,make,bs,n_traj", CASES, ids=[c[0] for c in CASES])
def test_expval_grad_matches_oracle(name, make, bs, n_traj):
    circ, th = make()
    n = circ.n_qubits
    terms = [(1.0 / n, (1 << q) | (1 << ((q + 1) % n))) for q in range(n)] + [(0.3, 1), (-0.2, 0)]
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=16, est_traj=n_traj)
    tr = ptn.ptn_presample_trajectories(plan, 99, n_traj, dedup=True)
    rows, mult = _traj_rows(tr)
    # a fresh angle vector (not the one the circuit was built with)
    theta = np.random.default_rng(7).standard_normal(circ.n_params())
    v, g = _gpu(plan, tr, terms, theta)
    f_ref = G.expval(circ, rows, mult, terms, theta)
    g_ref = G.expval_grad_shift(circ, rows, mult, terms, theta)
    S = _scale(G.at_angles(circ, theta), rows, mult, terms)
    assert abs(v - f_ref) <= 1e-4 * S, (v, f_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * S, np.max(np.abs(g - g_ref))
    # a second call at other angles reuses the uploaded plan
    theta2 = theta + 0.3
    v2, g2 = _gpu(plan, tr, terms, theta2)
    assert abs(v2 - G.expval(circ, rows, mult, terms, theta2)) <= 1e-4 * S
    assert np.max(np.abs(g2 - G.expval_grad_shift(circ, rows, mult, terms, theta2))) <= 1e-4 * S


def test_expval_sets_plan_angles_for_sampling():
    """After ptn_expval_grad the plan's rotations hold the new angles, so the
    marginals of ptn_contract_batch follow them."""
    circ, _ = _hea(6, 2, [W.depolarizing_kraus(0.05)], 8)
    plan = ptn.ptn_plan_path(circ, [6], hypersamples=8, est_traj=8)
    tr = ptn.ptn_presample_trajectories(plan, 5, 8, dedup=False)
    rows, _ = _traj_rows(tr)
    theta = np.linspace(-1, 1, circ.n_params())
    _gpu(plan, tr, [(1.0, 1)], theta)
    nt = torch.arange(8, dtype=torch.int32, device=DEV)
    npre = torch.zeros(8, dtype=torch.int64, device=DEV)
    marg = torch.empty((8, 64), dtype=torch.float32, device=DEV)
    Z = torch.empty(8, dtype=torch.float64, device=DEV)
    ptn.ptn_contract_batch(plan, tr, 0, nt, npre, marg, Z)
    torch.cuda.synchronize()
    c2 = G.at_angles(circ, theta)
    want = np.array([np.abs(sv.trajectory_state(c2, r)) ** 2 for r in rows])
    got = marg.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= 2e-5 * np.max(want)


def test_expval_rejects_bad_arguments():
    circ, th = _hea(4, 1, [W.depolarizing_kraus(0.05)], 9)
    plan = ptn.ptn_plan_path(circ, [4], hypersamples=4, est_traj=4)
    tr = ptn.ptn_presample_trajectories(plan, 5, 4)
    v = torch.empty(1, dtype=torch.float64, device=DEV)
    g = torch.empty(8, dtype=torch.float64, device=DEV)
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_expval_grad(plan, tr, [(1.0, 1, 1)], th, v, g)       # X component
    assert e.value.status == 7
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_expval_grad(plan, tr, [(1.0, 1)], th[:3], v, g)      # too few angles
    assert e.value.status == 1


def test_autograd_function():
    from paper_2604_08467_gb300.autograd import trajectory_expval
    circ, _ = _hea(5, 2, [W.depolarizing_kraus(0.05)], 10)
    plan = ptn.ptn_plan_path(circ, [5], hypersamples=8, est_traj=16)
    tr = ptn.ptn_presample_trajectories(plan, 3, 16, dedup=True)
    rows, mult = _traj_rows(tr)
    terms = [(0.5, 0b00011), (0.5, 0b11000)]
    theta = torch.tensor(np.random.default_rng(1).standard_normal(circ.n_params()), requires_grad=True)
    f = trajectory_expval(theta, plan, tr, terms)
    (3.0 * f).backward()
    th = theta.detach().numpy()
    S = _scale(G.at_angles(circ, th), rows, mult, terms)
    assert abs(f.item() - G.expval(circ, rows, mult, terms, th)) <= 1e-4 * S
    np.testing.assert_allclose(theta.grad.numpy(), 3.0 * G.expval_grad_shift(circ, rows, mult, terms, th),
                               atol=3e-4 * S)


def _c5_terms(n=16):
    return [(1.0 / n, (1 << q) | (1 << ((q + 1) % n))) for q in range(n)]


@pytest.mark.parametrize("ckpt", [False, True], ids=["keep_all", "checkpointed"])
def test_c5_all_components_against_oracle(ckpt):
    """16-qubit, 6-layer ansatz (192 angles): the value and every gradient
    entry against the oracle's FP64 reverse-mode state-vector gradient (pinned
    to the parameter-shift rule) on a small trajectory set, for the keep-all
    and the checkpointed gradient plans."""
    cfg = W.config_c5()
    circ, th = cfg["circuit"], cfg["thetas"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=cfg["n_traj"], grad_checkpoint=ckpt)
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], 4, dedup=True)
    rows, mult = _traj_rows(tr)
    terms = _c5_terms()
    v, g = _gpu(plan, tr, terms, th)
    v_ref, g_ref = G.expval_grad_adjoint(circ, rows, mult, terms, th)
    S = _scale(G.at_angles(circ, th), rows, mult, terms)
    assert abs(v - v_ref) <= 1e-4 * S
    assert g.shape == g_ref.shape == (192,)
    err = np.abs(g - g_ref)
    assert np.max(err) <= 1e-4 * S, (int(np.argmax(err)), float(np.max(err)), S)


def test_c5_family_10q_against_density_matrix_gradient():
    """A 10-qubit member of the ansatz family (6 layers of RY RZ + CZ ring,
    120 angles ~ N(0, 1), depolarizing 0.01 after every gate): the mean over
    32 independent sets of 256 trajectories of the GPU value and gradient
    against Tr(O rho) and its exact FP64 density-matrix gradient (reverse mode,
    pinned to parameter shift).  Per component the deviation must stay within
    5 standard errors of the set means (t with 31 degrees of freedom: about
    2e-5 per component, so 120 components pass together unless biased)."""
    n = 10
    r = np.random.default_rng(510)
    th = r.standard_normal(n * 6 * 2)
    circ = W.attach_noise(W.hea_ring(n, 6, th), [W.depolarizing_kraus(0.01)])
    terms = [(1.0 / n, (1 << q) | (1 << ((q + 1) % n))) for q in range(n)]
    plan = ptn.ptn_plan_path(circ, [n], hypersamples=8, est_traj=256, grad_checkpoint=True)
    vs, gs = [], []
    for k in range(32):
        tr = ptn.ptn_presample_trajectories(plan, 7000 + k, 256, dedup=True)
        v, g = _gpu(plan, tr, terms, th)
        vs.append(v)
        gs.append(g)
    vs, gs = np.array(vs), np.array(gs)
    se_v = vs.std(ddof=1) / np.sqrt(len(vs))
    se_g = gs.std(axis=0, ddof=1) / np.sqrt(len(gs))
    f_dm, g_dm = G.density_grad_adjoint(circ, terms, th)
    assert abs(vs.mean() - f_dm) <= 5 * se_v + 1e-6, (vs.mean(), f_dm, se_v)
    dev = np.abs(gs.mean(axis=0) - g_dm)
    assert np.all(dev <= 5 * se_g + 1e-6), float((dev / np.maximum(se_g, 1e-12)).max())


def test_c5_full_against_finite_differences():
    """1024 trajectories: the adjoint gradient against central differences
    (h = 1e-3) of the GPU's own values.  The FD error is the value's rounding
    error over 2h (complex64 states: ~1e-7 * S / 2e-3) plus O(h^2) truncation."""
    cfg = W.config_c5()
    circ, th = cfg["circuit"], cfg["thetas"]
    plan = ptn.ptn_plan_path(circ, cfg["block_sizes"], hypersamples=16, est_traj=cfg["n_traj"])
    tr = ptn.ptn_presample_trajectories(plan, cfg["seed"], cfg["n_traj"], dedup=True)
    terms = _c5_terms()
    v, g = _gpu(plan, tr, terms, th)
    assert np.all(np.isfinite(g)) and abs(v) <= 1.0 + 1e-6
    h = 1e-3
    rng = np.random.default_rng(0)
    for p in rng.choice(len(th), 6, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (_gpu(plan, tr, terms, tp)[0] - _gpu(plan, tr, terms, tm)[0]) / (2 * h)
        assert abs(fd - g[p]) <= 2e-3 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_gradient_converges_to_density_matrix():
    """Trajectory averages are unbiased for the exact noisy state: over 32
    independent trajectory sets the mean GPU value and gradient agree with
    Tr(O rho) and its FP64 density-matrix parameter-shift gradient within 5
    standard errors per component (seeds fixed, so the outcome is
    deterministic)."""
    circ, th = _hea(5, 2, [W.depolarizing_kraus(0.03), W.amplitude_damping_kraus(0.05)], 12)
    terms = [(0.2, (1 << q) | (1 << ((q + 1) % 5))) for q in range(5)]
    plan = ptn.ptn_plan_path(circ, [5], hypersamples=8, est_traj=256)
    vs, gs = [], []
    for k in range(32):
        tr = ptn.ptn_presample_trajectories(plan, 1000 + k, 256, dedup=True)
        v, g = _gpu(plan, tr, terms, th)
        vs.append(v)
        gs.append(g)
    vs, gs = np.array(vs), np.array(gs)
    se_v = vs.std(ddof=1) / np.sqrt(len(vs))
    se_g = gs.std(axis=0, ddof=1) / np.sqrt(len(gs))
    f_dm = G.density_expval(circ, terms, th)
    g_dm = G.density_grad_shift(circ, terms, th)
    assert abs(vs.mean() - f_dm) <= 5 * se_v + 1e-6, (vs.mean(), f_dm, se_v)
    dev = np.abs(gs.mean(axis=0) - g_dm)
    assert np.all(dev <= 5 * se_g + 1e-6), (dev / np.maximum(se_g, 1e-12)).max()


def test_checkpointed_gradients_match_keep_all():
    """Gradient plans that recompute forward intermediates segment by segment
    (grad_checkpoint) run the same kernels on the same inputs: values and
    gradients equal those of the keep-all plan, with a smaller trajectory arena."""
    r = np.random.default_rng(21)
    th = r.standard_normal(12 * 8 * 2)
    circ = W.attach_noise(W.hea_ring(12, 8, th), [W.depolarizing_kraus(0.02), W.amplitude_damping_kraus(0.02)])
    terms = [(1.0 / 12, (1 << q) | (1 << ((q + 1) % 12))) for q in range(12)]
    res = []
    for ck in (False, True):
        plan = ptn.ptn_plan_path(circ, [6, 6], hypersamples=16, est_traj=64, grad_checkpoint=ck)
        tr = ptn.ptn_presample_trajectories(plan, 5, 64, dedup=True)
        res.append(_gpu(plan, tr, terms, th) + (plan.describe(detail=2)["expval"]["arena"][1],))
    (v0, g0, a0), (v1, g1, a1) = res
    assert a1 < a0
    assert abs(v1 - v0) <= 1e-12 * max(1.0, abs(v0))
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-12)
