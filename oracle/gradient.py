"""Trajectory-averaged Pauli expectation values and their angle gradients.
TEST INFRASTRUCTURE (see the package docstring).

What is computed (the differentiation form of the hot path; the paper's
trajectories, Sec. II-B / II-C, with the UPV merge of Sec. III-A):

    F(theta) = sum_i c_i <psi_i(theta)| O |psi_i(theta)> / sum_i c_i

psi_i the unnormalised state of error set i (each sampled Kraus operator,
scaled by 1 / sqrt(q_k), merged into its gate), c_i its multiplicity and
O = sum_t a_t prod_{q in z_t} Z_q a diagonal Pauli sum.  Parametrised gates are
rotations R_P(t) = exp(-i t P / 2), P = Y or Z.

The gradient is taken by the parameter-shift rule: each occurrence of a
rotation contributes [F(t + pi/2) - F(t - pi/2)] / 2 with only that occurrence
shifted, because F is a trigonometric polynomial of degree one in its angle
(the state is linear in R_P(t) = cos(t/2) I - i sin(t/2) P and F quadratic in
the state).  This holds for unnormalised trajectory states and for the density
matrix alike.  Central finite differences are provided as an independent
second method, and reverse-mode (adjoint) forms on the state vector and on
the density matrix as a third: with the gate sequence E_L ... E_1, the
derivative of <O> with respect to the angle of gate l is the overlap of the
backward-propagated observable (adjoint state, or Heisenberg-evolved O for
the density matrix) after gate l with the derivative of gate l applied to the
forward state before it; d R_P(t) / dt = R_P(t) (-i P / 2).
"""
import copy

import numpy as np

from .densmat import _apply_left, apply_channel, apply_unitary
from .pts import gate_sites, merged_gate
from .statevector import apply_gate

PARAM_RY, PARAM_RZ = 1, 2
_PAULI = {PARAM_RY: np.array([[0, -1j], [1j, 0]]), PARAM_RZ: np.diag([1.0 + 0j, -1.0])}


def rotation(kind, angle):
    """exp(-i angle P / 2) = cos(angle/2) I - i sin(angle/2) P."""
    return np.cos(angle / 2) * np.eye(2) - 1j * np.sin(angle / 2) * _PAULI[kind]


def pauli_weights(n, terms):
    """w(x) = sum_t a_t (-1)^popcount(x & z_t): the diagonal of O."""
    x = np.arange(1 << n, dtype=np.int64)
    w = np.zeros(1 << n)
    for a, z in terms:
        par = np.zeros(1 << n, dtype=np.int64)
        for q in range(n):
            if (int(z) >> q) & 1:
                par ^= (x >> q) & 1
        w += a * (1 - 2 * par)
    return w


def at_angles(circ, theta, shift=None):
    """Copy of circ with every rotation set to theta[param_index]; shift =
    (gate index, delta) adds delta to one occurrence only."""
    c = copy.copy(circ)
    c.gates = []
    for l, g in enumerate(circ.gates):
        if g.param_kind in (PARAM_RY, PARAM_RZ):
            t = float(theta[g.param_index])
            if shift is not None and shift[0] == l:
                t += shift[1]
            g = copy.copy(g)
            g.matrix = rotation(g.param_kind, t)
        c.gates.append(g)
    return c


def trajectory_expval(circ, choices, w):
    """<psi_i| O |psi_i> for the unnormalised trajectory state."""
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    sg = gate_sites(circ)
    for l, g in enumerate(circ.gates):
        psi = apply_gate(psi, n, g.qubits, merged_gate(circ, l, choices, sg))
    return float(np.sum(w * np.abs(psi) ** 2))


def circuit_expval(c, kraus_rows, mult, w):
    """F for a circuit whose rotations are already set."""
    mult = np.asarray(mult, dtype=np.float64)
    f = np.array([trajectory_expval(c, row, w) for row in kraus_rows])
    return float(np.sum(mult * f) / np.sum(mult))


def expval(circ, kraus_rows, mult, terms, theta):
    """F(theta) over the error sets kraus_rows with multiplicities mult."""
    return circuit_expval(at_angles(circ, theta), kraus_rows, mult, pauli_weights(circ.n_qubits, terms))


def rotation_occurrences(circ):
    return [l for l, g in enumerate(circ.gates) if g.param_kind in (PARAM_RY, PARAM_RZ)]


def expval_grad_shift(circ, kraus_rows, mult, terms, theta, params=None):
    """dF/dtheta_p by the parameter-shift rule, summed over the occurrences of
    parameter p; params restricts the computed entries (the others are NaN)."""
    w = pauli_weights(circ.n_qubits, terms)
    grad = np.full(len(theta), np.nan)
    want = set(range(len(theta)) if params is None else params)
    for p in want:
        grad[p] = 0.0
    for l in rotation_occurrences(circ):
        p = circ.gates[l].param_index
        if p not in want:
            continue
        fp = circuit_expval(at_angles(circ, theta, (l, np.pi / 2)), kraus_rows, mult, w)
        fm = circuit_expval(at_angles(circ, theta, (l, -np.pi / 2)), kraus_rows, mult, w)
        grad[p] += 0.5 * (fp - fm)
    return grad


def expval_grad_fd(circ, kraus_rows, mult, terms, theta, h=1e-3, params=None):
    """Central finite differences [F(theta + h e_p) - F(theta - h e_p)] / (2h)."""
    theta = np.asarray(theta, dtype=np.float64)
    n_p = theta.size
    grad = np.full(n_p, np.nan)
    for p in (range(n_p) if params is None else params):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        grad[p] = (expval(circ, kraus_rows, mult, terms, tp) - expval(circ, kraus_rows, mult, terms, tm)) / (2 * h)
    return grad


# ------------------------------------------------------ density matrix ----

def density_expval(circ, terms, theta, shift=None):
    """Tr(O rho(theta)): exact noisy evolution, every channel applied in full."""
    c = at_angles(circ, theta, shift)
    n = c.n_qubits
    d = 1 << n
    rho = np.zeros((d, d), dtype=np.complex128)
    rho[0, 0] = 1.0
    sites_of = gate_sites(c)
    for l, g in enumerate(c.gates):
        rho = apply_unitary(rho, n, g.qubits, g.matrix)
        for s in sites_of[l]:
            site = c.sites[s]
            rho = apply_channel(rho, n, site.qubit, c.channels[site.channel].kraus)
    return float(np.real(np.sum(np.diag(rho) * pauli_weights(n, terms))))


def density_grad_shift(circ, terms, theta):
    """Parameter-shift gradient of Tr(O rho(theta)) (FP64 density matrix)."""
    grad = np.zeros(len(theta))
    for l in rotation_occurrences(circ):
        p = circ.gates[l].param_index
        grad[p] += 0.5 * (density_expval(circ, terms, theta, (l, np.pi / 2)) -
                          density_expval(circ, terms, theta, (l, -np.pi / 2)))
    return grad


# ------------------------------------------------------- reverse mode -----

def trajectory_grad_adjoint(circ, choices, w, n_params):
    """(<psi|O|psi>, d<psi|O|psi>/dtheta) for one unnormalised trajectory state
    by the adjoint method: forward states before every rotation are kept, the
    adjoint lambda = O psi is carried back through U_l^dagger, and rotation l
    (merged tensor U_l = N_l R_P(t), N_l its noise operators) contributes
    2 Re <lambda_l| U_l (-i P / 2) |phi_{l-1}>."""
    n = circ.n_qubits
    sg = gate_sites(circ)
    mats = [merged_gate(circ, l, choices, sg) for l in range(len(circ.gates))]
    phi = np.zeros(1 << n, dtype=np.complex128)
    phi[0] = 1.0
    before = {}
    for l, g in enumerate(circ.gates):
        if g.param_kind in (PARAM_RY, PARAM_RZ):
            before[l] = phi
        phi = apply_gate(phi, n, g.qubits, mats[l])
    lam = w * phi
    value = float(np.real(np.vdot(phi, lam)))
    grad = np.zeros(n_params)
    for l in range(len(circ.gates) - 1, -1, -1):
        g = circ.gates[l]
        if l in before:
            dU = mats[l] @ (-0.5j * _PAULI[g.param_kind])
            grad[g.param_index] += 2.0 * np.real(np.vdot(lam, apply_gate(before[l], n, g.qubits, dU)))
        lam = apply_gate(lam, n, g.qubits, mats[l].conj().T)
    return value, grad


def expval_grad_adjoint(circ, kraus_rows, mult, terms, theta):
    """(F, dF/dtheta) over the error sets kraus_rows with multiplicities mult,
    every entry of the gradient, by the adjoint method."""
    c = at_angles(circ, theta)
    w = pauli_weights(c.n_qubits, terms)
    mult = np.asarray(mult, dtype=np.float64)
    vals, grads = [], []
    for row in kraus_rows:
        v, g = trajectory_grad_adjoint(c, row, w, len(theta))
        vals.append(v)
        grads.append(g)
    return (float(np.sum(mult * np.array(vals)) / np.sum(mult)),
            (mult[:, None] * np.array(grads)).sum(axis=0) / np.sum(mult))


def _row_col(rho, n, q_row, q_col, m):
    """Apply the 4x4 matrix m (index order (o_row, o_col, i_row, i_col)) to
    the row qubit q_row and column qubit q_col of rho, seen as the 2n-qubit
    vector rho[r, c] -> r * 2^n + c (row qubit q is vector qubit q + n)."""
    d = 1 << n
    return apply_gate(rho.reshape(-1), 2 * n, [q_row + n, q_col], m).reshape(d, d)


def _unitary_super(U):
    """U rho U^dagger as a 4x4 (o_row, o_col, i_row, i_col) matrix on one qubit."""
    U = np.asarray(U)
    return np.kron(U, U.conj())


def _channel_super(kraus, adjoint=False):
    """sum_k K rho K^dagger (or, adjoint=True, the Heisenberg map
    sum_k K^dagger Lambda K) as a 4x4 matrix on one qubit."""
    S = np.zeros((4, 4), dtype=np.complex128)
    for K in kraus:
        K = np.asarray(K, dtype=np.complex128)
        S += np.kron(K.conj().T, K.T) if adjoint else np.kron(K, K.conj())
    return S


def _apply_unitary_rho(rho, n, qubits, U):
    """U rho U^dagger for a gate on one or two qubits."""
    U = np.asarray(U)
    if len(qubits) == 1:
        return _row_col(rho, n, qubits[0], qubits[0], _unitary_super(U))
    x = _apply_left(rho, n, qubits, U)
    d = 1 << n
    return apply_gate(x.reshape(-1), 2 * n, list(qubits), U.conj()).reshape(d, d)


def density_grad_adjoint(circ, terms, theta):
    """(Tr(O rho), dTr(O rho)/dtheta) for the exact noisy evolution by reverse
    mode on the density matrix: rho before every rotation is kept, Lambda = O
    is evolved back through the adjoint channels and unitaries, and rotation
    l contributes 2 Re Tr(Lambda_l dU rho_{l-1} U^dagger), dU = U (-i P / 2).
    One-qubit gates and channels act as 4x4 superoperators on the (row,
    column) qubit pair, which is the same sum as their Kraus form."""
    c = at_angles(circ, theta)
    n = c.n_qubits
    d = 1 << n
    rho = np.zeros((d, d), dtype=np.complex128)
    rho[0, 0] = 1.0
    sites_of = gate_sites(c)
    chan = [_channel_super(ch.kraus) for ch in c.channels]
    chan_adj = [_channel_super(ch.kraus, adjoint=True) for ch in c.channels]
    before = {}
    for l, g in enumerate(c.gates):
        if g.param_kind in (PARAM_RY, PARAM_RZ):
            before[l] = rho
        rho = _apply_unitary_rho(rho, n, g.qubits, g.matrix)
        for s in sites_of[l]:
            site = c.sites[s]
            rho = _row_col(rho, n, site.qubit, site.qubit, chan[site.channel])
    wdiag = pauli_weights(n, terms)
    value = float(np.real(np.sum(np.diag(rho) * wdiag)))
    lam = np.diag(wdiag).astype(np.complex128)
    grad = np.zeros(len(theta))
    for l in range(len(c.gates) - 1, -1, -1):
        g = c.gates[l]
        for s in reversed(sites_of[l]):
            site = c.sites[s]
            lam = _row_col(lam, n, site.qubit, site.qubit, chan_adj[site.channel])
        if l in before:
            U = np.asarray(g.matrix)
            dU = U @ (-0.5j * _PAULI[g.param_kind])
            # dU rho U^dagger on the gate's (row, column) qubit
            x = _row_col(before[l], n, g.qubits[0], g.qubits[0], np.kron(dU, U.conj()))
            grad[g.param_index] += 2.0 * np.real(np.sum(lam.T * x))
        lam = _apply_unitary_rho(lam, n, g.qubits, np.asarray(g.matrix).conj().T)
    return value, grad
