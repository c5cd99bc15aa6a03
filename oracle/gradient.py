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
second method.
"""
import copy

import numpy as np

from .densmat import apply_channel, apply_unitary
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
