"""Exact density-matrix evolution in complex128 (small n only).
TEST INFRASTRUCTURE (see the package docstring).

Paper, Sec. I / II-A: a noisy n-qubit system is described exactly by a
2^n x 2^n density matrix; each gate acts as rho -> G rho G^dagger and each noise
channel as rho -> sum_k K_k rho K_k^dagger.  Trajectory averages must converge
to this matrix.  Bit q of an index is qubit q.
"""
import numpy as np

from .statevector import apply_gate


def _apply_left(rho, n, qubits, m):
    """M acting on the row index of rho, i.e. on every column of rho.  The
    flattened matrix rho[r, c] -> r * 2^n + c is a 2n-qubit vector whose
    qubit q + n is the row's qubit q, so this is one gate application on it
    (the same sums as applying M to each column in turn)."""
    d = 1 << n
    return apply_gate(rho.reshape(-1), 2 * n, [q + n for q in qubits], m).reshape(d, d)


def apply_unitary(rho, n, qubits, m):
    """rho -> M rho M^dagger."""
    x = _apply_left(rho, n, qubits, m)
    return _apply_left(x.conj().T, n, qubits, m).conj().T


def apply_channel(rho, n, q, kraus):
    return sum(apply_unitary(rho, n, (q,), k) for k in kraus)


def density_matrix(circ):
    n = circ.n_qubits
    d = 1 << n
    rho = np.zeros((d, d), dtype=np.complex128)
    rho[0, 0] = 1.0
    sites_of = [[] for _ in circ.gates]
    for s in circ.sites:
        sites_of[s.gate].append(s)
    for l, g in enumerate(circ.gates):
        rho = apply_unitary(rho, n, g.qubits, g.matrix)
        for s in sites_of[l]:
            kr = circ.channels[s.channel].kraus
            if s.qubit < 0:    # two-qubit channel on the gate's qubits
                rho = sum(apply_unitary(rho, n, g.qubits, k) for k in kr)
            else:
                rho = apply_channel(rho, n, s.qubit, kr)
    return rho


def pauli_string_expectation(rho, n, paulis):
    """Tr(rho P) for P a product of Z on the listed qubits."""
    idx = np.arange(1 << n)
    sign = np.ones(1 << n)
    for q in paulis:
        sign = sign * (1 - 2 * ((idx >> q) & 1))
    return float(np.real(np.sum(np.diag(rho) * sign)))
