"""Per-trajectory state vectors and block marginals in complex128.
TEST INFRASTRUCTURE (see the package docstring).

Paper, Sec. II-B: a trajectory is the circuit with every noise channel replaced
by one sampled Kraus operator; its state |psi_i> (unnormalised when the
operators are not unitary) is measured block by block, block B_j's outcome
distribution being conditioned on the outcomes s_1..s_{j-1} already drawn.

The block-j marginal returned here is unnormalised:
p_i(s, x) = sum over the bits after the block of |<s, x, rest|psi_i>|^2,
the quantity whose normalisation (its sum over x) is p_i(s).
Bit q of a basis index is qubit q.
"""
import numpy as np

from .pts import gate_sites, merged_gate


def apply_1q(psi, n, q, m):
    v = psi.reshape(1 << (n - 1 - q), 2, 1 << q)
    return np.einsum("oi,aib->aob", m, v).reshape(-1)


def apply_2q(psi, n, a, b, m):
    """Apply a 4x4 gate with index order (o_a o_b, i_a i_b) to qubits a, b."""
    t = m.reshape(2, 2, 2, 2)   # [o_a, o_b, i_a, i_b]
    shape = [2] * n             # axis k <-> qubit n-1-k
    v = psi.reshape(shape)
    ax_a, ax_b = n - 1 - a, n - 1 - b
    v = np.tensordot(t, v, axes=([2, 3], [ax_a, ax_b]))   # -> [o_a, o_b, rest...]
    rest = [k for k in range(n) if k not in (ax_a, ax_b)]
    # position of each original axis in v
    perm = [0] * n
    perm[ax_a] = 0
    perm[ax_b] = 1
    for j, k in enumerate(rest):
        perm[k] = 2 + j
    return np.transpose(v, perm).reshape(-1)


def apply_gate(psi, n, qubits, m):
    if len(qubits) == 1:
        return apply_1q(psi, n, qubits[0], m)
    return apply_2q(psi, n, qubits[0], qubits[1], m)


def trajectory_state(circ, choices):
    """|psi_i> = prod_l (merged gate l) |0...0>, choices = Kraus row of trajectory i."""
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    sg = gate_sites(circ)
    for l, g in enumerate(circ.gates):
        psi = apply_gate(psi, n, g.qubits, merged_gate(circ, l, choices, sg))
    return psi


def pure_state(circ):
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for g in circ.gates:
        psi = apply_gate(psi, n, g.qubits, g.matrix)
    return psi


def block_marginals(probs, n, start, b):
    """All block marginals at once from the outcome probabilities |psi|^2:
    returns m[prefix, x] = sum_rest probs[prefix + (x << start) + (rest << (start + b))]."""
    t = np.asarray(probs).reshape(1 << (n - start - b), 1 << b, 1 << start)
    return t.sum(axis=0).T.copy()     # [prefix, x]


def block_marginal(psi, n, start, b, prefix):
    probs = np.abs(psi) ** 2
    return block_marginals(probs, n, start, b)[prefix]


def block_layout(n, block_sizes):
    """(start_j, b_j) of each block, qubits in ascending order."""
    starts, s = [], 0
    for b in block_sizes:
        starts.append(s)
        s += b
    assert s == n, "block sizes must cover all qubits"
    return list(zip(starts, block_sizes))


def default_blocks(n, b=10):
    """b_j = b for j < f, b_f = n - b (f - 1), f = ceil(n / b)."""
    f = -(-n // b)
    return [b] * (f - 1) + [n - b * (f - 1)]
