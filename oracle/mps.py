"""Exact matrix-product-state evolution for nearest-neighbour 1D circuits.
TEST INFRASTRUCTURE (see the package docstring).

A second, independent way to get trajectory block marginals when a 2^n state
vector is too large (n = 30 and up).  Each merged trajectory gate (the UPV
merge of Sec. III-A, via ``pts.merged_gate``) is applied to the MPS; a
two-qubit gate is absorbed into the two site tensors and split again by an SVD
that keeps every singular value above 1e-14 of the largest, so the result is
exact up to rounding.  Site tensors have shape (chi_left, 2, chi_right).

Block marginals (Sec. II-B): the prefix qubits are projected onto their
outcomes (a left row vector), the qubits after the block are traced (a right
chi x chi environment), and the block's 2^b outcome amplitudes are enumerated
site by site, bit q of x being qubit start+q.
"""
import numpy as np

from .pts import gate_sites, merged_gate


class MPS:
    def __init__(self, n):
        self.n = n
        self.t = [np.zeros((1, 2, 1), dtype=np.complex128) for _ in range(n)]
        for a in self.t:
            a[0, 0, 0] = 1.0

    def apply_1q(self, q, m):
        self.t[q] = np.einsum("oi,lir->lor", m, self.t[q])

    def apply_2q(self, a, b, m):
        g = m.reshape(2, 2, 2, 2)                      # [o_a, o_b, i_a, i_b]
        if b == a - 1:
            a, b = b, a
            g = g.transpose(1, 0, 3, 2)
        if b != a + 1:
            raise ValueError("MPS oracle needs nearest-neighbour gates")
        th = np.einsum("lir,rjs->lijs", self.t[a], self.t[b])
        th = np.einsum("abij,lijs->labs", g, th)
        cl, cs = th.shape[0], th.shape[3]
        u, s, vh = np.linalg.svd(th.reshape(cl * 2, 2 * cs), full_matrices=False)
        keep = max(1, int(np.sum(s > 1e-14 * s[0]))) if s[0] > 0 else 1
        self.t[a] = u[:, :keep].reshape(cl, 2, keep)
        self.t[b] = (s[:keep, None] * vh[:keep]).reshape(keep, 2, cs)

    def max_bond(self):
        return max(a.shape[2] for a in self.t)

    def right_env(self, start):
        """Trace of qubits start..n-1: R[a, a'] (chi x chi)."""
        r = np.ones((1, 1), dtype=np.complex128)
        for q in range(self.n - 1, start - 1, -1):
            a = self.t[q]
            r = sum(a[:, i, :] @ r @ a[:, i, :].conj().T for i in range(2))
        return r

    def block_marginal(self, start, b, prefix, renv=None):
        """p(s, x) for x in [0, 2^b), prefix bits s on qubits < start."""
        v = np.ones((1, 1), dtype=np.complex128)
        for q in range(start):
            v = v @ self.t[q][:, (int(prefix) >> q) & 1, :]
        for q in range(start, start + b):
            a = self.t[q]
            v = np.concatenate([v @ a[:, 0, :], v @ a[:, 1, :]], axis=0)
        r = self.right_env(start + b) if renv is None else renv
        return np.real(np.einsum("xa,ab,xb->x", v, r, v.conj()))


    def left_env(self, stop):
        """Trace of qubits 0..stop-1: L[a, a'] (chi x chi, ket index first)."""
        v = np.ones((1, 1), dtype=np.complex128)
        for q in range(stop):
            a = self.t[q]
            v = sum(a[:, i, :].T @ v @ a[:, i, :].conj() for i in range(2))
        return v

    def window_marginal(self, start, b):
        """p(x) for the b qubits start..start+b-1 with every other qubit
        traced (bit q of x = qubit start+q): sum over a, a', c, c' of
        L[a, a'] P_x[a, c] R[c, c'] conj(P_x[a', c']), P_x the product of the
        window's site matrices for outcome x."""
        L = self.left_env(start)
        R = self.right_env(start + b)
        out = np.empty(1 << b)
        for x in range(1 << b):
            P = np.eye(self.t[start].shape[0], dtype=np.complex128)
            for k in range(b):
                P = P @ self.t[start + k][:, (x >> k) & 1, :]
            out[x] = np.real(np.einsum("ac,ab,bd,cd->", L, P, R, P.conj()))
        return out


def trajectory_mps(circ, choices):
    m = MPS(circ.n_qubits)
    sg = gate_sites(circ)
    for l, g in enumerate(circ.gates):
        u = merged_gate(circ, l, choices, sg)
        if g.arity == 1:
            m.apply_1q(g.qubits[0], u)
        else:
            m.apply_2q(g.qubits[0], g.qubits[1], u)
    return m
