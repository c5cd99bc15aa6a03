"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module only *generates inputs*: circuit structures, Haar-random gate
matrices, Kraus operator sets of the noise models, probability vectors for the
sampling tests.  It holds none of the method's arithmetic (no pre-sampling,
no tensor merging, no contraction, no sampling), so the oracle and the CUDA
path can both consume its output without sharing any computation.

Conventions (used by both sides):

* qubit ``q`` is bit ``q`` of a basis-state index (little-endian);
* a 1-qubit matrix is ``M[out, in]``;
* a 2-qubit gate on ``(a, b) = qubits`` is the 4x4 matrix
  ``M[(o_a << 1) | o_b, (i_a << 1) | i_b]`` (``a`` is the high bit);
* noise sites are listed in application order: after gate ``l``, the channels
  of its first qubit, then those of its second qubit, each list in the order
  the channels act.

The random-circuit families follow the workloads of the paper's Sec. IV-B
(random gates with noise channels coupled to every coherent gate) with the
gate sets and noise models of the benchmark configurations below.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Gate", "Channel", "Site", "Circuit",
    "haar_u2", "depolarizing_kraus", "amplitude_damping_kraus",
    "brickwork_1d", "grid_4colour", "hea_ring", "attach_noise",
    "config_c1", "config_c2", "config_c3", "config_c4", "config_c4_slice",
    "config_c5", "synthetic_marginals", "circuit_seed", "philox_seed",
    "RY", "RZ", "CZ",
]

CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)

PARAM_NONE, PARAM_RY, PARAM_RZ = 0, 1, 2


def RY(theta: float) -> np.ndarray:
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def RZ(phi: float) -> np.ndarray:
    return np.array([[np.exp(-0.5j * phi), 0], [0, np.exp(0.5j * phi)]],
                    dtype=np.complex128)


@dataclass
class Gate:
    qubits: Tuple[int, ...]
    matrix: np.ndarray              # complex128, (2,2) or (4,4)
    param_kind: int = PARAM_NONE    # PARAM_RY / PARAM_RZ for differentiable rotations
    param_index: int = -1
    angle: float = 0.0

    @property
    def arity(self) -> int:
        return len(self.qubits)


@dataclass
class Channel:
    name: str
    kraus: List[np.ndarray]         # list of (2,2) complex128, or (4,4) for a two-qubit channel

    @property
    def n_qubits(self) -> int:
        return 2 if np.asarray(self.kraus[0]).shape[0] == 4 else 1


@dataclass
class Site:
    gate: int
    qubit: int                      # -1: a two-qubit channel on both qubits of its (two-qubit) gate
    channel: int


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    channels: List[Channel] = field(default_factory=list)
    sites: List[Site] = field(default_factory=list)
    layout: str = "1d"
    name: str = ""
    rows: int = 0
    cols: int = 0

    @property
    def n_sites(self) -> int:
        return len(self.sites)

    def n_params(self) -> int:
        return 1 + max([g.param_index for g in self.gates] + [-1])


def circuit_seed(config: int, instance: int = 0) -> int:
    return 1000 * config + instance


def philox_seed(instance: int = 0) -> int:
    return 0x5EED0000 + instance


def haar_u2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random 2x2 unitary: QR of a complex Ginibre matrix with the phases
    of R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def depolarizing_kraus(p: float) -> Channel:
    """Single-qubit depolarizing channel rho -> (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z)."""
    i2 = np.eye(2, dtype=np.complex128)
    x = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    a, b = np.sqrt(1.0 - p), np.sqrt(p / 3.0)
    return Channel(f"depolarizing({p})", [a * i2, b * x, b * y, b * z])


PAULI = {"I": np.eye(2, dtype=np.complex128), "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
         "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128), "Z": np.diag([1.0, -1.0]).astype(np.complex128)}


def pauli_channel(p: float, pauli: str) -> Channel:
    """Single Pauli error: rho -> (1-p) rho + p P rho P."""
    return Channel(f"pauli_{pauli}({p})", [np.sqrt(1.0 - p) * PAULI["I"], np.sqrt(p) * PAULI[pauli]])


def depolarizing2_kraus(p: float) -> Channel:
    """Two-qubit depolarizing channel rho -> (1-p) rho + p/15 sum over the 15
    non-identity Pauli products P (x) Q of (P (x) Q) rho (P (x) Q); Kraus index
    4 a + b for P = (I, X, Y, Z)[a] on the gate's first qubit (the high bit) and
    Q = (I, X, Y, Z)[b] on its second."""
    names = "IXYZ"
    ks = []
    for a in range(4):
        for b in range(4):
            c = np.sqrt(1.0 - p) if a == b == 0 else np.sqrt(p / 15.0)
            ks.append(c * np.kron(PAULI[names[a]], PAULI[names[b]]))
    return Channel(f"depolarizing2({p})", ks)


def amplitude_damping_kraus(gamma: float) -> Channel:
    """Amplitude damping: K0 = [[1,0],[0,sqrt(1-g)]], K1 = [[0,sqrt(g)],[0,0]]."""
    k0 = np.array([[1, 0], [0, np.sqrt(1.0 - gamma)]], dtype=np.complex128)
    k1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    return Channel(f"amplitude_damping({gamma})", [k0, k1])


def brickwork_1d(n: int, depth: int, rng: np.random.Generator) -> Circuit:
    """1D brickwork: layer l applies a Haar U(2) to every qubit, then CZ on the
    nearest-neighbour pairs (q, q+1) with q = l mod 2, open boundary."""
    gates: List[Gate] = []
    for layer in range(depth):
        for q in range(n):
            gates.append(Gate((q,), haar_u2(rng)))
        for q in range(layer % 2, n - 1, 2):
            gates.append(Gate((q, q + 1), CZ.copy()))
    return Circuit(n, gates, layout="1d", name=f"brickwork{n}q_d{depth}")


def _grid_colour_pairs(rows: int, cols: int, colour: int) -> List[Tuple[int, int]]:
    """Pairs of the 4-colour grid pattern; qubit (r, c) has index r*cols + c.

    colour 0: horizontal pairs starting at even columns, 1: at odd columns,
    2: vertical pairs starting at even rows, 3: at odd rows."""
    pairs = []
    if colour in (0, 1):
        for r in range(rows):
            for c in range(colour, cols - 1, 2):
                pairs.append((r * cols + c, r * cols + c + 1))
    else:
        start = colour - 2
        for r in range(start, rows - 1, 2):
            for c in range(cols):
                pairs.append((r * cols + c, (r + 1) * cols + c))
    return pairs


def grid_4colour(rows: int, cols: int, depth: int, rng: np.random.Generator) -> Circuit:
    """Grid circuit: layer l applies a Haar U(2) to every qubit, then CZ on the
    pairs of colour l mod 4."""
    n = rows * cols
    gates: List[Gate] = []
    for layer in range(depth):
        for q in range(n):
            gates.append(Gate((q,), haar_u2(rng)))
        for a, b in _grid_colour_pairs(rows, cols, layer % 4):
            gates.append(Gate((a, b), CZ.copy()))
    return Circuit(n, gates, layout="grid", name=f"grid{rows}x{cols}_d{depth}",
                   rows=rows, cols=cols)


def hea_ring(n: int, layers: int, thetas: Sequence[float]) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta) then RZ(phi) on every
    qubit, then CZ on the ring (q, q+1 mod n).  Angle index order is
    (layer, qubit, {theta, phi})."""
    thetas = np.asarray(thetas, dtype=np.float64)
    assert thetas.size == layers * n * 2
    gates: List[Gate] = []
    for layer in range(layers):
        for q in range(n):
            ia = (layer * n + q) * 2
            gates.append(Gate((q,), RY(thetas[ia]), PARAM_RY, ia, float(thetas[ia])))
            gates.append(Gate((q,), RZ(thetas[ia + 1]), PARAM_RZ, ia + 1, float(thetas[ia + 1])))
        for q in range(n):
            a, b = q, (q + 1) % n
            if n == 2 and q == 1:
                break
            gates.append(Gate((a, b), CZ.copy()))
    return Circuit(n, gates, layout="ring", name=f"hea{n}q_l{layers}")


def attach_noise(circ: Circuit, channels: Sequence[Channel]) -> Circuit:
    """Couple the given channels (in order) to every qubit of every gate."""
    circ.channels = list(channels)
    sites: List[Site] = []
    for l, g in enumerate(circ.gates):
        for q in g.qubits:
            for c in range(len(channels)):
                sites.append(Site(l, q, c))
    circ.sites = sites
    return circ


def _rx(theta: float) -> np.ndarray:
    c, s_ = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -1j * s_], [-1j * s_, c]], dtype=np.complex128)


def _controlled(u: np.ndarray) -> np.ndarray:
    """Controlled-u with the control on the gate's first qubit (the high bit)."""
    m = np.eye(4, dtype=np.complex128)
    m[2:, 2:] = u
    return m


def paper_random_circuit(n: int, n_gates: int, rng: np.random.Generator, frac_2q: float = 0.2,
                         p_range=(0.02, 0.2)) -> Circuit:
    """Random circuits of the paper's benchmark family (Sec. IV-B): single-qubit
    gates from {H, X, Y, Z, T, Rx} and, for a fraction frac_2q of the gates,
    nearest-neighbour controlled gates from {CX, CY, CZ, CH, CRx} (control and
    target order random); every single-qubit gate gets a single Pauli error
    channel with a random Pauli and every two-qubit gate a two-qubit
    depolarizing channel, with error probabilities drawn uniformly from p_range.
    Rx angles are uniform in [0, 2 pi)."""
    h = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
    t = np.diag([1.0, np.exp(1j * np.pi / 4)]).astype(np.complex128)
    gates, channels, sites = [], [], []
    for l in range(n_gates):
        p = float(rng.uniform(*p_range))
        if n > 1 and rng.random() < frac_2q:
            q = int(rng.integers(0, n - 1))
            a, b = (q, q + 1) if rng.random() < 0.5 else (q + 1, q)
            kind = int(rng.integers(0, 5))
            u = [PAULI["X"], PAULI["Y"], PAULI["Z"], h, _rx(float(rng.uniform(0, 2 * np.pi)))][kind]
            gates.append(Gate((a, b), _controlled(u)))
            channels.append(depolarizing2_kraus(p))
            sites.append(Site(l, -1, len(channels) - 1))
        else:
            q = int(rng.integers(0, n))
            kind = int(rng.integers(0, 6))
            u = [h, PAULI["X"], PAULI["Y"], PAULI["Z"], t, _rx(float(rng.uniform(0, 2 * np.pi)))][kind]
            gates.append(Gate((q,), u))
            channels.append(pauli_channel(p, "XYZ"[int(rng.integers(0, 3))]))
            sites.append(Site(l, q, len(channels) - 1))
    return Circuit(n, gates, channels, sites, layout="1d", name=f"paper_random_n{n}_g{n_gates}")


def config_paper(n: int = 50, n_gates: int = 200, instance: int = 0) -> dict:
    """One instance of the paper's random-circuit family (n qubits, n_gates
    gates, 20% two-qubit, Pauli / two-qubit depolarizing noise p ~ U[0.02,
    0.2]) with the paper's sampling parameters: blocks of b = 10 and a final
    block taking the remainder up to 28 qubits, one shot per non-final block."""
    rng = np.random.default_rng(circuit_seed(6, 1000 * n + n_gates + instance))
    circ = paper_random_circuit(n, n_gates, rng)
    b, bf = 10, min(28, n)
    rest = n - bf
    bs = [b] * (rest // b) + ([rest % b] if rest % b else []) + [bf]
    return dict(name=f"paper_n{n}_g{n_gates}", circuit=circ, block_sizes=bs, seed=philox_seed(instance))


# ---------------------------------------------------------------------------
# Benchmark configurations (input recipes with their sizes)
# ---------------------------------------------------------------------------

def config_c1(instance: int = 0) -> dict:
    rng = np.random.default_rng(circuit_seed(1, instance))
    circ = attach_noise(brickwork_1d(12, 8, rng), [depolarizing_kraus(0.01)])
    return dict(name="c1_brickwork12_d8", circuit=circ, n_traj=64, shots_per_traj=1000,
                total_shots=None, block_sizes=[10, 2], seed=philox_seed(instance))


def config_c2(instance: int = 0, n_traj: int = 4096, total_shots: int = 1_000_000) -> dict:
    rng = np.random.default_rng(circuit_seed(2, instance))
    circ = attach_noise(brickwork_1d(30, 12, rng),
                        [depolarizing_kraus(0.005), amplitude_damping_kraus(0.002)])
    return dict(name="c2_brickwork30_d12", circuit=circ, n_traj=n_traj, shots_per_traj=None,
                total_shots=total_shots, block_sizes=[10, 10, 10], seed=philox_seed(instance))


def config_c3(instance: int = 0, n_circuits: int = 64) -> List[dict]:
    """Mixed batch: per circuit n ~ U{20..40} (1D) or a 6x5 grid, depth ~ U{8..16},
    depolarizing p ~ U[0.001, 0.02], E log-uniform in [16, 8192], shots
    log-uniform in [1e3, 1e6]."""
    rng = np.random.default_rng(circuit_seed(3, instance))
    out = []
    for k in range(n_circuits):
        grid = rng.random() < 0.5
        depth = int(rng.integers(8, 17))
        p = float(rng.uniform(0.001, 0.02))
        e = int(round(np.exp(rng.uniform(np.log(16), np.log(8192)))))
        shots = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e6)))))
        if grid:
            circ = grid_4colour(6, 5, depth, rng)
        else:
            circ = brickwork_1d(int(rng.integers(20, 41)), depth, rng)
        attach_noise(circ, [depolarizing_kraus(p)])
        n = circ.n_qubits
        blocks = [10] * (n // 10) + ([n % 10] if n % 10 else [])
        out.append(dict(name=f"c3_{k}_{circ.name}", circuit=circ, n_traj=e, shots_per_traj=None,
                        total_shots=shots, block_sizes=blocks, seed=philox_seed(instance) + k,
                        circuit_id=k))
    return out


def config_c4(instance: int = 0) -> dict:
    rng = np.random.default_rng(circuit_seed(4, instance))
    circ = attach_noise(grid_4colour(6, 6, 10, rng), [depolarizing_kraus(0.003)])
    return dict(name="c4_grid6x6_d10", circuit=circ, n_traj=2048, shots_per_traj=None,
                total_shots=1 << 20, block_sizes=[10, 10, 10, 6], seed=philox_seed(instance))


def config_c4_slice(instance: int = 0) -> dict:
    rng = np.random.default_rng(circuit_seed(4, 100 + instance))
    circ = attach_noise(grid_4colour(4, 4, 10, rng), [depolarizing_kraus(0.003)])
    return dict(name="c4_grid4x4_d10", circuit=circ, n_traj=2048, shots_per_traj=None,
                total_shots=1 << 20, block_sizes=[10, 6], seed=philox_seed(instance))


def config_c5(instance: int = 0) -> dict:
    rng = np.random.default_rng(circuit_seed(5, instance))
    thetas = rng.standard_normal(16 * 6 * 2)
    circ = attach_noise(hea_ring(16, 6, thetas), [depolarizing_kraus(0.01)])
    return dict(name="c5_hea16_l6", circuit=circ, thetas=thetas, n_traj=1024,
                block_sizes=[10, 6], seed=philox_seed(instance))


def synthetic_marginals(n_net: int, b: int, seed: int, zero_frac: float = 0.1,
                        dtype=np.float32) -> np.ndarray:
    """Porter-Thomas-like (exponentially distributed) unnormalised probability
    vectors of length 2**b with a fraction of exact zeros and a spread of
    scales across rows, for tests of the sampling step."""
    rng = np.random.default_rng(seed)
    p = rng.exponential(1.0, size=(n_net, 1 << b))
    p[rng.random(p.shape) < zero_frac] = 0.0
    p[:, 0] += 1e-3  # no all-zero row
    scale = np.exp(rng.uniform(np.log(1e-6), 0.0, size=(n_net, 1)))
    return (p * scale).astype(dtype)
