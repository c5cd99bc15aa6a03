"""Pre-trajectory sampling (PTS) and the unified-path-variation (UPV) merge.
TEST INFRASTRUCTURE (see the package docstring).

Paper, Sec. II-C: E error sets K_i = {k_p^i} are drawn before any network is
built, by a rule the user picks (in proportion to the error probabilities, for
example).  Reading used here: each noise site s draws Kraus index k with the state-independent nominal
probability q_{s,k} = Tr(K_k^dagger K_k) / 2 (these sum to one by the
completeness relation), and the trajectory inserts K_k / sqrt(q_{s,k}), which
makes the average of |psi_i><psi_i| over draws equal to the density matrix.

Paper, Sec. III-A (UPV): every error operator is merged into the coherent gate
d_l it follows, so the network of every error set has the structure of the
error-free network; the merged gate is (N_a (x) N_b) d_l where N_q is the
product, in application order, of the scaled Kraus operators on qubit q.

Draw layout: site s of trajectory i uses the Philox4x32-10 counter
(s, 0, i, tag(KRAUS, circuit)) and key = seed; u = uniform53(x0, x1); the index
is the smallest k with u < C_s[k], C_s the running sum of q_{s,.} in index
order with its last entry set to 1.0.
"""
import numpy as np

from . import philox


def kraus_probs(kraus):
    """q_k = Tr(K_k^dagger K_k) / d (d = 2 or 4 for a one- or two-qubit
    channel), summed as re*re + im*im over the entries in row-major order (a
    fixed order, so every implementation gets the same bits)."""
    q = []
    for k in kraus:
        k = np.asarray(k, np.complex128)
        acc = 0.0
        for z in k.reshape(-1):
            acc = acc + (z.real * z.real + z.imag * z.imag)
        q.append(acc / float(k.shape[0]))
    return np.array(q, dtype=np.float64)


def kraus_cdf(kraus):
    """Running sum of q in index order, the last entry forced to 1.0."""
    q = kraus_probs(kraus)
    c = np.empty_like(q)
    acc = 0.0
    for i, v in enumerate(q):
        acc = acc + v
        c[i] = acc
    c[-1] = 1.0
    return c


def completeness_error(kraus):
    """max |sum_k K_k^dagger K_k - I| (zero for a trace-preserving channel)."""
    s = sum(np.conj(k).T @ k for k in kraus)
    return float(np.max(np.abs(s - np.eye(s.shape[0]))))


def presample(circ, n_traj: int, seed: int, circuit_id: int = 0, traj0: int = 0):
    """Draw the Kraus index of every site of trajectories traj0 .. traj0 +
    n_traj - 1 (trajectory i uses counter word i, so a range is the same rows
    of a draw that starts at 0).

    Returns (kraus[E, S] uint8, logq[E] float64) where logq_i = sum over sites,
    in site order, of log q_{s, k_{i,s}}."""
    S = circ.n_sites
    k0, k1 = philox.key_of(seed)
    t = philox.tag(philox.STREAM_KRAUS, circuit_id, 0)
    s_idx, i_idx = np.meshgrid(np.arange(S, dtype=np.uint64),
                               np.arange(traj0, traj0 + n_traj, dtype=np.uint64))
    x0, x1, _, _ = philox.philox4x32_10(s_idx, 0, i_idx, t, k0, k1)
    u = philox.uniform53(x0, x1)                           # [E, S]
    kraus = np.zeros((n_traj, S), dtype=np.uint8)
    logq = np.zeros(n_traj, dtype=np.float64)
    logtab = []
    for s, site in enumerate(circ.sites):
        ch = circ.channels[site.channel]
        cdf = kraus_cdf(ch.kraus)
        # smallest k with u < C[k]
        kk = np.searchsorted(cdf, u[:, s], side="right")
        kraus[:, s] = kk
        with np.errstate(divide="ignore"):
            logtab.append(np.log(kraus_probs(ch.kraus)))
    for i in range(n_traj):
        acc = 0.0
        for s in range(S):
            acc = acc + logtab[s][kraus[i, s]]
        logq[i] = acc
    return kraus, logq


def dedup(kraus, logq):
    """Distinct Kraus rows in first-occurrence order with their multiplicities.

    Returns (kraus_u, logq_u, mult, first_index)."""
    seen = {}
    order = []
    mult = []
    for i in range(kraus.shape[0]):
        key = kraus[i].tobytes()
        if key in seen:
            mult[seen[key]] += 1
        else:
            seen[key] = len(order)
            order.append(i)
            mult.append(1)
    order = np.array(order, dtype=np.int64)
    return kraus[order], logq[order], np.array(mult, dtype=np.int64), order


def gate_sites(circ):
    """For every gate, the list of site indices attached to it (in order)."""
    per_gate = [[] for _ in circ.gates]
    for s, site in enumerate(circ.sites):
        per_gate[site.gate].append(s)
    return per_gate


def noise_operator(circ, sites, choices, qubit):
    """N_q: product, in application order, of K_k / sqrt(q_k) over the sites on
    ``qubit`` (later operators multiply from the left)."""
    n = np.eye(2, dtype=np.complex128)
    for s in sites:
        site = circ.sites[s]
        if site.qubit != qubit:
            continue
        ch = circ.channels[site.channel]
        k = int(choices[s])
        q = kraus_probs(ch.kraus)[k]
        n = (ch.kraus[k] / np.sqrt(q)) @ n
    return n


def merged_gate(circ, l: int, choices, sites_of_gate=None):
    """UPV merge of gate l with its sampled error operators: (N_a (x) N_b) d_l,
    or, when a two-qubit channel acts on the gate, the product in application
    order of every site's scaled operator (a one-qubit one embedded on its
    qubit, the gate's first qubit being the high bit) times d_l."""
    g = circ.gates[l]
    sites = (sites_of_gate or gate_sites(circ))[l]
    if g.arity == 1:
        return noise_operator(circ, sites, choices, g.qubits[0]) @ g.matrix
    if any(circ.sites[s].qubit < 0 for s in sites):
        t = np.eye(4, dtype=np.complex128)
        for s in sites:
            site = circ.sites[s]
            ch = circ.channels[site.channel]
            k = int(choices[s])
            op = ch.kraus[k] / np.sqrt(kraus_probs(ch.kraus)[k])
            if site.qubit < 0:
                e = op
            elif site.qubit == g.qubits[0]:
                e = np.kron(op, np.eye(2))
            else:
                e = np.kron(np.eye(2), op)
            t = e @ t
        return t @ g.matrix
    na = noise_operator(circ, sites, choices, g.qubits[0])
    nb = noise_operator(circ, sites, choices, g.qubits[1])
    return np.kron(na, nb) @ g.matrix
