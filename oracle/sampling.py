"""Exact-integer CDF sampling and proportional non-degenerate batched sampling.
TEST INFRASTRUCTURE (see the package docstring).

Paper, Sec. III-B (NBS, proportional case): at each batch B_j the m_i shots of a
trajectory are drawn from conditional marginal distributions; block B_1 needs
one contraction per trajectory, and for j > 1 each *distinct* prefix
(s_1..s_{j-1}) already drawn is contracted once and all shots sharing it are
drawn from its conditional marginal.  Shots are carried as (prefix, count)
pairs, so no contraction is repeated for a repeated prefix.

Conventions (readings of points the paper leaves open):

* a marginal row p[0 .. 2^b) (unnormalised, FP32 or FP64, negatives clamped to
  zero) is quantised to integers P_x = rint(p_x * 2^sigma) held exactly in FP64,
  sigma = 52 - bits - e where max p = f * 2^e, f in [0.5, 1), and bits =
  ceil(log2(#bins)); the running sum C of P is then exact in any order;
* a draw takes the 64-bit word a = (x0 << 32) | x1 of one Philox4x32-10 call,
  r = floor(a * T / 2^64) with T = C[last], and returns the smallest x with
  r < C[x] (entries with P_x = 0 are never returned);
* shot rank r of trajectory i in block j (0-based) uses the counter
  (r_lo, r_hi, i, tag(SAMPLE, circuit, j)); the c shots of a parent take the
  ranks R .. R+c-1, R the sum of the counts of the trajectory's earlier
  parents in canonical order;
* a network whose marginal row is all zero (a zero-norm trajectory, possible
  with non-unitary Kraus operators) has zero probability; its shots cannot be
  drawn and are dropped, as proportional allocation gives it none;
* canonical order: trajectories in their listed order, then prefixes
  lexicographic by (x_1, x_2, ...), block 1 most significant; a child's bits
  are prefix | (x << start_j);
* proportional shot allocation draws the M shots of the whole run over the
  trajectory weights a_i = c_i * w_i (multiplicity times norm) with shot t using
  the counter (t_lo, t_hi, 0, tag(ALLOC, circuit)).
"""
import math

import numpy as np

from . import philox


def quantise(p):
    """Integer-valued FP64 weights and their running sum for one row p."""
    p = np.asarray(p, dtype=np.float64)
    p = np.where(p > 0.0, p, 0.0)
    n_bins = p.shape[-1]
    bits = int(math.ceil(math.log2(n_bins))) if n_bins > 1 else 0
    m = float(p.max())
    if m <= 0.0:
        raise ValueError("all-zero probability row")
    _, e = math.frexp(m)
    sigma = 52 - bits - e
    P = np.rint(np.ldexp(p, sigma))
    C = np.empty_like(P)
    acc = 0.0
    for i, v in enumerate(P):
        acc = acc + v
        C[i] = acc
    return P, C


def inverse_cdf(C, a):
    """Smallest x with floor(a * T / 2^64) < C[x], T = C[-1]; a uint64 array."""
    T = np.uint64(int(C[-1]))
    r = philox.mulhi64(a, T).astype(np.float64)     # < T <= 2^52: exact
    return np.searchsorted(C, r, side="right")


def draw_words(ranks, traj, tagw, seed):
    k0, k1 = philox.key_of(seed)
    ranks = np.asarray(ranks, dtype=np.uint64)
    x0, x1, _, _ = philox.philox4x32_10(ranks & philox.MASK32, ranks >> philox.S32,
                                        traj, tagw, k0, k1)
    return philox.word64(x0, x1)


def sample_block(p_rows, traj, counts, rank0, seed, block, circuit=0):
    """Draw counts[n] shots from row n of p_rows for every parent n.

    Returns the list of child bins: (parent index, x, count) in canonical order."""
    tagw = philox.tag(philox.STREAM_SAMPLE, circuit, block)
    out_parent, out_x, out_c = [], [], []
    for n in range(len(counts)):
        c = int(counts[n])
        if c == 0 or not np.any(np.asarray(p_rows[n]) > 0):
            continue        # no shots, or a zero-norm network whose shots cannot be drawn
        _, C = quantise(p_rows[n])
        ranks = np.arange(int(rank0[n]), int(rank0[n]) + c, dtype=np.uint64)
        a = draw_words(ranks, np.uint64(int(traj[n])), tagw, seed)
        xs = inverse_cdf(C, a)
        hist = np.bincount(xs, minlength=len(C))
        nz = np.nonzero(hist)[0]
        out_parent.extend([n] * len(nz))
        out_x.extend(nz.tolist())
        out_c.extend(hist[nz].tolist())
    return (np.array(out_parent, dtype=np.int64), np.array(out_x, dtype=np.int64),
            np.array(out_c, dtype=np.int64))


def rank_offsets(traj, counts):
    """Exclusive running sum of counts within each trajectory (canonical order)."""
    r0 = np.zeros(len(counts), dtype=np.int64)
    acc = {}
    for n in range(len(counts)):
        t = int(traj[n])
        r0[n] = acc.get(t, 0)
        acc[t] = r0[n] + int(counts[n])
    return r0


def allocate_shots(weights, total, seed, circuit=0):
    """m_i: one multinomial draw of ``total`` shots over the trajectory weights
    (no shot is allocated when every weight is zero)."""
    if not np.any(np.asarray(weights) > 0):
        return np.zeros(len(weights), dtype=np.int64)
    _, C = quantise(weights)
    tagw = philox.tag(philox.STREAM_ALLOC, circuit, 0)
    m = np.zeros(len(weights), dtype=np.int64)
    chunk = 1 << 20
    for t0 in range(0, total, chunk):
        t = np.arange(t0, min(total, t0 + chunk), dtype=np.uint64)
        a = draw_words(t, np.uint64(0), tagw, seed)
        m += np.bincount(inverse_cdf(C, a), minlength=len(weights))
    return m


# Bitstrings are plain integers: uint64 arrays while every block ends below
# bit 64, arrays of Python integers (dtype object) for wider circuits.
def _is_wide(blocks):
    return any(start + b > 64 for start, b in blocks)


def _zero_prefix(n, wide):
    return np.array([0] * n, dtype=object) if wide else np.zeros(n, dtype=np.uint64)


def _child_prefix(pre, xs, start, wide):
    """prefix | (x << start) for every parent prefix and outcome."""
    if not wide:
        return pre | (np.asarray(xs).astype(np.uint64) << np.uint64(start))
    return np.array([int(p) | (int(x) << start) for p, x in zip(pre, xs)], dtype=object)


def nbs_proportional(marginal_fn, blocks, seed, n_traj, circuit=0, shots=None,
                     total_shots=None, mult=None):
    """Proportional NBS over all blocks.

    marginal_fn(j, traj[], prefix[]) -> unnormalised marginal rows [n, 2^{b_j}]
    (FP64 or FP32), blocks = [(start_j, b_j)].  ``shots`` gives m_i per
    trajectory (fixed allocation); otherwise ``total_shots`` are allocated over
    a_i = mult_i * Z_i, Z_i the sum of trajectory i's block-1 marginal.

    Returns (traj, bits, count) of the final level in canonical order, the
    per-block numbers of parents D_j and the allocation m."""
    all_traj = np.arange(n_traj, dtype=np.int64)
    wide = _is_wide(blocks)
    rows0 = marginal_fn(0, all_traj, _zero_prefix(n_traj, wide))
    if shots is None:
        z = np.asarray(rows0, dtype=np.float64).sum(axis=1)
        w = z * (np.ones(n_traj) if mult is None else np.asarray(mult, np.float64))
        m = allocate_shots(w, int(total_shots), seed, circuit)
    else:
        m = np.asarray(shots, dtype=np.int64)
    keep = m > 0
    traj = all_traj[keep]
    prefix = _zero_prefix(len(traj), wide)
    counts = m[keep]
    levels = []
    for j, (start, b) in enumerate(blocks):
        levels.append(len(traj))
        rows = rows0[keep] if j == 0 else marginal_fn(j, traj, prefix)
        r0 = rank_offsets(traj, counts)
        par, xs, cs = sample_block(rows, traj, counts, r0, seed, j, circuit)
        traj = traj[par]
        prefix = _child_prefix(prefix[par], xs, start, wide)
        counts = cs
    return traj, prefix, counts, levels, m


# ------------------------------------------------ non-proportional NBS ----
#
# Paper, Sec. III-B (non-proportional case): every non-final batch draws one or
# more shots per distinct prefix from its conditional marginal (the prefixes
# branch at a user-set rate), and the final batch B_f, whose outcomes feed no
# later contraction, is harvested in bulk from its 2^{b_f} population vector,
# either by direct sampling (many shots drawn from it) or exhaustively (every
# entry above a user threshold, optionally with its probability).
#
# Readings (points the paper leaves open):
#
# * branching: parent n of a non-final block draws `branch` shots (the same
#   for every parent; 1 in the paper's experiments, Sec. IV-C), with the shot
#   ranks and Philox counters of the proportional case; its distinct outcomes
#   become the next block's prefixes;
# * the final population vector of a network with b_f bits is quantised to
#   64-bit integers, P_x = rint(max(p_x, 0) * 2^s), s = 62 - bits - e with
#   max p = f * 2^e, f in [0.5, 1) (T = sum P_x < 2^62, so the running sum is
#   exact in uint64; relative resolution 2^-(61 - b_f) of the largest entry,
#   which keeps b_f up to 30 exact enough for direct draws and thresholds);
# * direct sampling: each final network draws `final_shots` shots with the
#   proportional counters (ranks continue within the trajectory), a draw
#   taking r = floor(a T / 2^64) and the smallest x with r < C[x]; the
#   distinct outcomes are returned with their counts;
# * exhaustive sampling: the entries with P_x > 0 and P_x >= tau * T (FP64
#   product; tau is the threshold on the conditional probability p(x |
#   prefix)) are returned in increasing x with probability P_x / T (FP64).


def quantise64(p):
    """64-bit integer weights of one final population vector and their running
    sum (Python ints held in uint64 arrays)."""
    p = np.asarray(p, dtype=np.float64)
    p = np.where(p > 0.0, p, 0.0)
    n_bins = p.shape[-1]
    bits = int(math.ceil(math.log2(n_bins))) if n_bins > 1 else 0
    m = float(p.max())
    if m <= 0.0:
        raise ValueError("all-zero probability row")
    _, e = math.frexp(m)
    s = 62 - bits - e
    P = np.rint(np.ldexp(p, s)).astype(np.uint64)
    C = np.cumsum(P, dtype=np.uint64)
    return P, C


def inverse_cdf64(C, a):
    """Smallest x with floor(a * T / 2^64) < C[x], T = C[-1] < 2^62."""
    r = philox.mulhi64(a, np.uint64(int(C[-1])))
    return np.searchsorted(C, r, side="right")


def harvest_direct(p_rows, traj, prefix, start, n_shots, seed, block, circuit=0):
    """Direct sampling of the final block: n_shots draws per network (ranks
    continuing within each trajectory); returns (traj, bits, count) of the
    distinct outcomes, networks in order, x increasing."""
    tagw = philox.tag(philox.STREAM_SAMPLE, circuit, block)
    counts = np.full(len(traj), int(n_shots), dtype=np.int64)
    r0 = rank_offsets(traj, counts)
    out_t, out_b, out_c = [], [], []
    for n in range(len(traj)):
        if n_shots == 0 or not np.any(np.asarray(p_rows[n]) > 0):
            continue
        _, C = quantise64(p_rows[n])
        ranks = np.arange(int(r0[n]), int(r0[n]) + int(n_shots), dtype=np.uint64)
        xs = inverse_cdf64(C, draw_words(ranks, np.uint64(int(traj[n])), tagw, seed))
        hist = np.bincount(xs, minlength=len(C))
        nz = np.nonzero(hist)[0]
        out_t.extend([int(traj[n])] * len(nz))
        out_b.extend([int(prefix[n]) | (int(x) << start) for x in nz])
        out_c.extend(hist[nz].tolist())
    wide = start + (len(p_rows[0]) - 1).bit_length() > 64 if len(p_rows) else False
    return (np.array(out_t, dtype=np.int64), np.array(out_b, dtype=object if wide else np.uint64),
            np.array(out_c, dtype=np.int64))


def harvest_exhaustive(p_rows, traj, prefix, start, tau):
    """Exhaustive sampling of the final block: every entry with P_x > 0 and
    P_x >= tau * T; returns (traj, bits, probability P_x / T)."""
    out_t, out_b, out_p = [], [], []
    for n in range(len(traj)):
        if not np.any(np.asarray(p_rows[n]) > 0):
            continue
        P, C = quantise64(p_rows[n])
        T = float(int(C[-1]))
        Pf = P.astype(np.float64)             # each P_x rounded to FP64, like float(int(P_x))
        keep = np.nonzero((P > 0) & (Pf >= tau * T))[0]
        out_t.append(np.full(len(keep), int(traj[n]), dtype=np.int64))
        if start + (len(P) - 1).bit_length() > 64:
            out_b.append(np.array([int(prefix[n]) | (int(x) << start) for x in keep], dtype=object))
        else:
            out_b.append(np.uint64(int(prefix[n])) | (keep.astype(np.uint64) << np.uint64(start)))
        out_p.append(Pf[keep] / T)
    if not out_t:
        return np.zeros(0, np.int64), np.zeros(0, np.uint64), np.zeros(0, np.float64)
    return np.concatenate(out_t), np.concatenate(out_b), np.concatenate(out_p)


def nbs_nonproportional(marginal_fn, blocks, seed, n_traj, branch=1, mode="exhaustive", final_shots=0,
                        tau=0.0, circuit=0):
    """Non-proportional NBS over all blocks: `branch` shots per parent on every
    non-final block, then the final block harvested by direct sampling
    (`final_shots` per network) or exhaustively (threshold `tau`).

    Returns the final records ((traj, bits, count) or (traj, bits, probability))
    and the number of networks contracted per block."""
    traj = np.arange(n_traj, dtype=np.int64)
    wide = _is_wide(blocks)
    prefix = _zero_prefix(n_traj, wide)
    nets = []
    for j, (start, b) in enumerate(blocks[:-1]):
        nets.append(len(traj))
        rows = marginal_fn(j, traj, prefix)
        counts = np.full(len(traj), int(branch), dtype=np.int64)
        par, xs, _ = sample_block(rows, traj, counts, rank_offsets(traj, counts), seed, j, circuit)
        traj = traj[par]
        prefix = _child_prefix(prefix[par], xs, start, wide)
    jf = len(blocks) - 1
    start, b = blocks[jf]
    nets.append(len(traj))
    rows = marginal_fn(jf, traj, prefix)
    if mode == "direct":
        rec = harvest_direct(rows, traj, prefix, start, final_shots, seed, jf, circuit)
    elif mode == "exhaustive":
        rec = harvest_exhaustive(rows, traj, prefix, start, tau)
    else:
        raise ValueError(mode)
    return rec, nets
