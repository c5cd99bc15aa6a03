"""Helpers of the end-to-end replay tests: the oracle's NBS procedure run level
by level on given marginal rows, and the per-draw comparison of two marginal
sources on the same parents.

Reading of the end-to-end criterion: the GPU path and the oracle use the same
Philox words and the same exact-integer CDF rule, so with identical marginal
rows their shots are identical.  With complex64 (GPU) and complex128 (oracle)
marginals a draw can land in a different bin only when its CDF position lies
within delta of the boundary between the two bins, delta the L1 distance of
the two normalised rows (the CDFs differ by at most that at any point), plus
the quantisation and floor errors of the integer CDF (below 1e-9 here)."""
import numpy as np

from oracle import philox, sampling


def nbs_levels(rows_fn, blocks, seed, m, circuit=0):
    """Proportional NBS with the per-trajectory shot counts m, marginal rows
    from rows_fn(j, traj, prefix).  Returns the final (traj, bits, count) and
    per level the parents (traj, prefix, count) with their rows."""
    n_traj = len(m)
    keep = np.asarray(m) > 0
    traj = np.arange(n_traj, dtype=np.int64)[keep]
    prefix = np.zeros(len(traj), dtype=np.uint64)
    counts = np.asarray(m, dtype=np.int64)[keep]
    levels = []
    for j, (start, b) in enumerate(blocks):
        rows = np.asarray(rows_fn(j, traj, prefix), dtype=np.float64)
        levels.append((traj, prefix, counts, rows))
        r0 = sampling.rank_offsets(traj, counts)
        par, xs, cs = sampling.sample_block(rows, traj, counts, r0, seed, j, circuit)
        traj = traj[par]
        prefix = prefix[par] | (xs.astype(np.uint64) << np.uint64(start))
        counts = cs
    return (traj, prefix, counts), levels


def _norm(row):
    row = np.where(np.asarray(row, np.float64) > 0, row, 0.0)
    s = row.sum()
    return row / s if s > 0 else row


def boundary_mismatches(rows_a, rows_b, traj, counts, seed, block, circuit=0, stream=philox.STREAM_SAMPLE):
    """Draw every parent's shots from rows_a and from rows_b with the same
    Philox words.  Returns (draws, mismatches, worst) where worst is the
    largest ratio |u - F_b(min(x_a, x_b))| / (delta + 1e-9) over mismatching
    draws (<= 1 when every mismatch is a near-boundary event)."""
    tagw = philox.tag(stream, circuit, block)
    r0 = sampling.rank_offsets(traj, counts)
    draws = mism = 0
    worst = 0.0
    for n in range(len(counts)):
        c = int(counts[n])
        if c == 0 or not np.any(rows_a[n] > 0) or not np.any(rows_b[n] > 0):
            continue
        _, Ca = sampling.quantise(rows_a[n])
        _, Cb = sampling.quantise(rows_b[n])
        ranks = np.arange(int(r0[n]), int(r0[n]) + c, dtype=np.uint64)
        a = sampling.draw_words(ranks, np.uint64(int(traj[n])), tagw, seed)
        xa = sampling.inverse_cdf(Ca, a)
        xb = sampling.inverse_cdf(Cb, a)
        draws += c
        bad = np.nonzero(xa != xb)[0]
        if len(bad) == 0:
            continue
        mism += len(bad)
        delta = np.abs(_norm(rows_a[n]) - _norm(rows_b[n])).sum()
        Tb = float(Cb[-1])
        u = philox.mulhi64(a[bad], np.uint64(int(Tb))).astype(np.float64) / Tb
        edge = Cb[np.minimum(xa[bad], xb[bad])] / Tb
        worst = max(worst, float(np.max(np.abs(u - edge) / (delta + 1e-9))))
    return draws, mism, worst
