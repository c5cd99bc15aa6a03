"""Philox4x32-10 counter-based generator, written from its published definition
(J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11, Sec. 3.3 / Table 2).  TEST INFRASTRUCTURE (see the
package docstring).

One call maps a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1) to
four 32-bit words.  Each of the 10 rounds multiplies c0 and c2 by the two
round constants, takes the 64-bit products' high and low halves and mixes them
with c1, c3 and the key; the key is bumped by the two Weyl constants between
rounds.

Every random number the method draws comes from this generator through a
counter layout that names what is drawn (see ``counters``), so any subset of
draws can be reproduced independently and in any order.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)

# stream tags (top byte of counter word 3)
STREAM_KRAUS = 1
STREAM_ALLOC = 2
STREAM_SAMPLE = 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Arguments are integer arrays (broadcast);
    returns four uint64 arrays holding the 32-bit output words."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0            # < 2**64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> S32, p0 & MASK32
        hi1, lo1 = p1 >> S32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def key_of(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def tag(stream: int, circuit: int = 0, block: int = 0) -> int:
    """Counter word 3: (stream << 24) | (circuit << 8) | block."""
    return ((stream & 0xFF) << 24) | ((circuit & 0xFFFF) << 8) | (block & 0xFF)


def word64(x0, x1):
    """The 64-bit value (x0 << 32) | x1 from the first two output words."""
    return (np.asarray(x0, np.uint64) << S32) | np.asarray(x1, np.uint64)


def uniform53(x0, x1):
    """u = (a >> 11) * 2**-53 in [0, 1) with a = (x0 << 32) | x1; exact in FP64."""
    a = word64(x0, x1)
    return (a >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def mulhi64(a, t):
    """floor(a * t / 2**64) for uint64 arrays a and t, exact (carries tracked)."""
    a = np.asarray(a, np.uint64)
    t = np.asarray(t, np.uint64)
    a_hi, a_lo = a >> S32, a & MASK32
    t_hi, t_lo = t >> S32, t & MASK32
    ll = a_lo * t_lo
    lh = a_lo * t_hi            # < 2**54
    hl = a_hi * t_lo            # < 2**64
    hh = a_hi * t_hi
    mid = hl + lh + (ll >> S32)     # may wrap past 2**64
    # carry detection: compute in two steps
    s1 = hl + lh
    carry1 = (s1 < hl).astype(np.uint64)
    s2 = s1 + (ll >> S32)
    carry2 = (s2 < s1).astype(np.uint64)
    del mid
    return hh + (s2 >> S32) + ((carry1 + carry2) << S32)
