"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror & Shaw 2011, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3.2): a 4 x 32-bit counter and a 2 x 32-bit key; each of
ten rounds multiplies counter words 0 and 2 by two fixed 32-bit constants,
takes the high/low halves of the 64-bit products, XORs the high halves with
the other counter words and the round key, and permutes; the key is bumped by
two Weyl constants between rounds.

Test infrastructure only (see oracle/__init__.py).

Vectorised over numpy arrays of counters.  Counter layout used by the nested
sampler (both implementations follow it):

    word0 = purpose | (j << 8)   j = draw index inside one move (chunk / step)
    word1 = iteration (or replay index for the error estimate)
    word2 = chain index (or point index / dead-point index)
    word3 = move index
    key   = (seed & 0xffffffff, seed >> 32)
"""

from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

PURPOSE_INIT = 1
PURPOSE_START = 2
PURPOSE_DIR = 3
PURPOSE_STEPOUT = 4
PURPOSE_SHRINK = 5
PURPOSE_ERR = 6


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Returns the four 32-bit output words (as uint64 arrays) for counters
    (c0..c3) and key (k0, k1); arguments broadcast."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & MASK32
            k1 = (k1 + np.uint64(W1)) & MASK32
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def philox4x32_10_int(c0, c1, c2, c3, k0, k1):
    """Same definition on Python integers (scalar counters)."""
    M = 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & M
            k1 = (k1 + W1) & M
        p0 = 0xD2511F53 * c0
        p1 = 0xCD9E8D57 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0), p1 & M, ((p0 >> 32) ^ c3 ^ k1), p0 & M
    return c0, c1, c2, c3


def uniform_scalar(seed, purpose, j, w1, w2, w3):
    """u_a of one counter, as a Python float (same bits as `uniform`)."""
    k0, k1 = key_of(seed)
    x0, x1, _x2, _x3 = philox4x32_10_int((purpose | (j << 8)) & 0xFFFFFFFF, w1 & 0xFFFFFFFF,
                                         w2 & 0xFFFFFFFF, w3 & 0xFFFFFFFF, k0, k1)
    m = ((x0 << 32) | x1) >> 12
    return (2.0 * m + 1.0) * 2.0 ** -53


def _u01(hi, lo):
    """52 random bits -> (2m + 1) * 2^-53, strictly inside (0, 1), exact."""
    m = ((hi << np.uint64(32)) | lo) >> np.uint64(12)
    return (2.0 * m.astype(np.float64) + 1.0) * 2.0 ** -53


def key_of(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def uniforms(seed, purpose, j, w1, w2, w3):
    """Two uniforms (u_a, u_b) per counter."""
    k0, k1 = key_of(seed)
    w0 = np.uint64(purpose) | (np.asarray(j, dtype=np.uint64) << np.uint64(8))
    x0, x1, x2, x3 = philox4x32_10(w0, w1, w2, w3, k0, k1)
    return _u01(x0, x1), _u01(x2, x3)


def uniform(seed, purpose, j, w1, w2, w3):
    return uniforms(seed, purpose, j, w1, w2, w3)[0]


def normals(seed, purpose, w1, w2, w3, d):
    """d standard normals by the Box-Muller transform (Box & Muller 1958) of the
    uniform pairs from chunks j = 0 .. ceil(d/2)-1: dims 2j and 2j+1 take
    r cos(2 pi u_b) and r sin(2 pi u_b) with r = sqrt(-2 ln u_a)."""
    nch = (d + 1) // 2
    j = np.arange(nch, dtype=np.uint64)
    ua, ub = uniforms(seed, purpose, j, w1, w2, w3)
    r = np.sqrt(-2.0 * np.log(ua))
    ang = 6.283185307179586 * ub
    z = np.empty(2 * nch)
    z[0::2] = r * np.cos(ang)
    z[1::2] = r * np.sin(ang)
    return z[:d]


def init_point(seed, idx, d):
    """Uniform point in the unit cube for live point idx: dims 2j, 2j+1 from chunk j."""
    nch = (d + 1) // 2
    j = np.arange(nch, dtype=np.uint64)
    ua, ub = uniforms(seed, PURPOSE_INIT, j, 0, idx, 0)
    x = np.empty(2 * nch)
    x[0::2] = ua
    x[1::2] = ub
    return x[:d]
