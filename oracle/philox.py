"""Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), written out from its published definition.

The paper's method draws binomial/multinomial splits (Sec. II.C) but fixes no
generator; the sampler here takes its uniforms from this counter-based
generator so that the GPU sampler and the oracle draw identical numbers.

Pinned against numpy's own Philox bit generator (a library implementation of
the same published algorithm) in tests/test_oracle_philox.py.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
MASK64 = (1 << 64) - 1


def philox4x64(ctr, key, rounds: int = 10):
    """One block of four 64-bit words for counter (c0..c3) and key (k0, k1).

    Plain Python integers: each round multiplies c0 by M0 and c2 by M1 into
    128-bit products and mixes them with c1, c3 and the key; the key is
    advanced by the Weyl constants between rounds.
    """
    c0, c1, c2, c3 = (int(c) & MASK64 for c in ctr)
    k0, k1 = (int(k) & MASK64 for k in key)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + W0) & MASK64
            k1 = (k1 + W1) & MASK64
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _mulhilo(a: np.ndarray, b: int):
    """64x64 -> 128-bit product of a uint64 array and a constant, in numpy."""
    mask32 = np.uint64(0xFFFFFFFF)
    a_lo = a & mask32
    a_hi = a >> np.uint64(32)
    b_lo = np.uint64(b & 0xFFFFFFFF)
    b_hi = np.uint64(b >> 32)
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> np.uint64(32)) + (lh & mask32) + (hl & mask32)
    lo = (ll & mask32) | ((mid & mask32) << np.uint64(32))
    hi = hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))
    return hi, lo


def philox4x64_np(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Vectorised Philox4x64-10 over uint64 counter arrays (same definition)."""
    with np.errstate(over="ignore"):
        c = [np.asarray(v, dtype=np.uint64).copy() for v in np.broadcast_arrays(c0, c1, c2, c3)]
        kk0, kk1 = k0 & MASK64, k1 & MASK64
        for r in range(rounds):
            if r > 0:
                kk0 = (kk0 + W0) & MASK64
                kk1 = (kk1 + W1) & MASK64
            hi0, lo0 = _mulhilo(c[0], M0)
            hi1, lo1 = _mulhilo(c[2], M1)
            c = [hi1 ^ c[1] ^ np.uint64(kk0), lo1, hi0 ^ c[3] ^ np.uint64(kk1), lo0]
    return c


def uniform_from_word(w):
    """Map a 64-bit word to a double in [0, 1): the top 53 bits times 2^-53."""
    return (np.asarray(w, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
