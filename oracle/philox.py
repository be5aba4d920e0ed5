"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,
3", SC'11) in plain Python integers, and the uniform double the single-path strategy
draws at each mid-circuit measurement (Alg. 1, the sampled outcome m of Measure).

Stream layout (a reading; the paper does not say how outcomes are sampled):
key = (seed mod 2^32, seed >> 32); counter = (measurement ordinal, 0, shot mod 2^32,
shot >> 32).  The uniform u in [0, 1) is built from output words 0 and 1 as
((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53.
"""
from __future__ import annotations

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9  # golden ratio
PHILOX_W1 = 0xBB67AE85  # sqrt(3) - 1


def philox4x32_10(ctr, key):
    """Ten Philox rounds on a 4-word counter and 2-word key; returns 4 words."""
    c0, c1, c2, c3 = (int(x) & MASK32 for x in ctr)
    k0, k1 = (int(x) & MASK32 for x in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return (c0, c1, c2, c3)


def uniform(seed: int, shot: int, ordinal: int) -> float:
    """u in [0,1) with 53 random bits for measurement ``ordinal`` of ``shot``."""
    w = philox4x32_10((ordinal, 0, shot & MASK32, (shot >> 32) & MASK32),
                      (seed & MASK32, (seed >> 32) & MASK32))
    return ((w[0] >> 5) * 67108864 + (w[1] >> 6)) * (1.0 / 9007199254740992.0)
