"""Philox4x32-10 counter-based generator, plain Python (CPU).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: it is the oracle side of
the counter-based random numbers that the GPU event generator draws, written
from the published definition (J. K. Salmon, M. A. Moraes, R. O. Dror,
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4):
a 128-bit counter (four 32-bit words) and a 64-bit key; each of ten rounds
multiplies counter words 0 and 2 by two constants (64-bit products), and the
new counter is (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
lo(M0 c0)); the key words grow by two Weyl constants between rounds.
Pinned by the known-answer vectors published with the generator."""
from __future__ import annotations

MASK = 0xFFFFFFFF
M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(counter, key):
    """Four 32-bit words from a four-word counter and a two-word key."""
    c0, c1, c2, c3 = (int(x) & MASK for x in counter)
    k0, k1 = (int(x) & MASK for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
    return c0, c1, c2, c3


def u01(a: int, b: int) -> float:
    """A double in [0, 1) from 53 bits: the 32 bits of a and the top 21 of b."""
    return float(((a & MASK) << 21) | ((b & MASK) >> 11)) / 9007199254740992.0
