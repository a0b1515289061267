"""Philox4x32-10, written from its published definition (Salmon, Moraes, Dror &
Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Sec. 4 "Philox").

Alg. 2 draws its control samples xi ~ U^{M x N}; a counter-based generator lets
the oracle and the CUDA path draw the *same* samples independently, each from
its own implementation of this definition.

Definition used (4 words of 32 bits, 2 key words, 10 rounds):
  * one round maps counter (c0, c1, c2, c3) with key (k0, k1) to
        (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
    where hi/lo are the upper/lower 32 bits of the 64-bit product;
  * between consecutive rounds the key is bumped by the Weyl constants
    (k0 += W0, k1 += W1 mod 2^32);
  * M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9 (golden ratio),
    W1 = 0xBB67AE85 (sqrt(3) - 1).

Pins: the published known-answer vectors of Philox4x32-10 (Random123, the
library that accompanies the SC'11 paper; tests/golden/philox4x32_10_kat.json)
fix the whole bit pattern; tests also pin the one- and two-round forms, the
64-bit product split against Python integers and the statistical properties the
method needs (uniform, independent words, full avalanche on counter and key).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF
ROUNDS = 10


def mulhilo32(a: int, b: np.ndarray):
    """(hi, lo) 32-bit halves of the exact 64-bit product a*b (b uint32 array)."""
    p = np.uint64(a) * np.asarray(b, dtype=np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & np.uint64(MASK32)).astype(np.uint32)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = ROUNDS):
    """Apply Philox4x32-`rounds` to counters (arrays of uint32) under key (k0, k1)."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        hi0, lo0 = mulhilo32(M0, c0)
        hi1, lo1 = mulhilo32(M1, c2)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint32(k0), lo1,
                          hi0 ^ c3 ^ np.uint32(k1), lo0)
    return c0, c1, c2, c3
