"""Candidate control samples (Alg. 2, first step; Sec. IV-B).

Alg. 2 draws xi ~ U^{M x N} (uniform, i.i.d.); Sec. IV-B also describes an
equally spaced discretisation of the input space.  Both are given here.

Uniform stream (the reading both implementations follow):
  * key = (seed mod 2^32, seed div 2^32);
  * sample s (0-based) of tick t in stream sigma uses counter
    (s, t mod 2^32, t div 2^32, sigma);
  * output word j (j < M, M <= 4) gives u_j = (word_j >> 8) * 2^-24, exact in
    binary32, in [0, 1);
  * xi_j = fl32(lo32_j + fl32(w32_j * u_j)), with lo32 = fl32(lo) and
    w32 = fl32(hi - lo): one binary32 multiply and one binary32 add, each
    rounded to nearest.  Candidate values are therefore binary32 numbers; the
    oracle holds them in float64 without loss.

Grid (Sec. IV-B, used with Eq. 2): for N = G^M samples, dimension j takes the
cell midpoints lo_j + (g + 1/2) (hi_j - lo_j) / G, g = 0..G-1; sample s has
digits g_j = (s div G^j) mod G.  Each value is computed in float64 as
((g + 0.5) * (hi - lo)) / G + lo and then rounded once to binary32.  With
midpoints the spacing is lambda/N for M = 1, so the largest distance from any
u_h in [lo, hi] to its nearest sample is lambda/(2N), the value of Eq. 2.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32

TWO_M24 = np.float32(2.0 ** -24)


def uniform_samples(seed: int, stream: int, tick: int, n: int, lo, hi) -> np.ndarray:
    """(n, M) float64 array of binary32 candidate values from the Philox stream."""
    lo = np.atleast_1d(np.asarray(lo, dtype=np.float64))
    hi = np.atleast_1d(np.asarray(hi, dtype=np.float64))
    m = lo.shape[0]
    if not 1 <= m <= 4:
        raise ValueError("input dimension must be 1..4")
    s = np.arange(n, dtype=np.uint64).astype(np.uint32)
    t_lo = np.uint32(int(tick) & 0xFFFFFFFF)
    t_hi = np.uint32((int(tick) >> 32) & 0xFFFFFFFF)
    words = philox4x32(s, np.full(n, t_lo, np.uint32), np.full(n, t_hi, np.uint32),
                       np.full(n, np.uint32(int(stream) & 0xFFFFFFFF), np.uint32),
                       int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    out = np.empty((n, m), dtype=np.float64)
    for j in range(m):
        u = (words[j] >> np.uint32(8)).astype(np.float32) * TWO_M24
        lo32 = np.float32(lo[j])
        w32 = np.float32(hi[j] - lo[j])
        xi = lo32 + (w32 * u).astype(np.float32)
        out[:, j] = xi.astype(np.float32).astype(np.float64)
    return out


def grid_samples(n: int, lo, hi) -> np.ndarray:
    """(n, M) float64 array of binary32 grid midpoints; n must be G**M."""
    lo = np.atleast_1d(np.asarray(lo, dtype=np.float64))
    hi = np.atleast_1d(np.asarray(hi, dtype=np.float64))
    m = lo.shape[0]
    g = int(round(n ** (1.0 / m)))
    while g ** m > n:
        g -= 1
    while (g + 1) ** m <= n:
        g += 1
    if g ** m != n:
        raise ValueError("grid sampling needs N = G**M")
    s = np.arange(n)
    out = np.empty((n, m), dtype=np.float64)
    for j in range(m):
        digit = (s // (g ** j)) % g
        v = ((digit + 0.5) * (hi[j] - lo[j])) / g + lo[j]
        out[:, j] = v.astype(np.float32).astype(np.float64)
    return out
