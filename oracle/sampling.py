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


# ---- Alg. 2's per-step Gaussian noise z_i -----------------------------------
#
# Alg. 2 adds white Gaussian noise z_i to every predicted state; the paper gives
# neither its variance nor where it enters the lifted state.  Reading: after each
# prediction step t (1..H) the first n_noise lifted coordinates (the state
# read-out) get sigma_j * n_j with n_j standard normal, before that step's safety
# test; the perturbed state is carried into the next step.  sigma = 0 is Alg. 2
# without noise.
#
# Normals (Box & Muller, "A note on the generation of random normal deviates",
# Ann. Math. Stat. 29, 1958): two uniform words (w_a, w_b) give
#     u1 = ((w_a >> 8) + 1) 2^-24 in (0, 1],  u2 = (w_b >> 8) 2^-24 in [0, 1),
#     r = sqrt(-2 ln u1),  n = (r cos(2 pi u2), r sin(2 pi u2)).
# Words: Philox4x32-10 under the session's key with counter
#     (slot, t mod 2^32, (t div 2^32 mod 2^16) + 2^16 step + 2^25 block, stream),
# for a tick t below 2^48, step in 1..H and block b = 0, 1 (coordinates 4b..4b+3).
# Because step >= 1 the third word is >= 2^16, so these counters never meet the
# candidate counters (slot, t lo, t hi, stream) of any tick below 2^48.  Block b's
# words (w0, w1, w2, w3) give coordinates 4b, 4b+1 from (w0, w1) and 4b+2, 4b+3
# from (w2, w3).

def box_muller(wa, wb):
    """Two standard normals from two uint32 words (arrays), float64."""
    wa = np.asarray(wa, dtype=np.uint32)
    wb = np.asarray(wb, dtype=np.uint32)
    u1 = ((wa >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (wb >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def noise_counter(slot, tick: int, step: int, block: int, stream: int):
    """The Philox counter words of the noise for (slot, step, block) of a tick."""
    tick = int(tick)
    if not 0 <= tick < 2 ** 48:
        raise ValueError("noise needs tick < 2^48")
    slot = np.asarray(slot, dtype=np.uint64).astype(np.uint32)
    c1 = np.uint32(tick & 0xFFFFFFFF)
    c2 = np.uint32(((tick >> 32) & 0xFFFF) + (int(step) << 16) + (int(block) << 25))
    c3 = np.uint32(int(stream) & 0xFFFFFFFF)
    n = slot.shape[0]
    return (slot, np.full(n, c1, np.uint32), np.full(n, c2, np.uint32),
            np.full(n, c3, np.uint32))


def gaussian_noise(seed: int, stream: int, tick: int, n_slots: int, H: int,
                   n_noise: int) -> np.ndarray:
    """(H, n_slots, n_noise) standard normals of a tick, float64 (n_noise <= 8)."""
    if not 0 <= n_noise <= 8:
        raise ValueError("noise covers at most 8 state coordinates")
    out = np.zeros((H, n_slots, n_noise), dtype=np.float64)
    slots = np.arange(n_slots)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    for t in range(1, H + 1):
        for b in range((n_noise + 3) // 4):
            w = philox4x32(*noise_counter(slots, tick, t, b, stream), k0, k1)
            n0, n1 = box_muller(w[0], w[1])
            n2, n3 = box_muller(w[2], w[3])
            for j, v in enumerate((n0, n1, n2, n3)):
                if 4 * b + j < n_noise:
                    out[t - 1, :, 4 * b + j] = v
    return out
