"""isSafe: geometric safety checks on a predicted configuration (Sec. V-C.1).

The paper deems a state unsafe when it violates a physical barrier (balance
bot: body hits the ground; race car: leaves the road) and guards against model
error with a hand-tuned inflated barrier.  Readings (stated in the design
notes):

  * the predicted state is the read-out z[:nx] of the lifted state;
  * the safe set is an intersection of open per-coordinate intervals
    lo_j + iota < x_j < hi_j - iota (infinite bounds leave a coordinate free)
    and, for the race car, dist((x, y), centre line) < w - iota where the
    centre line is a closed polyline and w is half the road width;
  * strict inequalities: a state exactly on a bound is unsafe; any NaN is
    unsafe (every comparison with NaN is false).

The distance to the centre line is the plain definition: the minimum over all
polyline segments of the Euclidean distance to the segment, brute force.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SafetySpec:
    lo: np.ndarray                      # (nx,) lower bounds (may be -inf)
    hi: np.ndarray                      # (nx,) upper bounds (may be +inf)
    inflation: float = 0.0              # iota >= 0
    track: np.ndarray | None = None     # (S, 2) closed polyline vertices, or None
    half_width: float = 0.0             # w
    track_xy: tuple = (0, 1)            # state coordinates holding the position
    extra: dict = field(default_factory=dict)


def point_segment_distance(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Euclidean distance from points p (..., 2) to segments [a, b] (a, b (..., 2))."""
    d = b - a
    len2 = np.sum(d * d, axis=-1)
    t = np.sum((p - a) * d, axis=-1) / np.where(len2 > 0, len2, 1.0)
    t = np.clip(t, 0.0, 1.0)
    q = a + t[..., None] * d
    return np.sqrt(np.sum((p - q) ** 2, axis=-1))


def distance_to_polyline(track: np.ndarray, p: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Minimum distance from each point p (P, 2) to the closed polyline track (S, 2)."""
    p = np.asarray(p, dtype=np.float64).reshape(-1, 2)
    a = np.asarray(track, dtype=np.float64)
    d = np.roll(a, -1, axis=0) - a                     # segment i: a_i -> a_{i+1}
    len2 = np.sum(d * d, axis=1)
    inv = np.where(len2 > 0, 1.0 / np.where(len2 > 0, len2, 1.0), 0.0)
    ax, ay, dx, dy = a[:, 0], a[:, 1], d[:, 0], d[:, 1]
    out = np.empty(p.shape[0])
    for s in range(0, p.shape[0], chunk):
        rx = p[s:s + chunk, 0:1] - ax                  # p - a
        ry = p[s:s + chunk, 1:2] - ay
        t = np.clip((rx * dx + ry * dy) * inv, 0.0, 1.0)  # clamped projection
        ex = rx - t * dx                               # p - (a + t d)
        ey = ry - t * dy
        out[s:s + chunk] = np.sqrt(np.min(ex * ex + ey * ey, axis=1))
    return out


def is_safe(spec: SafetySpec, z: np.ndarray) -> np.ndarray:
    """Boolean safety of each lifted state z (P, n); reads the state from z[:, :nx]."""
    z = np.atleast_2d(np.asarray(z, dtype=np.float64))
    nx = len(spec.lo)
    x = z[:, :nx]
    lo = np.asarray(spec.lo, dtype=np.float64) + spec.inflation
    hi = np.asarray(spec.hi, dtype=np.float64) - spec.inflation
    ok = np.all((x > lo) & (x < hi), axis=1)
    if spec.track is not None:
        ix, iy = spec.track_xy
        pts = np.stack([x[:, ix], x[:, iy]], axis=1)
        d = np.full(len(pts), np.nan)
        finite = np.all(np.isfinite(pts), axis=1)
        if finite.any():
            d[finite] = distance_to_polyline(spec.track, pts[finite])
        ok &= d < (spec.half_width - spec.inflation)
    return ok


def margin(spec: SafetySpec, z: np.ndarray) -> np.ndarray:
    """Signed distance of each state from the nearest bound of the safe set (in
    read-out units; negative outside).  Used to decide whether a disagreement
    between two implementations lies at a boundary."""
    z = np.atleast_2d(np.asarray(z, dtype=np.float64))
    nx = len(spec.lo)
    x = z[:, :nx]
    lo = np.asarray(spec.lo, dtype=np.float64) + spec.inflation
    hi = np.asarray(spec.hi, dtype=np.float64) - spec.inflation
    with np.errstate(invalid="ignore"):
        m = np.minimum(x - lo, hi - x).min(axis=1)
    if spec.track is not None:
        ix, iy = spec.track_xy
        pts = np.stack([x[:, ix], x[:, iy]], axis=1)
        d = np.full(len(pts), np.nan)
        finite = np.all(np.isfinite(pts), axis=1)
        if finite.any():
            d[finite] = distance_to_polyline(spec.track, pts[finite])
        m = np.minimum(m, (spec.half_width - spec.inflation) - d)
    return m
