"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

Nothing here is part of the controller's arithmetic (no lifting, no rollout, no
safety test, no selection).  It produces the data a controller consumes:

* training transitions (x_m, u_m, x_{m+1}) for the model fit (Sec. IV-A, Sec. V-C.3);
* the race-car track as a closed centre-line polyline (Sec. V-A, Sec. V-B: a
  random road per trial, seeded);
* the user's input stream, an Ornstein-Uhlenbeck process clipped to the input box;
* the safety-set parameters of the two environments (Sec. V-C.1) as plain numbers.

Every generator takes an explicit seed and uses numpy's PCG64; none of them
touches the counter-based stream the controller draws its candidates from.
"""
from __future__ import annotations

import numpy as np

from . import plants

# State boxes the transitions are drawn from (wider than the safety set so the
# fit sees the dynamics near and across the boundary).
BOT_STATE_BOX = np.array([[-0.6, 0.6], [-2.0, 2.0], [-2.5, 2.5], [-2.0, 2.0]])
CAR_STATE_BOX = np.array([[-100.0, 100.0], [-100.0, 100.0], [-np.pi, np.pi],
                          [0.0, 30.0], [-3.0, 3.0], [-1.5, 1.5]])

# Safety sets (Sec. V-C.1): balance bot must keep |theta| < 0.5 rad and |x| < 2 m;
# race car must stay within 4 m of the centre line (8 m road) and keep vx < 25 m/s.
BOT_SAFE_LO = np.array([-0.5, -np.inf, -2.0, -np.inf])
BOT_SAFE_HI = np.array([0.5, np.inf, 2.0, np.inf])
CAR_SAFE_LO = np.array([-np.inf] * 6)
CAR_SAFE_HI = np.array([np.inf, np.inf, np.inf, 25.0, np.inf, np.inf])
CAR_TRACK_HALF_WIDTH = 4.0

TRACK_CONTROL_POINTS = 12
TRACK_SAMPLES_PER_SPAN = 32
TRACK_RADIUS = 60.0


def transitions(kind: str, seed: int, count: int):
    """i.i.d. one-step transitions: states uniform over the kind's state box,
    inputs uniform over its input box, next state from the plant."""
    p = plants.PLANTS[kind]
    box = BOT_STATE_BOX if kind == "bot" else CAR_STATE_BOX
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(box[:, 0], box[:, 1], size=(count, p["nx"]))
    u = rng.uniform(p["input_lo"], p["input_hi"], size=(count, p["nu"]))
    xn = p["step"](x, u)
    return x, u, xn


def track_control_points(seed: int, jitter: float = 0.1, radius_spread: float = 0.3):
    """12 control points at angles 2*pi*k/12 (+-jitter of the angular spacing)
    with radii TRACK_RADIUS * U(1 - spread, 1 + spread)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.arange(TRACK_CONTROL_POINTS)
    spacing = 2.0 * np.pi / TRACK_CONTROL_POINTS
    ang = k * spacing + jitter * spacing * rng.uniform(-1.0, 1.0, TRACK_CONTROL_POINTS)
    rad = TRACK_RADIUS * rng.uniform(1.0 - radius_spread, 1.0 + radius_spread,
                                     TRACK_CONTROL_POINTS)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)


def catmull_rom_closed(ctrl: np.ndarray, samples_per_span: int = TRACK_SAMPLES_PER_SPAN):
    """Periodic uniform Catmull-Rom spline through ctrl, sampled at
    samples_per_span points per span; returns the closed polyline's vertices."""
    m = len(ctrl)
    s = np.arange(samples_per_span) / samples_per_span
    out = []
    for i in range(m):
        p0, p1, p2, p3 = ctrl[(i - 1) % m], ctrl[i], ctrl[(i + 1) % m], ctrl[(i + 2) % m]
        c0 = 2.0 * p1
        c1 = p2 - p0
        c2 = 2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3
        c3 = -p0 + 3.0 * p1 - 3.0 * p2 + p3
        out.append(0.5 * (c0 + np.outer(s, c1) + np.outer(s * s, c2) + np.outer(s ** 3, c3)))
    return np.concatenate(out, axis=0)


def track_polyline(seed: int, circular: bool = False) -> np.ndarray:
    """Closed centre line (TRACK_CONTROL_POINTS*TRACK_SAMPLES_PER_SPAN vertices,
    float64).  circular=True gives the zero-jitter, constant-radius track whose
    vertices lie exactly on a circle (used by closed-form tests)."""
    if circular:
        n = TRACK_CONTROL_POINTS * TRACK_SAMPLES_PER_SPAN
        a = 2.0 * np.pi * np.arange(n) / n
        return np.stack([TRACK_RADIUS * np.cos(a), TRACK_RADIUS * np.sin(a)], axis=1)
    return catmull_rom_closed(track_control_points(seed))


def car_start_state(track: np.ndarray, vx: float = 10.0) -> np.ndarray:
    """On the centre line at vertex 0, heading along the first segment."""
    d = track[1] - track[0]
    return np.array([track[0, 0], track[0, 1], np.arctan2(d[1], d[0]), vx, 0.0, 0.0])


def ou_user_input(seed: int, ticks: int, dt: float, lo, hi,
                  theta: float = 1.0, sigma: float = 0.5) -> np.ndarray:
    """User input stream: per input dim an Ornstein-Uhlenbeck process with mean 0
    in normalised units, Euler-Maruyama at the tick dt, clipped to [-1, 1] and
    mapped affinely onto the input box [lo, hi].  Returns (ticks, M) float64."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    m = lo.shape[0]
    u = np.zeros(m)
    out = np.empty((ticks, m))
    sq = np.sqrt(dt)
    for t in range(ticks):
        u = u - theta * u * dt + sigma * sq * rng.standard_normal(m)
        u = np.clip(u, -1.0, 1.0)
        out[t] = lo + 0.5 * (u + 1.0) * (hi - lo)
    return out


def user_input_once(seed: int, lo, hi) -> np.ndarray:
    """One user input uniform over the input box (single-tick workloads)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.uniform(np.asarray(lo, float), np.asarray(hi, float))


def states_in_box(seed: int, count: int, lo, hi) -> np.ndarray:
    """count states uniform over the box [lo, hi] (per-tick state batches)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(np.asarray(lo, float), np.asarray(hi, float),
                       size=(count, len(lo)))


def to_f32_exact(a) -> np.ndarray:
    """Round to binary32 and return as float64 (values both sides can hold exactly)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def screener_init(seed: int, hidden: int = 128, n_in: int = 12) -> dict:
    """Initial weights of the learned screener (He-normal, zero biases), float32
    values held in float64 so both implementations start from the same numbers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    return {"W1": f32(rng.normal(0.0, np.sqrt(2.0 / n_in), (hidden, n_in))),
            "b1": np.zeros(hidden),
            "W2": f32(rng.normal(0.0, np.sqrt(2.0 / hidden), (hidden, hidden))),
            "b2": np.zeros(hidden),
            "w3": f32(rng.normal(0.0, np.sqrt(1.0 / hidden), hidden)),
            "b3": np.zeros(())}
