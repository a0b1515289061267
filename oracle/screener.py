"""Learned candidate screener (not in the paper): float64 reference.

The screener predicts, for a state x_t and a candidate input xi, the normalised
time to violation ttv / H of Alg. 2's prediction, so that only the most
promising candidates need the exact rollout.  This module is the plain
statement of what the CUDA screener computes: its input features, the network
(12 -> 128 -> 128 -> 1, GELU, sigmoid output), the squared-error loss, the
backward pass by the chain rule, one Adam step, and the screening rule (which
slots a screened tick rolls out exactly: a prefix of the cost order whose length
the network sets, so that the selection is always the exhaustive one).

The hidden activation is GELU in its tanh form (Hendrycks & Gimpel 2016).

Features (12), per tick from the race-car state and the track, per candidate
from the input:
  * nearest segment i* of the closed centre line (lowest index on ties), the
    clamped projection q of the position, the unit tangent tau of segment i*
    and its left normal n;
  * e_y = (p - q) . n / w  (signed lateral offset over the half width);
  * sin(e_psi), cos(e_psi) with e_psi = psi - atan2(tau_y, tau_x);
  * vx / 25, vy / 5, omega / 2;
  * 10 x the signed curvature at the first vertex at least 5, 10, 20, 40 m of
    arc ahead of vertex i* (Menger curvature of each vertex and its two
    neighbours, positive for a left turn);
  * delta / 0.4, a  (the candidate's steer and throttle).

Parity unpinned: whether the trained network screens well is a property of the
data, not of the arithmetic; it is measured against the exhaustive evaluation.
"""
from __future__ import annotations

import math

import numpy as np

LOOKAHEAD_M = (5.0, 10.0, 20.0, 40.0)
HIDDEN = 128
N_IN = 12


# ------------------------------------------------------------------ features
def vertex_curvature(track: np.ndarray) -> np.ndarray:
    """Signed Menger curvature at each vertex of the closed polyline."""
    v = np.asarray(track, dtype=np.float64)
    prev, nxt = np.roll(v, 1, axis=0), np.roll(v, -1, axis=0)
    a, b, c = v - prev, nxt - v, nxt - prev
    cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    denom = np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1) * np.linalg.norm(c, axis=1)
    return 2.0 * cross / denom


def lookahead_table(track: np.ndarray) -> np.ndarray:
    """(S, 4): curvature at the first vertex >= each look-ahead arc length ahead of
    vertex i (walking forward along increasing index)."""
    v = np.asarray(track, dtype=np.float64)
    S = len(v)
    seg = np.linalg.norm(np.roll(v, -1, axis=0) - v, axis=1)
    kappa = vertex_curvature(v)
    out = np.empty((S, len(LOOKAHEAD_M)))
    for i in range(S):
        for m, ell in enumerate(LOOKAHEAD_M):
            acc, j = 0.0, i
            while True:
                acc += seg[j % S]
                j += 1
                if acc >= ell:
                    break
            out[i, m] = kappa[j % S]
    return out


def tick_features(track: np.ndarray, half_width: float, x: np.ndarray) -> np.ndarray:
    """The 10 per-tick features of the state x = (px, py, psi, vx, vy, omega)."""
    v = np.asarray(track, dtype=np.float64)
    a = v
    d = np.roll(v, -1, axis=0) - v
    p = np.asarray(x[:2], dtype=np.float64)
    len2 = np.sum(d * d, axis=1)
    t = np.clip(np.sum((p - a) * d, axis=1) / len2, 0.0, 1.0)
    q = a + t[:, None] * d
    dist = np.linalg.norm(p - q, axis=1)
    i = int(np.argmin(dist))
    tau = d[i] / math.sqrt(len2[i])
    nrm = np.array([-tau[1], tau[0]])
    e_y = float(np.dot(p - q[i], nrm)) / half_width
    e_psi = x[2] - math.atan2(tau[1], tau[0])
    look = lookahead_table(v)[i]
    return np.array([e_y, math.sin(e_psi), math.cos(e_psi), x[3] / 25.0, x[4] / 5.0,
                     x[5] / 2.0, *(10.0 * look)])


def candidate_features(tick_feat: np.ndarray, cands: np.ndarray) -> np.ndarray:
    """(N, 12) network inputs: the tick's 10 features and each candidate's 2."""
    cands = np.atleast_2d(np.asarray(cands, dtype=np.float64))
    n = cands.shape[0]
    return np.hstack([np.broadcast_to(tick_feat, (n, 10)),
                      np.stack([cands[:, 0] / 0.4, cands[:, 1]], axis=1)])


# ------------------------------------------------------------------ network
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    """GELU in its tanh form (Hendrycks & Gimpel 2016):
    0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params: dict, f: np.ndarray) -> dict:
    """Forward pass on inputs f (B, 12); returns every intermediate."""
    W1, b1, W2, b2, w3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    z1 = f @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    z3 = h2 @ w3 + b3
    y = sigmoid(z3)
    return dict(f=f, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, y=y)


def loss(y: np.ndarray, target: np.ndarray) -> float:
    return float(np.mean((y - target) ** 2))


def backward(params: dict, cache: dict, target: np.ndarray) -> dict:
    """Gradients of the mean squared error by the chain rule."""
    B = target.shape[0]
    y = cache["y"]
    d3 = (2.0 / B) * (y - target) * y * (1.0 - y)          # dL/dz3
    g = {"w3": cache["h2"].T @ d3, "b3": np.sum(d3)}
    d2 = np.outer(d3, params["w3"]) * gelu_grad(cache["z2"])
    g["W2"] = d2.T @ cache["h1"]
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ params["W2"]) * gelu_grad(cache["z1"])
    g["W1"] = d1.T @ cache["f"]
    g["b1"] = d1.sum(axis=0)
    return g


def adam_step(params: dict, grads: dict, state: dict, step: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place (Kingma & Ba 2015); step counts from 1."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** step)
        vh = v / (1 - beta2 ** step)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------------ screening rule
BIN_SHIFT = 20  # cost bins: float32 exponent and the top three mantissa bits


def cost_bin(cost) -> np.ndarray:
    """Bin of a candidate's cost (>= 0) in the screened tick: the bits of the
    cost as a float32 shifted right by BIN_SHIFT.  For non-negative floats the bit
    pattern is monotone in the value, so bins never invert the cost order."""
    c = np.ascontiguousarray(np.asarray(cost, dtype=np.float32))
    return (c.view(np.uint32) >> np.uint32(BIN_SHIFT)).astype(np.int64)


def screen(scores: np.ndarray, cost: np.ndarray, k: int, tau: float, m: int = 1) -> np.ndarray:
    """Slots a screened tick rolls out, ascending: the shortest prefix of the cost
    order, cut between cost bins, that holds at least k slots and -- when tau > 0
    -- at least m slots the network predicts safe (score >= tau); every slot when
    no prefix does.  Every slot left out costs more than every slot kept."""
    b = cost_bin(cost)
    safe = np.asarray(scores) >= tau
    for edge in np.unique(b):  # ascending
        inside = b <= edge
        if inside.sum() >= k and (tau <= 0 or np.count_nonzero(inside & safe) >= m):
            return np.flatnonzero(inside)
    return np.arange(len(b))


def screened_selection(ttv: np.ndarray, cost: np.ndarray, kept: np.ndarray, H: int) -> int:
    """Slot a screened tick selects from the exact rollout of the kept slots: the
    least (cost, slot) safe kept slot; when none is safe, the full evaluation's
    choice over all slots (least (H - ttv, cost, slot))."""
    kept = np.asarray(kept)
    safe = kept[np.asarray(ttv)[kept] == H]
    if len(safe):
        return int(safe[np.lexsort((safe, np.asarray(cost)[safe]))[0]])
    slot = np.arange(len(ttv))
    return int(np.lexsort((slot, cost, H - np.asarray(ttv)))[0])
