"""Lifted features Psi(x, u) of the learned linear model (Sec. IV-A).

The paper models the plant with a Koopman operator: a linear map K acting on a
vector of functions of state and input, so one prediction step is z <- K z
(Sec. IV-A: one matrix-vector product per step, one matrix-matrix product for a
batch).  The paper selects 6 and 26 functions out of 50 and 150 random ones
(Sec. V-C.3) with code that is not available; the bases below are fixed lists
of the same kinds (state coordinates, trig and polynomial terms, input terms),
with the state coordinates first so the predicted state is read off z[:nx].

Readings (stated in the design notes):
  * the input is held constant over the horizon (Sec. VII-B, implicit user
    model), so z contains input features and the fit target is
    Psi(x_{m+1}, u_m);
  * features are listed in the order below; nothing else depends on the order.

Feature lists:
  bot (n = 12, x = (theta, theta_dot, x, x_dot), u scalar):
      theta, theta_dot, x, x_dot, u, sin th, cos th, thd^2, thd*u,
      thd^2*sin th, u*cos th, 1
  car (n = 32, x = (px, py, psi, vx, vy, om), u = (delta, a)):
      px, py, psi, vx, vy, om, delta, a, sin psi, cos psi,
      vx cos, vx sin, vy cos, vy sin, om vx, om vy, vx^2, vy^2, om^2,
      delta vx, delta vy, delta om, a vx, delta cos, delta sin, a cos, a sin,
      om cos, om sin, vx vy, delta^2, 1
  linear (n = nx + nu): x, u  (closed-form tests: K = [[A, B], [0, I]])
"""
from __future__ import annotations

import numpy as np

BASES = {
    "bot": dict(n=12, nx=4, nu=1),
    "car": dict(n=32, nx=6, nu=2),
}


# Features that depend on the input alone (and the constant).  With the input
# held over the horizon (Sec. VII-B) a prediction step leaves them unchanged, so
# their rows of K are unit rows (see ``fit``).
HELD = {"bot": (4, 11), "car": (6, 7, 30, 31)}


def held_features(basis: str, nx: int | None = None, nu: int | None = None):
    """Indices of the held (input-only and constant) features of a basis."""
    if basis == "linear":
        return tuple(range(nx, nx + nu))
    return HELD[basis]


def dims(basis: str, nx: int | None = None, nu: int | None = None):
    """(n, nx, nu) of a basis; the linear basis takes nx, nu explicitly."""
    if basis == "linear":
        return nx + nu, nx, nu
    b = BASES[basis]
    return b["n"], b["nx"], b["nu"]


def lift_bot(x: np.ndarray, u: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    th, thd, pos, vel = x[..., 0], x[..., 1], x[..., 2], x[..., 3]
    uu = u[..., 0]
    s, c = np.sin(th), np.cos(th)
    feats = [th, thd, pos, vel, uu, s, c, thd * thd, thd * uu,
             thd * thd * s, uu * c, np.ones_like(th)]
    return np.stack(np.broadcast_arrays(*feats), axis=-1)


def lift_car(x: np.ndarray, u: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    px, py, psi = x[..., 0], x[..., 1], x[..., 2]
    vx, vy, om = x[..., 3], x[..., 4], x[..., 5]
    d, a = u[..., 0], u[..., 1]
    s, c = np.sin(psi), np.cos(psi)
    feats = [px, py, psi, vx, vy, om, d, a, s, c,
             vx * c, vx * s, vy * c, vy * s, om * vx, om * vy,
             vx * vx, vy * vy, om * om,
             d * vx, d * vy, d * om, a * vx,
             d * c, d * s, a * c, a * s,
             om * c, om * s, vx * vy, d * d, np.ones_like(px)]
    return np.stack(np.broadcast_arrays(*feats), axis=-1)


def lift(basis: str, x: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Psi(x, u) in float64; x (..., nx), u (..., nu) broadcast against each other."""
    if basis == "bot":
        return lift_bot(x, u)
    if basis == "car":
        return lift_car(x, u)
    if basis == "linear":
        x = np.asarray(x, dtype=np.float64)
        u = np.asarray(u, dtype=np.float64)
        shape = np.broadcast_shapes(x.shape[:-1], u.shape[:-1])
        x = np.broadcast_to(x, shape + x.shape[-1:])
        u = np.broadcast_to(u, shape + u.shape[-1:])
        return np.concatenate([x, u], axis=-1)
    raise ValueError(f"unknown basis {basis!r}")
