"""Analytic stand-ins for the two simulated plants of Sec. V-A.

The paper drives a PyBullet balance bot and a Box2D race car.  Neither engine is
available, so the workloads use two textbook models with fixed constants:

* balance bot: the classic cart-pole (Barto, Sutton & Anderson 1983), state
  (theta, theta_dot, x, x_dot), one input u in [-1, 1] scaled to a 10 N force,
  dt = 0.01 s (the 100 Hz loop of Sec. VI-C);
* race car: a dynamic bicycle with linear tyres, state (x, y, psi, vx, vy, omega)
  with body-frame velocities, inputs (steer delta in [-0.4, 0.4] rad,
  throttle a in [-1, 1]), dt = 1/60 s (the 60 Hz loop of Sec. VI-C).

Both integrate with semi-implicit Euler (velocities first, then positions with
the new velocities).  These functions are the plant, i.e. the environment the
controller acts on; they are not part of the controller's arithmetic.  All
functions are vectorised over a leading batch axis and run in float64.
"""
from __future__ import annotations

import numpy as np

# --- balance bot (cart-pole) ------------------------------------------------
BOT_DT = 0.01
BOT_G = 9.8
BOT_M_CART = 1.0
BOT_M_POLE = 0.1
BOT_HALF_LEN = 0.5
BOT_FORCE = 10.0
BOT_NX, BOT_NU = 4, 1
BOT_INPUT_LO, BOT_INPUT_HI = np.array([-1.0]), np.array([1.0])

# --- race car (dynamic bicycle) ---------------------------------------------
CAR_DT = 1.0 / 60.0
CAR_MASS = 1500.0
CAR_IZ = 2250.0
CAR_LF = 1.2
CAR_LR = 1.4
CAR_CF = 8.0e4
CAR_CR = 8.0e4
CAR_FX = 5000.0
CAR_VX_MIN_SLIP = 1.0
CAR_NX, CAR_NU = 6, 2
CAR_INPUT_LO, CAR_INPUT_HI = np.array([-0.4, -1.0]), np.array([0.4, 1.0])


def cartpole_step(x: np.ndarray, u: np.ndarray, dt: float = BOT_DT) -> np.ndarray:
    """One semi-implicit Euler step of the cart-pole; x (..., 4), u (..., 1)."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    th, thd, pos, vel = x[..., 0], x[..., 1], x[..., 2], x[..., 3]
    force = BOT_FORCE * u[..., 0]
    total = BOT_M_CART + BOT_M_POLE
    s, c = np.sin(th), np.cos(th)
    tmp = (force + BOT_M_POLE * BOT_HALF_LEN * thd * thd * s) / total
    th_acc = (BOT_G * s - c * tmp) / (
        BOT_HALF_LEN * (4.0 / 3.0 - BOT_M_POLE * c * c / total))
    x_acc = tmp - BOT_M_POLE * BOT_HALF_LEN * th_acc * c / total
    thd_n = thd + dt * th_acc
    vel_n = vel + dt * x_acc
    out = np.empty_like(x)
    out[..., 0] = th + dt * thd_n
    out[..., 1] = thd_n
    out[..., 2] = pos + dt * vel_n
    out[..., 3] = vel_n
    return out


def bicycle_step(x: np.ndarray, u: np.ndarray, dt: float = CAR_DT) -> np.ndarray:
    """One semi-implicit Euler step of the dynamic bicycle; x (..., 6), u (..., 2)."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    px, py, psi = x[..., 0], x[..., 1], x[..., 2]
    vx, vy, om = x[..., 3], x[..., 4], x[..., 5]
    delta, acc = u[..., 0], u[..., 1]
    vx_c = np.maximum(vx, CAR_VX_MIN_SLIP)
    alpha_f = delta - np.arctan2(vy + CAR_LF * om, vx_c)
    alpha_r = -np.arctan2(vy - CAR_LR * om, vx_c)
    fyf = CAR_CF * alpha_f
    fyr = CAR_CR * alpha_r
    fx = CAR_FX * acc
    vx_dot = (fx - fyf * np.sin(delta)) / CAR_MASS + vy * om
    vy_dot = (fyf * np.cos(delta) + fyr) / CAR_MASS - vx * om
    om_dot = (CAR_LF * fyf * np.cos(delta) - CAR_LR * fyr) / CAR_IZ
    vx_n = vx + dt * vx_dot
    vy_n = vy + dt * vy_dot
    om_n = om + dt * om_dot
    psi_n = psi + dt * om_n
    c, s = np.cos(psi_n), np.sin(psi_n)
    out = np.empty_like(x)
    out[..., 0] = px + dt * (vx_n * c - vy_n * s)
    out[..., 1] = py + dt * (vx_n * s + vy_n * c)
    out[..., 2] = psi_n
    out[..., 3] = vx_n
    out[..., 4] = vy_n
    out[..., 5] = om_n
    return out


def linear_step(A: np.ndarray, B: np.ndarray, x: np.ndarray, u: np.ndarray) -> np.ndarray:
    """x' = A x + B u for a linear plant (used by the closed-form pins)."""
    return np.asarray(x) @ np.asarray(A).T + np.asarray(u) @ np.asarray(B).T


PLANTS = {
    "bot": dict(step=cartpole_step, nx=BOT_NX, nu=BOT_NU, dt=BOT_DT,
                input_lo=BOT_INPUT_LO, input_hi=BOT_INPUT_HI),
    "car": dict(step=bicycle_step, nx=CAR_NX, nu=CAR_NU, dt=CAR_DT,
                input_lo=CAR_INPUT_LO, input_hi=CAR_INPUT_HI),
}
