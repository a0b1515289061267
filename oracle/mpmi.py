"""Alg. 2 (MPMI-SC): sample, predict, reject, choose the least intervention.

One control tick, given the current state x_t and the user's input u_h:

  1. candidates xi_i (Alg. 2: xi ~ U^{M x N}; see ``sampling``).  Reading: the
     user's own input is candidate slot 0 ahead of the N samples, so a safe u_h
     passes through unchanged as Alg. 1's text requires (Sec. III-C); with
     include_user=False the slots are the samples alone, as Alg. 2 is printed.
  2. for every candidate (Alg. 2 "in parallel"): lift z_0 = Psi(x_t, xi_i)
     (Sec. IV-A), then for t = 1..H: z <- K z (+ noise, sigma = 0 by default),
     test isSafe on the predicted state, and stop at the first violation
     (Alg. 2's while-loop).  ttv_i counts the steps passed before the first
     violation; the candidate is safe iff ttv_i = H (x_t itself is not tested).
  3. cost_i = ||xi_i - u_h||^2 (Sec. IV-D: Euclidean distance; squaring keeps
     the order).
  4. u_r = argmin cost over the safe candidates (Alg. 2's store), ties to the
     lowest slot.  The paper does not say what happens when no candidate is
     safe; reading: fall back to the least-violating candidate, the one that
     survives longest (max ttv), then least cost, then lowest slot.  Both cases
     are the lexicographic minimum of (H - ttv, cost, slot).

Everything is float64.  K is used as given (tests pass the binary32-rounded
operator so only arithmetic error separates the oracle from a binary32 rollout).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .basis import lift
from .safety import SafetySpec, is_safe

SAFE = 0
FALLBACK = 1


@dataclass
class TickResult:
    u_r: np.ndarray          # (M,) selected input (u_h itself when slot 0 wins)
    index: int               # selected slot
    status: int              # SAFE or FALLBACK
    n_safe: int              # number of safe candidates
    ttv: np.ndarray          # (N_eff,) steps passed before the first violation
    cost: np.ndarray         # (N_eff,) squared distance to u_h
    candidates: np.ndarray   # (N_eff, M) candidate inputs, slot order
    executed_steps: int      # prediction steps actually taken (early exit)
    traj: np.ndarray | None  # (N_eff, H+1, n) lifted states, NaN where not predicted


def candidate_slots(u_h, samples, include_user: bool) -> np.ndarray:
    samples = np.atleast_2d(np.asarray(samples, dtype=np.float64))
    if include_user:
        return np.vstack([np.atleast_2d(np.asarray(u_h, dtype=np.float64)), samples])
    return samples


def tick(K, basis: str, x_t, u_h, samples, H: int, spec: SafetySpec,
         include_user: bool = True, record: bool = False,
         noise: np.ndarray | None = None) -> TickResult:
    """One MPMI-SC tick (Alg. 2).  samples (N, M); noise, if given, is an
    (H, N_eff, n_noise) array added to the first n_noise lifted coordinates after
    each prediction step (Alg. 2's z_i; a reading: only the state read-out is
    perturbed)."""
    K = np.asarray(K, dtype=np.float64)
    u_h = np.atleast_1d(np.asarray(u_h, dtype=np.float64))
    cands = candidate_slots(u_h, samples, include_user)
    n_eff = cands.shape[0]
    z = lift(basis, np.asarray(x_t, dtype=np.float64)[None, :], cands)
    n = z.shape[1]
    traj = None
    if record:
        traj = np.full((n_eff, H + 1, n), np.nan)
        traj[:, 0] = z
    ttv = np.zeros(n_eff, dtype=np.int64)
    alive = np.ones(n_eff, dtype=bool)
    executed = 0
    with np.errstate(over="ignore", invalid="ignore"):
        for t in range(1, H + 1):
            idx = np.nonzero(alive)[0]
            if idx.size == 0:
                break
            executed += idx.size
            zn = z[idx] @ K.T
            if noise is not None:
                k = noise.shape[2]
                zn[:, :k] += noise[t - 1, idx]
            z[idx] = zn
            if record:
                traj[idx, t] = zn
            ok = is_safe(spec, zn)
            ttv[idx[ok]] = t
            alive[idx[~ok]] = False
    cost = np.sum((cands - u_h[None, :]) ** 2, axis=1)
    slot = np.arange(n_eff)
    order = np.lexsort((slot, cost, H - ttv))
    best = int(order[0])
    n_safe = int(np.count_nonzero(ttv == H))
    status = SAFE if ttv[best] == H else FALLBACK
    u_r = u_h.copy() if (include_user and best == 0) else cands[best].copy()
    return TickResult(u_r=u_r, index=best, status=status, n_safe=n_safe, ttv=ttv,
                      cost=cost, candidates=cands, executed_steps=executed, traj=traj)


def deviation(u_r, u_h) -> float:
    """||u_h, u_r|| of Sec. IV-D (Euclidean)."""
    return float(np.linalg.norm(np.asarray(u_r, float) - np.asarray(u_h, float)))


def closed_loop(K, basis: str, spec: SafetySpec, plant_step, x0, user_inputs,
                sample_fn, H: int, include_user: bool = True):
    """Receding-horizon loop (Sec. IV-C): re-solve Alg. 2 each tick from the
    plant's current state and apply u_r.  sample_fn(tick) -> (N, M) samples.
    Returns per-tick (x_t, u_h, TickResult) records."""
    x = np.asarray(x0, dtype=np.float64)
    out = []
    for t, u_h in enumerate(user_inputs):
        r = tick(K, basis, x, u_h, sample_fn(t), H, spec, include_user)
        out.append((x.copy(), np.asarray(u_h, float), r))
        x = plant_step(x, r.u_r)
    return out
