"""Comparison of the CUDA tick against the FP64 oracle (test helper).

Tolerances (stated in the design notes):
  * trajectories: at every step both sides computed,
        ||z_gpu - z_ref||_inf / max(||z_ref||_inf, 1) <= 1e-4;
  * time-to-violation: equal for every candidate, except where the two sides
    disagree at a step whose reference state lies at a safety boundary, i.e.
    |margin(z_ref)| <= ||z_gpu - z_ref||_inf + 1e-5 * max(||z_ref||_inf, 1);
  * cost: float32 vs float64, relative 1e-6;
  * selection: the same slot, except when the two picks tie in cost within 1e-6
    (relative) or either pick's time-to-violation differs at a boundary;
  * integer outputs (slot, status, n_safe, executed steps) are checked exactly
    against the GPU's own per-candidate arrays.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import fit as ofit
from oracle import mpmi as omp
from oracle import safety as osafe
from oracle import sampling as osamp
from workloads import data, plants

TRAJ_RTOL = 1e-4
BOUNDARY_TOL = 1e-5
TIE_RTOL = 1e-6
COST_RTOL = 1e-6

BOT_BOX = (data.BOT_SAFE_LO, data.BOT_SAFE_HI)
CAR_BOX = (data.CAR_SAFE_LO, data.CAR_SAFE_HI)


@dataclass
class Env:
    basis: str
    K32: np.ndarray           # binary32-rounded operator, float64
    spec: osafe.SafetySpec
    lo: np.ndarray
    hi: np.ndarray
    track: np.ndarray | None


def bot_env(seed: int = 1, m: int = 5000, inflation: float = 0.0) -> Env:
    x, u, xn = data.transitions("bot", seed, m)
    K = ofit.round_to_f32(ofit.fit_koopman("bot", x, u, xn)[0])
    spec = osafe.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI, inflation=inflation)
    return Env("bot", K, spec, plants.BOT_INPUT_LO, plants.BOT_INPUT_HI, None)


def car_env(seed: int = 3, m: int = 20000, track_seed: int = 3,
            inflation: float = 0.0) -> Env:
    x, u, xn = data.transitions("car", seed, m)
    K = ofit.round_to_f32(ofit.fit_koopman("car", x, u, xn)[0])
    track = data.track_polyline(track_seed)
    spec = osafe.SafetySpec(lo=data.CAR_SAFE_LO, hi=data.CAR_SAFE_HI, track=track,
                            half_width=data.CAR_TRACK_HALF_WIDTH, inflation=inflation)
    return Env("car", K, spec, plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, track)


def gpu_model(lib, ctx, env: Env):
    m = lib.model_from_operator(ctx, env.basis, env.K32)
    lib.set_safety_set(m, env.spec.lo, env.spec.hi, env.spec.inflation, env.track,
                       env.spec.half_width)
    return m


def run_gpu(lib, sess, x_t, u_h, tick=0, traj=False, candidates=None):
    import torch
    dev = torch.device("cuda")
    x = torch.tensor(np.asarray(x_t, float), dtype=torch.float64, device=dev)
    u = torch.tensor(np.asarray(u_h, float), dtype=torch.float64, device=dev)
    res = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    ttv = torch.full((sess.n_slots,), -1, dtype=torch.int32, device=dev)
    cost = torch.full((sess.n_slots,), float("nan"), dtype=torch.float32, device=dev)
    tr = None
    if traj:
        tr = torch.full((sess.n_slots, sess.horizon + 1, sess.n), float("nan"),
                        dtype=torch.float32, device=dev)
        lib.debug_trajectories(sess, x, u, res, tr, candidates=candidates, tick=tick,
                               ttv_dev=ttv, cost_dev=cost)
    else:
        lib.evaluate_candidates_device(sess, x, u, res, candidates=candidates, tick=tick,
                                       ttv_dev=ttv, cost_dev=cost)
    torch.cuda.synchronize()
    out = dict(result=lib.result_from_bytes(res.cpu(), sess.nu),
               ttv=ttv.cpu().numpy().astype(np.int64), cost=cost.cpu().numpy())
    out["traj"] = None if tr is None else tr.cpu().numpy().astype(np.float64)
    return out


def oracle_samples(env: Env, n, seed, stream, tick, sampler="uniform"):
    if sampler == "grid":
        return osamp.grid_samples(n, env.lo, env.hi)
    return osamp.uniform_samples(seed, stream, tick, n, env.lo, env.hi)


def compare(g, o: omp.TickResult, env: Env, H: int, include_user: bool = True):
    """Assert the GPU tick g (run_gpu output) against the oracle tick o; return
    the number of boundary-excused candidates."""
    n_slots = len(o.ttv)
    tg, to = g["ttv"], o.ttv
    assert tg.shape == to.shape and np.all(tg >= 0) and np.all(tg <= H)
    # trajectories, at every step both sides computed
    err_at = None
    if g["traj"] is not None and o.traj is not None:
        zg, zo = g["traj"], o.traj
        steps = np.minimum(np.minimum(tg, to) + 1, H)
        t_idx = np.arange(H + 1)[None, :]
        mask = t_idx <= steps[:, None]
        diff = np.abs(zg - zo).max(axis=2)
        scale = np.maximum(np.abs(zo).max(axis=2), 1.0)
        rel = np.where(mask, diff / scale, 0.0)
        worst = np.nanmax(rel)
        assert np.all(np.isfinite(rel[mask])), "NaN in a computed step"
        assert worst <= TRAJ_RTOL, f"trajectory error {worst:.3g} > {TRAJ_RTOL}"
        err_at = diff
    # time to violation: disagreements only at a boundary
    excused = np.nonzero(tg != to)[0]
    for i in excused:
        s = int(min(tg[i], to[i])) + 1
        zref = o.traj[i, s] if o.traj is not None else None
        assert zref is not None, "ttv mismatch without trajectories to judge it"
        marg = float(osafe.margin(env.spec, zref[None, :])[0])
        scale = max(1.0, float(np.abs(zref).max()))
        err = float(err_at[i, s]) if err_at is not None and np.isfinite(err_at[i, s]) \
            else TRAJ_RTOL * scale
        assert abs(marg) <= err + BOUNDARY_TOL * scale, (
            f"slot {i}: ttv gpu {tg[i]} oracle {to[i]} with margin {marg:.3g} "
            f"(err {err:.3g}) at step {s}")
    # costs
    assert np.allclose(g["cost"], o.cost, rtol=COST_RTOL, atol=1e-12)
    # the GPU's pick is the lexicographic minimum of its own per-candidate outputs
    slots = np.arange(n_slots)
    order = np.lexsort((slots, g["cost"].astype(np.float64), H - tg))
    r = g["result"]
    assert r["index"] == int(order[0])
    assert r["status"] == (omp.SAFE if tg[r["index"]] == H else omp.FALLBACK)
    assert r["ttv"] == tg[r["index"]]
    assert r["n_safe"] == int(np.count_nonzero(tg == H))
    assert r["executed_steps"] == int(np.minimum(tg + 1, H).sum())
    assert r["n_slots"] == n_slots
    # u_r is the picked candidate's value (u_h itself for slot 0)
    assert np.array_equal(r["u_r"], o.candidates[r["index"]]) or (
        include_user and r["index"] == 0)
    # selection against the oracle
    gi, oi = r["index"], o.index
    if gi != oi:
        tie = (H - to[gi] == H - to[oi]) and abs(o.cost[gi] - o.cost[oi]) <= \
            TIE_RTOL * max(o.cost[gi], o.cost[oi]) + 1e-12
        boundary = tg[gi] != to[gi] or tg[oi] != to[oi]
        assert tie or boundary, f"selection gpu {gi} oracle {oi} not excused"
    return len(excused)
