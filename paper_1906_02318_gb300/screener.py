"""Training and evaluation driver of the learned candidate screener.

Labels come from the plain method itself: a race-car closed loop driven by the
exact tick (mpmi_evaluate_candidates_device, which also returns every slot's
time to violation), with the user's input from an Ornstein-Uhlenbeck process and
a new trial whenever the car leaves the safe set.  Each label is (the 12 network
inputs of a slot, ttv / H).  Training runs the library's own forward, backward
and Adam kernels; evaluation compares the screened tick with the exhaustive one.
Every computation runs in libmpmi; this module moves tensors and loops.
"""
from __future__ import annotations

import numpy as np

from . import mpmi as lib


def car_in_safe_set(x: np.ndarray, track: np.ndarray, half_width: float, vx_max: float) -> bool:
    """Whether a simulated race-car state is still in the safe set (on the road and
    below vx_max); leaving it ends a trial (Sec. V-B).  A plant-side check of the
    closed loops, not part of a tick."""
    if not np.all(np.isfinite(x)) or x[3] >= vx_max:
        return False
    d = np.roll(track, -1, axis=0) - track
    r = x[:2] - track
    t = np.clip(np.sum(r * d, axis=1) / np.sum(d * d, axis=1), 0.0, 1.0)
    dist = np.linalg.norm(r - t[:, None] * d, axis=1)
    return float(dist.min()) < half_width


def collect_labels(session, screener, plant_step, x0, user_inputs, track, half_width,
                   vx_max=25.0, tick0=0):
    """Runs the closed loop for len(user_inputs) ticks; returns (features, targets,
    states) with features (ticks * n_slots, 12) and targets ttv / H on the device."""
    import torch
    dev = torch.device("cuda")
    T, n = len(user_inputs), session.n_slots
    feats = torch.empty((T, n, 12), dtype=torch.float32, device=dev)
    ttv = torch.empty((T, n), dtype=torch.int32, device=dev)
    res = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    xs = np.empty((T, 6))
    x = np.asarray(x0, dtype=np.float64).copy()
    for t in range(T):
        xs[t] = x
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        ud = torch.tensor(user_inputs[t], dtype=torch.float64, device=dev)
        screener.features(session, xd, ud, feats[t], tick=tick0 + t)
        lib.evaluate_candidates_device(session, xd, ud, res, tick=tick0 + t, ttv_dev=ttv[t])
        r = lib.result_from_bytes(res.cpu(), 2)
        x = plant_step(x, r["u_r"])
        if not car_in_safe_set(x, track, half_width, vx_max):
            x = np.asarray(x0, dtype=np.float64).copy()
    targets = (ttv.to(torch.float32) / float(session.horizon)).reshape(-1)
    return feats.reshape(-1, 12), targets, xs


def train(screener, feats, targets, epochs=3, batch=8192, lr=2e-3, seed=0):
    """Minibatch Adam over shuffled labels; returns the per-epoch mean losses."""
    import torch
    g = torch.Generator(device=feats.device)
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=feats.device)
    out = []
    n = feats.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, device=feats.device, generator=g)
        total, steps = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            f = feats.index_select(0, idx).contiguous()
            y = targets.index_select(0, idx).contiguous()
            screener.train_step(f, y, loss, lr=lr)
            total += float(loss.item())
            steps += 1
        out.append(total / max(steps, 1))
    return out


def compare(session, screener, states, user_inputs, k=4096, tau=0.9, m=8, tick0=0):
    """Screened vs exhaustive tick on each (state, user input): returns a dict with
    the agreement (same selected slot), the number of reported-safe picks that the
    exhaustive evaluation finds unsafe (safety misses), the fallback count, the
    mean number of kept slots and the mean rollout steps each form executed."""
    import torch
    dev = torch.device("cuda")
    n = session.n_slots
    r_plain = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    r_scr = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    ttv = torch.empty(n, dtype=torch.int32, device=dev)
    nl = torch.zeros(1, dtype=torch.int32, device=dev)
    agree = misses = fallbacks = 0
    kept, steps, plain_steps = [], [], []
    for t, (x, u) in enumerate(zip(states, user_inputs)):
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        ud = torch.tensor(u, dtype=torch.float64, device=dev)
        lib.evaluate_candidates_device(session, xd, ud, r_plain, tick=tick0 + t, ttv_dev=ttv)
        lib.evaluate_screened(session, screener, xd, ud, r_scr, k=k, tau=tau, m=m,
                              tick=tick0 + t, n_list_dev=nl)
        a = lib.result_from_bytes(r_plain.cpu(), 2)
        b = lib.result_from_bytes(r_scr.cpu(), 2)
        full = ttv.cpu().numpy()
        agree += a["index"] == b["index"]
        if b["status"] == lib.SAFE and full[b["index"]] != session.horizon:
            misses += 1
        fallbacks += (b["flags"] & 2) != 0
        kept.append(int(nl.item()))
        steps.append(b["executed_steps"])
        plain_steps.append(a["executed_steps"])
    T = len(states)
    return dict(ticks=T, agreement=agree / T, safety_misses=misses, fallbacks=fallbacks,
                mean_kept=float(np.mean(kept)), mean_executed_steps=float(np.mean(steps)),
                plain_executed_steps=float(np.mean(plain_steps)))


def calibrate(session, screener, states, user_inputs, taus=(0.5, 0.8, 0.9, 0.95),
              ms=(1, 4, 16), k=1, tick0=0):
    """Picks the screen's threshold tau and predicted-safe count m on held-out
    calibration ticks: the pair with the fewest mean executed rollout steps (every
    pair selects exactly, so only the work differs).  Returns the pair and the
    table of means."""
    table = {}
    for tau in taus:
        for m in ms:
            r = compare(session, screener, states, user_inputs, k=k, tau=tau, m=m, tick0=tick0)
            table[(tau, m)] = r["mean_executed_steps"]
    tau, m = min(table, key=lambda key: (table[key], -key[0], key[1]))
    return dict(tau=tau, m=m, k=k,
                table={f"tau={a},m={b}": v for (a, b), v in table.items()})
