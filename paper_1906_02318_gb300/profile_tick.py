"""Runs a fixed number of device-resident MPMI-SC ticks for profiling (ncu).

python -m paper_1906_02318_gb300.profile_tick --basis bot --n 16384 --horizon 50 --ticks 20

--mode plain (default): each tick is exactly one launch of the fused tick
kernel; nothing else runs on the GPU after set-up except an optional L2 flush
(one memset) before each tick.  Prints the mean CUDA-event duration and the
executed steps.
--mode screened (race car): each tick is one screened tick (score, compaction,
exact rollout of the kept slots, fallback) with an untrained screener and the
given --tau / --k.
--mode serve: --ticks batches of --sessions requests (N log-uniform 1k..64k, H
20..100) through one continuous-batching server of the chosen model, one batch
at a time (host wall time from launch to collected result).
--rollout factored: plain ticks in the factorised read-out form (one launch of
the factorised kernel per tick after the one-off powers of K).
--noise s1,s2,..: Alg. 2's per-step noise with these standard deviations on the
first state coordinates.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    from paper_1906_02318_gb300 import build, mpmi as lib
    from workloads import data, plants

    ap = argparse.ArgumentParser()
    ap.add_argument("--basis", choices=["bot", "car"], default="bot")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--horizon", type=int, default=50)
    ap.add_argument("--ticks", type=int, default=20)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--cands", type=int, default=0, help="candidates per thread (one lane)")
    ap.add_argument("--flush", action="store_true", help="write 256 MB before each tick")
    ap.add_argument("--mode", choices=["plain", "screened", "serve"], default="plain")
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--tau", type=float, default=0.0)
    ap.add_argument("--m", type=int, default=8, help="predicted-safe slots the prefix holds")
    ap.add_argument("--sessions", type=int, default=64)
    ap.add_argument("--rollout", choices=["full", "factored", "tensor"], default="full")
    ap.add_argument("--noise", default="", help="comma-separated sigma per state coordinate")
    args = ap.parse_args()

    build.build()
    ctx = lib.Context(0)
    if args.basis == "bot":
        x, u, xn = data.transitions("bot", 1, 5000)
        model, _ = lib.fit_model(ctx, "bot", x, u, xn)
        lib.set_safety_set(model, data.BOT_SAFE_LO, data.BOT_SAFE_HI)
        lo, hi = plants.BOT_INPUT_LO, plants.BOT_INPUT_HI
        states = data.states_in_box(2, args.ticks, [-0.1, -0.5, -0.5, -0.5], [0.1, 0.5, 0.5, 0.5])
    else:
        x, u, xn = data.transitions("car", 3, 20000)
        model, _ = lib.fit_model(ctx, "car", x, u, xn)
        track = data.track_polyline(3)
        lib.set_safety_set(model, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.0, track,
                           data.CAR_TRACK_HALF_WIDTH)
        lo, hi = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI
        x0 = data.car_start_state(track, vx=12.0)
        jit = data.states_in_box(3, args.ticks, [-1, -1, -0.05, -2, -0.2, -0.1],
                                 [1, 1, 0.05, 2, 0.2, 0.1])
        states = x0[None, :] + jit
    uhs = data.ou_user_input(2, args.ticks, 0.01, lo, hi)
    if args.mode == "serve":
        return serve_mode(args, ctx, model, lo, hi, states, uhs)
    sess = lib.Session(ctx, model, args.n, args.horizon, lo, hi, seed=2, lanes=args.lanes,
                       block=args.block, cands=args.cands)
    if args.rollout != "full":
        sess.set_rollout(args.rollout)
    if args.noise:
        sess.set_noise([float(v) for v in args.noise.split(",")])
    scr = None
    if args.mode == "screened":
        if args.basis != "car":
            raise SystemExit("--mode screened needs --basis car")
        scr = lib.Screener(ctx, model, data.screener_init(5), max_batch=256,
                           max_slots=args.n + 1)
    dev = torch.device("cuda")
    xs = torch.tensor(states, dtype=torch.float64, device=dev)
    us = torch.tensor(uhs, dtype=torch.float64, device=dev)
    res = torch.zeros((args.ticks, lib.RESULT_BYTES), dtype=torch.uint8, device=dev)
    flush = torch.empty((64 << 20,), dtype=torch.float32, device=dev) if args.flush else None
    st = torch.cuda.current_stream()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.ticks)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.ticks)]
    for t in range(args.ticks):
        if flush is not None:
            flush.zero_()
        e0[t].record(st)
        if args.mode == "screened":
            lib.evaluate_screened(sess, scr, xs[t], us[t], res[t], k=args.k, tau=args.tau,
                                  m=args.m, tick=t, stream=st)
        else:
            lib.evaluate_candidates_device(sess, xs[t], us[t], res[t], tick=t, stream=st)
        e1[t].record(st)
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in zip(e0, e1)])
    ex = [lib.result_from_bytes(r, sess.nu)["executed_steps"] for r in res.cpu().numpy()]
    lanes, cands, block = sess.launch_shape()
    n = 12 if args.basis == "bot" else 32
    fl = np.mean(ex) * 2 * n * n
    print(f"{args.basis} N={args.n} H={args.horizon} lanes={lanes} cands={cands} block={block} "
          f"ticks={args.ticks} mean_us={ms[1:].mean() * 1e3 if len(ms) > 1 else ms[0] * 1e3:.2f} "
          f"min_us={ms.min() * 1e3:.2f} executed={np.mean(ex):.0f} "
          f"nominal={(args.n + 1) * args.horizon} "
          f"tflops={fl / (ms[1:].mean() * 1e-3 if len(ms) > 1 else ms[0] * 1e-3) / 1e12:.2f}")
    sess.close()
    if scr is not None:
        scr.free()
    model.free()


def serve_mode(args, ctx, model, lo, hi, states, uhs):
    import torch

    from paper_1906_02318_gb300 import mpmi as lib
    srv = lib.Server(ctx, model, args.sessions)
    rng = np.random.default_rng(4)
    ns = np.exp(rng.uniform(np.log(1024), np.log(65536), args.sessions)).astype(int)
    hs = rng.integers(20, 101, args.sessions)
    slots = [srv.admit(int(n), int(h), lo, hi, seed=i, stream_id=i)
             for i, (n, h) in enumerate(zip(ns, hs))]
    import time
    st = torch.cuda.current_stream()
    ms = []
    for t in range(args.ticks):
        idx = [i % len(states) for i in range(args.sessions)]
        srv.submit(slots, states[idx], np.repeat(uhs[t:t + 1], args.sessions, axis=0),
                   [t] * args.sessions)
        # the batch runs on the server's own stream: time launch to collected result
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        srv.launch(st)
        srv.collect()
        ms.append((time.perf_counter() - t0) * 1e3)
    steps = float(np.sum((ns + 1) * hs))
    t = np.mean(ms[1:]) * 1e-3 if len(ms) > 1 else ms[0] * 1e-3
    print(f"serve {args.basis} sessions={args.sessions} batches={args.ticks} "
          f"mean_us={t * 1e6:.1f} steps_per_batch={steps:.0f} steps_per_s={steps / t:.3e}")
    srv.free()
    model.free()


if __name__ == "__main__":
    main()
