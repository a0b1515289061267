"""Runs a fixed number of device-resident MPMI-SC ticks for profiling (ncu).

python -m paper_1906_02318_gb300.profile_tick --basis bot --n 16384 --horizon 50 --ticks 20

Each tick is exactly one launch of the fused tick kernel; nothing else runs on
the GPU after set-up except an optional L2 flush (one memset) before each tick.
Prints the mean CUDA-event duration of the tick kernel and the executed steps.
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
    sess = lib.Session(ctx, model, args.n, args.horizon, lo, hi, seed=2, lanes=args.lanes,
                       block=args.block, cands=args.cands)
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
    model.free()


if __name__ == "__main__":
    main()
