"""Benchmark: MPMI-SC control ticks on one GB300 (or N replicas under torchrun).

Workload (the configuration the headline metric is quoted on): balance-bot
closed loop at paper scale -- model fit on 5000 seeded cart-pole transitions
(12 lifted features), N = 16384 sampled candidates (+ the user's input), H = 50
prediction steps, 100 Hz, 1000 ticks, user input from a seeded Ornstein-Uhlenbeck
process (theta = 1.0, sigma = 0.5) clipped to [-1, 1].

One "step" is one control tick: sample, lift, predict with early exit, safety
test, cost, device-wide argmin and decode (every row of the hot path).

  value        rollout steps/s = (N + 1) * H per tick / device time per tick, with
               the tick inputs resident in HBM (device-side API), L2 flushed
               (256 MB write) before every timed tick, CUDA events on the launch
               stream around each tick.
  e2e          the same metric through the host C-ABI call (evaluate_candidates +
               select_input) driving the closed loop, with persistent host ticks
               (a resident kernel reads x_t/u_h from a pinned mailbox and writes the
               result to pinned memory, every tick); e2e_launched: the same loop
               with one kernel launch per tick.  Both loops must visit the same
               states (persistent_loop_identical).
  roofline     FP32 CUDA-core (ALU) bound: algorithmic flops per tick (2 n^2 per
               executed prediction step + lifting + cost) / mean tick duration,
               against 152 SMs x 128 FP32 lanes x 2 flops x max SM clock.
  cpu_baseline the FP64 oracle on the host cores (spawned worker processes), on
               a bounded sample of the same ticks.
  roofline_over_n  the same plain tick (bot H = 50, race car H = 60) at N = 16384
               .. 1048576, one session each: the fraction of the FP32 peak as the
               candidates fill the GPU.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import data, plants  # noqa: E402
from paper_1906_02318_gb300 import metrics  # noqa: E402

# ---- workload constants -----------------------------------------------------
N_SAMPLES = 16384
HORIZON = 50
TICKS = 1000
FIT_SEED, FIT_COUNT = 1, 5000
LOOP_SEED = 2
X0 = np.array([0.05, 0.0, 0.0, 0.0])
CAR_SEED, CAR_TRACK_SEED, CAR_FIT_COUNT = 3, 3, 20000
CAR_ORACLE_N = 4096  # candidates per oracle tick in the race car's CPU sample
LIFTED_N = 12
FLUSH_BYTES = 256 << 20
SM_FP32_LANES = 128

# The paper's own throughput figures (its System Performance subsection; its only
# hardware is a GeForce 860M laptop GPU), quoted beside the measurements as context:
# another machine and other workloads, not a target.  The rollout-step rates are
# derived here from its loop rates, sample counts and horizons.
PAPER_CONTEXT = {
    "hardware": "GeForce 860M",
    "trajectories_per_tick": ">10,000 (balance bot N = 10,000, T = 30; race car N = 10,120, "
                             "T = 25)",
    "control_rate_hz": {"balance_bot": 100, "race_car": 60},
    "trajectories_per_s": "600,000-1,000,000 with the safety checks",
    "derived_rollout_steps_per_s": {"balance_bot": 100 * 10000 * 30, "race_car": 60 * 10120 * 25},
    "note": "context only, not comparable: other hardware and workloads",
}

# DRAM bytes per tick-kernel launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum); valid only for the kernel source and launch shape
# (lanes, candidates per thread, block) it was taken on.
TRAFFIC = {"tick_kernel_sha1": "97d5b009fbabb862887c3ebbe6a7ebfe623f6776",
           "bytes_per_launch": {(1, 1, 128): 26880, (1, 1, 64): 26624}}


def kernel_sha1() -> str:
    p = os.path.join(ROOT, "paper_1906_02318_gb300", "csrc", "tick_kernel.cuh")
    return hashlib.sha1(open(p, "rb").read()).hexdigest()


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


# ---- clocks during the timed region ----------------------------------------
class NvmlClocks:
    """Polls the SM clock and the clock-event reasons through NVML (read-only)
    every ~2 ms from a background thread."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str):
        import ctypes
        self.ct = ctypes
        self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByUUID failed")
        self.samples: list[tuple[int, int]] = []
        self.stop_flag = False
        self.thread = None

    def _one(self):
        c = self.ct.c_uint()
        r = self.ct.c_ulonglong()
        self.nv.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c))
        fn = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self.h, self.ct.byref(r))
        return c.value, r.value

    def _loop(self):
        while not self.stop_flag:
            self.samples.append(self._one())
            time.sleep(0.002)

    def start(self):
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def stop(self) -> dict | None:
        self.stop_flag = True
        if self.thread:
            self.thread.join(timeout=2)
        m = self.ct.c_uint()
        self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(m))
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median([c for c, _ in self.samples]),
                "sm_max_mhz": m.value, "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "nvml"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- oracle leg (host cores) -----------------------------------------------
def _oracle_worker(args):
    """Spawned worker: oracle ticks over the given tick indices until the time
    budget runs out.  Returns (rollout steps, seconds)."""
    (basis, K32, ticks, states, uhs, n, H, budget) = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from oracle import mpmi as omp
    from oracle import safety as osafe
    from oracle import sampling as osamp
    if basis == "bot":
        spec = osafe.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
        lo, hi, seed = plants.BOT_INPUT_LO, plants.BOT_INPUT_HI, LOOP_SEED
    else:
        spec = osafe.SafetySpec(lo=data.CAR_SAFE_LO, hi=data.CAR_SAFE_HI,
                                track=data.track_polyline(CAR_TRACK_SEED),
                                half_width=data.CAR_TRACK_HALF_WIDTH)
        lo, hi, seed = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, CAR_SEED
    steps = 0
    t0 = time.perf_counter()
    for t in ticks:
        s = osamp.uniform_samples(seed, 0, int(t), n, lo, hi)
        omp.tick(K32, basis, states[t], uhs[t], s, H, spec)
        steps += (n + 1) * H
        if time.perf_counter() - t0 > budget:
            break
    return steps, time.perf_counter() - t0


def oracle_rate(K32, states, uhs, n, H, budget_s, workers, tick_ids, basis="bot"):
    """Rollout steps/s of the oracle on `workers` spawned processes."""
    import multiprocessing as mp
    chunks = [tick_ids[w::workers] for w in range(workers)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        outs = pool.map(_oracle_worker,
                        [(basis, K32, c, states, uhs, n, H, budget_s) for c in chunks if len(c)])
    steps = sum(s for s, _ in outs)
    t_max = max(t for _, t in outs)
    oracle_rate.per_core = float(np.mean([s / t for s, t in outs if t > 0]))
    return steps / t_max, steps, t_max


def oracle_model():
    from oracle import fit as ofit
    x, u, xn = data.transitions("bot", FIT_SEED, FIT_COUNT)
    return ofit.round_to_f32(ofit.fit_koopman("bot", x, u, xn)[0])


def reference_states():
    """Tick inputs for the oracle legs: the oracle's own closed loop is too slow to
    run 1000 ticks, so it replays the user input stream from a fixed set of states
    drawn near the upright equilibrium."""
    uhs = data.to_f32_exact(data.ou_user_input(LOOP_SEED, TICKS, plants.BOT_DT,
                                               plants.BOT_INPUT_LO, plants.BOT_INPUT_HI))
    states = data.states_in_box(LOOP_SEED, TICKS, [-0.1, -0.5, -0.5, -0.5],
                                [0.1, 0.5, 0.5, 0.5])
    return states, uhs


# ---- GPU leg ----------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    from paper_1906_02318_gb300 import build as pbuild
    from paper_1906_02318_gb300 import mpmi as lib

    pbuild.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    ctx = lib.Context(dev.index)
    x, u, xn = data.transitions("bot", FIT_SEED, FIT_COUNT)
    model, residual = lib.fit_model(ctx, "bot", x, u, xn)
    lib.set_safety_set(model, data.BOT_SAFE_LO, data.BOT_SAFE_HI)
    seed = LOOP_SEED + 1000 * rank
    ticks = max(TICKS, args.warmup + args.steps)
    uhs = data.ou_user_input(seed, ticks, plants.BOT_DT, plants.BOT_INPUT_LO,
                             plants.BOT_INPUT_HI)
    # the library's autotuner picks the launch shape for this configuration (any
    # shape gives bit-identical results); the session below takes its choice
    tuned = lib.tune_launch_shape(ctx, model, N_SAMPLES, HORIZON, plants.BOT_INPUT_LO,
                                  plants.BOT_INPUT_HI, X0, uhs[0], reps=30, seed=seed,
                                  stream_id=rank)
    sess = lib.Session(ctx, model, N_SAMPLES, HORIZON, plants.BOT_INPUT_LO,
                       plants.BOT_INPUT_HI, seed=seed, stream_id=rank)
    lanes, cands, block = sess.launch_shape()
    n_slots = sess.n_slots
    stream = torch.cuda.current_stream(dev)
    gpu_id = None
    try:
        gpu_id = f"GPU-{props.uuid}"
    except Exception:
        pass

    # closed loop through the host C-ABI (e2e): W warm-up ticks, then timed ticks.
    # As in the paper's trials, a trial ends when the plant leaves the safe set
    # and the next one starts from x_0.
    def closed_loop(recs=None):
        x_t = X0.copy()
        states = np.empty((ticks, 4))
        lat = []
        n_fallback = 0
        trials = 1
        for t in range(ticks):
            states[t] = x_t
            t0 = time.perf_counter()
            lib.evaluate_candidates(sess, x_t, uhs[t], tick=t, stream=stream)
            r = lib.select_input(sess)
            dt = time.perf_counter() - t0
            if t >= args.warmup:
                lat.append(dt)
            n_fallback += r["status"] == lib.FALLBACK
            x_t = plants.cartpole_step(x_t, r["u_r"])
            inside = np.all(np.isfinite(x_t)) and np.all(x_t > data.BOT_SAFE_LO) and \
                np.all(x_t < data.BOT_SAFE_HI)
            if recs is not None and t >= args.warmup:
                recs.append(metrics.tick_record(r, uhs[t], t, trials - 1, N_SAMPLES,
                                                latency_s=dt, failed=not inside))
            if not inside:
                x_t = X0.copy()
                trials += 1
        return states, np.array(lat), n_fallback, trials

    # launched host ticks (one kernel launch per tick, zero-copy inputs/result)
    recs_launched, recs_persist = [], []
    states, lat_launched, n_fallback, trials = closed_loop(recs_launched)
    # the same loop with persistent host ticks (a resident kernel fed through a
    # pinned mailbox); it must retrace the launched loop's states exactly
    lat_persist, persist_note, persist_same = None, "launched host ticks requested", None
    if not args.launched_host_ticks:
        try:
            sess.set_persistent(True)
        except lib.MpmiError as e:
            persist_note = f"persistent host ticks unavailable: {e}"
        else:
            states_p, lat_persist, _, _ = closed_loop(recs_persist)
            sess.set_persistent(False)
            persist_same = bool(np.array_equal(states_p, states))
    lat = lat_persist if lat_persist is not None else lat_launched
    e2e_rate = n_slots * HORIZON * len(lat) / lat.sum()
    # the paper's run metrics (Sec. VI, Table I) over the timed closed loop
    paper_metrics = metrics.summarize(recs_persist if lat_persist is not None else recs_launched,
                                      plants.BOT_DT)
    paper_metrics["eq2_bound"] = 2.0 / (2 * N_SAMPLES)  # lambda*(U) / (2N), 1-D input box

    # device-resident ticks: inputs in HBM, L2 flushed before each timed tick
    xs = torch.tensor(states, dtype=torch.float64, device=dev)
    us = torch.tensor(uhs, dtype=torch.float64, device=dev)
    results = torch.zeros((ticks, lib.RESULT_BYTES), dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    n_ev = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]

    def tick(i):
        lib.evaluate_candidates_device(sess, xs[i % ticks], us[i % ticks], results[i % ticks],
                                       tick=i % ticks, stream=stream)

    for i in range(args.warmup):
        flush.zero_()
        tick(i)
    torch.cuda.synchronize()
    try:
        clocks = NvmlClocks(gpu_id)
    except Exception:
        clocks = ClockSampler(gpu_id)
    clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(n_ev):
        i = args.warmup + k
        flush.zero_()
        ev0[k].record(stream)
        tick(i)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    durs = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)]) * 1e-3
    # the device's FP32 FMA rate measured by the library's own FMA loop (context
    # for the roofline, whose peak is the nominal unit count x maximum clock)
    ffma_tflops = lib.measure_fp32_peak(dev.index, 0.5)
    dev_time = float(durs.sum())
    res = results.cpu().numpy()
    executed = []
    agree = 0
    for k in range(n_ev):
        i = (args.warmup + k) % ticks
        rr = lib.result_from_bytes(res[i], 1)
        executed.append(rr["executed_steps"])
    executed = np.array(executed, dtype=np.float64)
    # the device path reproduces the closed loop's selections on the same ticks
    for i in range(min(ticks, 200)):
        rr = lib.result_from_bytes(res[i], 1)
        agree += rr["tick"] == i
    sess.close()
    model.free()
    return dict(dev_time=dev_time, durs=durs, executed=executed, lat=lat, e2e_rate=e2e_rate,
                lat_launched=lat_launched, persistent=lat_persist is not None,
                persist_note=persist_note, persist_same=persist_same,
                wall=wall, clocks=clk, lanes=lanes, cands=cands, block=block, n_slots=n_slots,
                residual=residual, n_fallback=int(n_fallback), trials=trials, states=states,
                paper_metrics=paper_metrics,
                ffma_tflops=ffma_tflops, tuned=tuned,
                sm_count=props.multi_processor_count,
                gpu_name=props.name)


SCREEN_FLOPS_PER_SLOT = 2 * 12 * 128 + 2 * 128 * 128  # the two tensor-core layers
CAR_LIFTED_N = 32


def run_learned(args):
    """Learned screener vs plain exhaustive evaluation on the race car (N = 16384 and
    65536, H = 60): a screener trained on ~2M labels from the plain path's own
    closed-loop rollouts; its threshold tau and predicted-safe count m calibrated
    on held-out ticks (fewest executed steps), then agreement, safety misses,
    executed steps, tick times and per-kernel rooflines on other held-out ticks.
    Also reports the exact cost-ordered search (tau = 0, fixed k = N / 16, no
    network), the method without the learned part.  Every screened form selects
    exactly what the exhaustive evaluation selects."""
    import torch
    from paper_1906_02318_gb300 import mpmi as lib
    from paper_1906_02318_gb300 import screener as drv
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * SM_FP32_LANES * 2 * sm_max * 1e6 / 1e12
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    ctx = lib.Context(dev.index)
    x, u, xn = data.transitions("car", CAR_SEED, CAR_FIT_COUNT)
    model, _ = lib.fit_model(ctx, "car", x, u, xn)
    track = data.track_polyline(CAR_TRACK_SEED)
    lib.set_safety_set(model, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.0, track,
                       data.CAR_TRACK_HALF_WIDTH)
    lo, hi = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI
    x0 = data.car_start_state(track, vx=12.0)
    scr = lib.Screener(ctx, model, data.screener_init(5), max_batch=8192, max_slots=65537)
    t0 = time.perf_counter()
    sess = lib.Session(ctx, model, 16384, 60, lo, hi, seed=5)
    feats, targets, _ = drv.collect_labels(sess, scr, plants.bicycle_step, x0,
                                           data.ou_user_input(5, 122, plants.CAR_DT, lo, hi),
                                           track, data.CAR_TRACK_HALF_WIDTH)
    sess.close()
    losses = drv.train(scr, feats, targets, epochs=6, batch=8192, lr=2e-3)
    train_s = time.perf_counter() - t0
    n_labels = int(feats.shape[0])
    del feats, targets

    def held_out(seed, ticks, tick0):
        s1 = lib.Session(ctx, model, 1023, 60, lo, hi, seed=6)
        uu = data.ou_user_input(seed, ticks, plants.CAR_DT, lo, hi)
        _, _, xx = drv.collect_labels(s1, scr, plants.bicycle_step, x0, uu, track,
                                      data.CAR_TRACK_HALF_WIDTH, tick0=tick0)
        s1.close()
        return xx, uu

    ticks = args.learned_ticks
    xev, uev = held_out(6, ticks, 10000)
    xcal, ucal = held_out(8, 100, 20000)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    res = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    out = {"workload": "race car, H=60, held-out closed-loop states", "labels": n_labels,
           "train_epochs": len(losses), "train_loss": losses[-1], "train_s": train_s,
           "ticks": ticks, "calibration_ticks": len(xcal), "runs": [],
           "what": "every form selects exactly the exhaustive evaluation's slot; the learned "
                   "form rolls out the cost-order prefix holding m predicted-safe slots",
           "rates": "executed = rollout steps actually run / tick time; "
                    "nominal_equivalent = (N + 1) * H / tick time, the rate of the exhaustive "
                    "evaluation the tick replaces"}
    for N in (16384, 65536):
        sess = lib.Session(ctx, model, N, 60, lo, hi, seed=7)
        k = N // 16
        cal = drv.calibrate(sess, scr, xcal, ucal, taus=(0.8, 0.9, 0.95, 0.98, 0.99),
                            ms=(16, 64, 256, 1024), k=1, tick0=50000)

        def timed(fn):
            ts = []
            for t in range(ticks):
                xd = torch.tensor(xev[t], dtype=torch.float64, device=dev)
                ud = torch.tensor(uev[t], dtype=torch.float64, device=dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                e0.record()
                fn(xd, ud, 40000 + t)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
            return np.array(ts)

        def phases(k_, tau_, m_):
            """Per-launch CUDA-event durations of the screened ticks (a separate pass)."""
            scr.set_timing(True)
            acc = {"screen": [], "compact": [], "rollout": [], "fallback": []}
            for t in range(ticks):
                xd = torch.tensor(xev[t], dtype=torch.float64, device=dev)
                ud = torch.tensor(uev[t], dtype=torch.float64, device=dev)
                flush.zero_()
                lib.evaluate_screened(sess, scr, xd, ud, res, k=k_, tau=tau_, m=m_,
                                      tick=40000 + t)
                for key, v in scr.phase_times().items():
                    acc[key].append(v * 1e-3)
            scr.set_timing(False)
            return {key: float(np.mean(v)) for key, v in acc.items()}

        tp = timed(lambda xd, ud, t: lib.evaluate_candidates_device(sess, xd, ud, res, tick=t))
        st_plain = drv.compare(sess, scr, xev, uev, k=N + 1, tau=0.0, tick0=40000)
        ex_plain = st_plain["plain_executed_steps"]
        run = {"N": N, "k_cost_ordered": k, "calibration": cal,
               "plain": {"mean_us": tp.mean() * 1e6, "p99_us": np.percentile(tp, 99) * 1e6,
                         "executed_steps_per_tick": ex_plain,
                         "executed_steps_per_s": ex_plain / tp.mean(),
                         "nominal_equivalent_steps_per_s": (N + 1) * 60 / tp.mean(),
                         "roofline": {"kernel": "tick_kernel (full rollout)", "bound": "alu",
                                      "achieved": ex_plain * 2 * CAR_LIFTED_N ** 2
                                      / tp.mean() / 1e12,
                                      "peak": fp32_peak, "unit": "TFLOP/s"}}}
        run["plain"]["roofline"]["frac"] = run["plain"]["roofline"]["achieved"] / fp32_peak
        for name, kk, tau, m in (("cost_ordered", k, 0.0, 1),
                                 ("learned", 1, cal["tau"], cal["m"])):
            st = drv.compare(sess, scr, xev, uev, k=kk, tau=tau, m=m, tick0=40000)
            ts = timed(lambda xd, ud, t: lib.evaluate_screened(sess, scr, xd, ud, res, k=kk,
                                                               tau=tau, m=m, tick=t))
            ph = phases(kk, tau, m)
            ex = st["mean_executed_steps"]
            roll = {"kernel": "tick_kernel over the kept slots (and the fallback launch)",
                    "bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
                    "achieved": ex * 2 * CAR_LIFTED_N ** 2
                    / max(ph["rollout"] + ph["fallback"], 1e-9) / 1e12,
                    "mean_us": (ph["rollout"] + ph["fallback"]) * 1e6}
            roll["frac"] = roll["achieved"] / fp32_peak
            forms = {"rollout": roll}
            if tau > 0:
                scr_tf = (N + 1) * SCREEN_FLOPS_PER_SLOT / ph["screen"] / 1e12
                forms["screen_score"] = {"kernel": "screen_score (tcgen05, bf16 x bf16 -> f32)",
                                         "bound": "tensor", "unit": "TFLOP/s",
                                         "achieved": scr_tf, "peak": bf16_peak,
                                         "frac": scr_tf / bf16_peak,
                                         "mean_us": ph["screen"] * 1e6}
            else:
                forms["screen_cost"] = {"kernel": "screen_cost (costs and histogram)",
                                        "mean_us": ph["screen"] * 1e6}
            forms["compact_us"] = ph["compact"] * 1e6
            run[name] = dict(st, tau=tau, m=m, k=kk, mean_us=ts.mean() * 1e6,
                             p99_us=np.percentile(ts, 99) * 1e6,
                             executed_steps_per_tick=ex,
                             executed_steps_per_s=ex / ts.mean(),
                             nominal_equivalent_steps_per_s=(N + 1) * 60 / ts.mean(),
                             roofline=forms)
        run["host_ticks"] = host_screened(lib, sess, scr, k, cal, xev, uev)
        run["concurrent"] = concurrent_screened(lib, ctx, model, scr, N, k, cal, xev, uev, lo,
                                                hi)
        out["runs"].append(run)
        sess.close()
    scr.free()
    model.free()
    return out


def host_screened(lib, sess, scr, k, cal, xev, uev):
    """Host-to-host control-tick latency through the host C ABI on the same
    held-out states: the plain tick (mpmi_evaluate_candidates) and the two screened
    forms (mpmi_evaluate_screened_host), each collected with mpmi_select_input;
    wall clock around the two calls, one tick at a time, no cache flush; the same
    ticks (states, user inputs, candidate draws) as the device-timed forms."""
    import torch
    forms = {"plain": None, "cost_ordered": (k, 0.0, 1), "learned": (1, cal["tau"], cal["m"])}
    out = {"what": "host-to-host tick (evaluate + select_input), one launch chain per tick, "
                   "p50/p99 over the held-out ticks, 16.7 ms deadline (60 Hz)"}
    for name, form in forms.items():
        lat = []
        for t in range(len(xev)):
            t0 = time.perf_counter()
            if form is None:
                lib.evaluate_candidates(sess, xev[t], uev[t], tick=40000 + t)
            else:
                lib.evaluate_screened_host(sess, scr, xev[t], uev[t], k=form[0], tau=form[1],
                                           m=form[2], tick=40000 + t)
            lib.select_input(sess)
            lat.append(time.perf_counter() - t0)
        lat = np.array(lat[3:])  # the first ticks warm the host path
        out[name] = {"p50_ms": float(np.percentile(lat, 50) * 1e3),
                     "p99_ms": float(np.percentile(lat, 99) * 1e3),
                     "misses": int(np.count_nonzero(lat > 1.0 / 60.0))}
    torch.cuda.synchronize()
    return out


def concurrent_screened(lib, ctx, model, scr, N, k, cal, xev, uev, lo, hi, S=8, ticks=60):
    """Throughput when S sessions share the GPU: each with its own screener (same
    trained weights) and stream, every session queues `ticks` ticks back to back;
    ticks/s and executed rollout steps/s over the wall time, for the plain,
    cost-ordered and learned forms.  A lone tick is a latency chain; here the
    executed steps are what the GPU spends."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    weights = scr.get_weights()
    sessions = [lib.Session(ctx, model, N, 60, lo, hi, seed=11 + i) for i in range(S)]
    screeners = [lib.Screener(ctx, model, weights, max_batch=256, max_slots=N + 1)
                 for _ in range(S)]
    streams = [torch.cuda.Stream(dev) for _ in range(S)]
    xs = torch.tensor(np.asarray(xev[:ticks]), dtype=torch.float64, device=dev)
    us = torch.tensor(np.asarray(uev[:ticks]), dtype=torch.float64, device=dev)
    res = torch.zeros((S, ticks, lib.RESULT_BYTES), dtype=torch.uint8, device=dev)
    forms = {"plain": None, "cost_ordered": (k, 0.0, 1), "learned": (1, cal["tau"], cal["m"])}
    out = {"sessions": S, "ticks_per_session": ticks,
           "what": "S sessions on S streams queue their ticks back to back; wall time from the "
                   "first launch to the last result"}
    for name, form in forms.items():
        def launch(t):
            for i in range(S):
                if form is None:
                    lib.evaluate_candidates_device(sessions[i], xs[t], us[t], res[i, t],
                                                   tick=70000 + t, stream=streams[i])
                else:
                    lib.evaluate_screened(sessions[i], screeners[i], xs[t], us[t], res[i, t],
                                          k=form[0], tau=form[1], m=form[2], tick=70000 + t,
                                          stream=streams[i])
        launch(0)                       # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(ticks):
            launch(t)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        r = res.cpu().numpy()
        ex = sum(lib.result_from_bytes(r[i, t], 2)["executed_steps"]
                 for i in range(S) for t in range(ticks))
        out[name] = {"ticks_per_s": S * ticks / wall, "executed_steps_per_s": ex / wall,
                     "nominal_equivalent_steps_per_s": S * ticks * (N + 1) * 60 / wall}
    for s_ in sessions:
        s_.close()
    for sc in screeners:
        sc.free()
    return out


INFLATION_GRID = (0.0, 0.1, 0.2, 0.3, 0.35, 0.4)
INFLATION_SEEDS = (102, 103)  # held-out user-input seeds for choosing the radius


def run_inflation(args):
    """The paper's inflated barrier (Sec. V-C.1) in the balance-bot closed loop: the
    radius is chosen on held-out user-input seeds (fewest trial failures, then the
    smallest radius), then the benchmark's own closed loop (N = 16384, H = 50, 1000
    ticks, seed 2) runs with and without it."""
    import torch
    from paper_1906_02318_gb300 import mpmi as lib
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = lib.Context(dev.index)
    x, u, xn = data.transitions("bot", FIT_SEED, FIT_COUNT)

    def loop(seed, iota):
        model, _ = lib.fit_model(ctx, "bot", x, u, xn)
        lib.set_safety_set(model, data.BOT_SAFE_LO, data.BOT_SAFE_HI, iota)
        sess = lib.Session(ctx, model, N_SAMPLES, HORIZON, plants.BOT_INPUT_LO,
                           plants.BOT_INPUT_HI, seed=seed)
        uhs = data.ou_user_input(seed, TICKS, plants.BOT_DT, plants.BOT_INPUT_LO,
                                 plants.BOT_INPUT_HI)
        x_t, trials, recs = X0.copy(), 1, []
        for t in range(TICKS):
            lib.evaluate_candidates(sess, x_t, uhs[t], tick=t)
            r = lib.select_input(sess)
            x_t = plants.cartpole_step(x_t, r["u_r"])
            inside = bool(np.all(np.isfinite(x_t)) and np.all(x_t > data.BOT_SAFE_LO)
                          and np.all(x_t < data.BOT_SAFE_HI))
            recs.append(metrics.tick_record(r, uhs[t], t, trials - 1, N_SAMPLES,
                                            failed=not inside))
            if not inside:
                x_t, trials = X0.copy(), trials + 1
        sess.close()
        model.free()
        pm = metrics.summarize(recs, plants.BOT_DT)
        return {"trials": pm["trials"], "failures": trials - 1,
                "fallback_ticks": pm["fallback_ticks"],
                "safe_trial_fraction": pm["safe_trial_fraction"],
                "mean_time_to_failure_s": pm["mean_time_to_failure_s"],
                "avg_deviation": pm["avg_deviation"]}

    sweep = {}
    for iota in INFLATION_GRID:
        sweep[iota] = sum(loop(seed, iota)["failures"] for seed in INFLATION_SEEDS)
    best = min(INFLATION_GRID, key=lambda i: (sweep[i], i))
    return {"workload": "balance-bot closed loop: N=16384 (+u_h), H=50, 100 Hz, 1000 ticks, "
                        f"user-input seed {LOOP_SEED}",
            "selection": {"seeds": list(INFLATION_SEEDS),
                          "failures_by_radius": {str(k): v for k, v in sweep.items()},
                          "rule": "fewest trial failures on the held-out seeds, then the "
                                  "smallest radius"},
            "radius": best, "without": loop(LOOP_SEED, 0.0), "with": loop(LOOP_SEED, best)}


def run_serving(args, bot_states):
    """256 concurrent sessions, half balance bot and half race car, N log-uniform in
    1k..64k, H uniform in 20..100, ticks at 100 / 60 Hz with +-2 ms jitter, served
    by one continuous-batching server per model (two streams), for a fixed wall
    time.  Latency runs from a tick's scheduled arrival to its collected result."""
    import torch
    from paper_1906_02318_gb300 import mpmi as lib
    from paper_1906_02318_gb300 import serve
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = lib.Context(dev.index)
    x, u, xn = data.transitions("bot", FIT_SEED, FIT_COUNT)
    bm, _ = lib.fit_model(ctx, "bot", x, u, xn)
    lib.set_safety_set(bm, data.BOT_SAFE_LO, data.BOT_SAFE_HI)
    x, u, xn = data.transitions("car", 3, 20000)
    cm, _ = lib.fit_model(ctx, "car", x, u, xn)
    track = data.track_polyline(3)
    lib.set_safety_set(cm, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.0, track,
                       data.CAR_TRACK_HALF_WIDTH)
    n_sess = args.serve_sessions
    bs = lib.Server(ctx, bm, n_sess)
    cs = lib.Server(ctx, cm, n_sess)
    x0 = data.car_start_state(track, vx=13.0)
    car_pool = x0[None, :] + data.states_in_box(4, 256, [-1.5, -1.5, -0.1, -3, -0.3, -0.2],
                                                [1.5, 1.5, 0.1, 3, 0.3, 0.2])
    meta = [(bs, plants.BOT_INPUT_LO, plants.BOT_INPUT_HI, 0.01),
            (cs, plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, 1.0 / 60.0)]
    sessions = serve.make_sessions(meta, n_sess, 4, [bot_states, car_pool])
    # the servers' autotuner: every compiled serve shape and block size on a small
    # batch like the mix's typical one (three sessions of the model)
    tuned = {}
    for m, (srv, lo, hi, _) in enumerate(meta):
        mine = [ss for ss in sessions if ss.server == m][:3]
        reqs = [(ss.n, ss.horizon, lo, hi, 90 + i, 900 + i) for i, ss in enumerate(mine)]
        xs = np.stack([ss.states[0] for ss in mine])
        us = np.stack([ss.user[0] for ss in mine])
        r = srv.tune(reqs, xs, us, reps=5)
        tuned["bot" if m == 0 else "car"] = {k: r[k] for k in ("lanes", "cands", "block",
                                                                 "n_tried", "us", "default_us")}
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

    def serve_twice(servers, sess_list, seconds):
        """The same sessions served with up to four batches per model on the GPU at
        once, then with one batch at a time (ticks restart at 0 for the second run)."""
        runs = {}
        for name, overlap in (("overlap", 4), ("one_batch_at_a_time", 1)):
            for ss in sess_list:
                ss.next_tick, ss.outstanding, ss.latencies = 0, False, []
            runs[name] = serve.run(servers, sess_list, duration=seconds, streams=streams,
                                   overlap=overlap)
        return runs

    runs = serve_twice([bs, cs], sessions, args.serve_seconds)
    stats = dict(runs["overlap"])
    stats.update(sessions=n_sess, mix="half balance bot (100 Hz), half race car (60 Hz)",
                 n_range="log-uniform 1024..65536", h_range="uniform 20..100",
                 launch="one graph-replayed launch per batch; up to 4 batches per model in "
                        "flight, each on the server's own stream",
                 autotuned=tuned,
                 one_batch_at_a_time={k: runs["one_batch_at_a_time"][k]
                                      for k in ("ticks_per_s", "rollout_steps_per_s",
                                                "batches", "mean_batch", "latency")})
    bs.free()
    cs.free()
    # a heavier race-car-only mix (the GPU busy most of the time), with and without
    # overlapping batches
    n_heavy = 320
    hs = lib.Server(ctx, cm, n_heavy + n_heavy // 4)  # spare slots for the tuner's batch
    heavy = serve.make_sessions([(hs, plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, 1.0 / 60.0)],
                                n_heavy, 5, [car_pool])
    # tuned on a batch of a quarter of the sessions (the saturated run's batch cap)
    mine = heavy[:n_heavy // 4]
    reqs = [(ss.n, ss.horizon, plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, 190 + i, 1900 + i)
            for i, ss in enumerate(mine)]
    rh = hs.tune(reqs, np.stack([ss.states[0] for ss in mine]),
                 np.stack([ss.user[0] for ss in mine]), reps=3)
    hruns = serve_twice([hs], heavy, min(args.serve_seconds, 3.0))
    stats["car_heavy"] = {
        "sessions": n_heavy, "mix": "race car only, 60 Hz, N log-uniform 1024..65536, "
                                    "H uniform 20..100",
        "autotuned": {k: rh[k] for k in ("lanes", "cands", "block", "n_tried", "us",
                                          "default_us")},
        **{name: {k: r[k] for k in ("ticks_per_s", "rollout_steps_per_s", "batches",
                                     "mean_batch", "latency")} for name, r in hruns.items()}}
    # capacity: the same sessions, each submitting its next tick as soon as its last
    # result is back (no pacing): the ticks/s the server sustains for this mix and
    # the FP32 work its batches run (executed prediction steps x 2 n^2)
    for ss in heavy:
        ss.next_tick, ss.outstanding, ss.latencies = 0, False, []
        ss.period, ss.offset = 1e-9, 0.0
        ss.jitter = np.zeros_like(ss.jitter)
    rec = {}
    sat = serve.run([hs], heavy, duration=min(args.serve_seconds, 3.0), streams=streams,
                    record=rec, overlap=4, max_batch=n_heavy // 4)
    executed = float(sum(int(r["executed_steps"]) for r in rec.values()))
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(measured_peaks().get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * SM_FP32_LANES * 2 * sm_max * 1e6 / 1e12
    tflops = executed * 2 * CAR_LIFTED_N ** 2 / sat["wall_s"] / 1e12
    stats["car_saturated"] = {
        "sessions": n_heavy, "what": "the car_heavy sessions without pacing: each submits its "
                                     "next tick when its last result is back; at most a "
                                     "quarter of them per batch, up to four batches in flight",
        "seconds": sat["wall_s"], "ticks_per_s": sat["ticks_per_s"],
        "rollout_steps_per_s": sat["rollout_steps_per_s"],
        "executed_steps_per_s": executed / sat["wall_s"], "batches": sat["batches"],
        "mean_batch": sat["mean_batch"],
        "roofline": {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": tflops / fp32_peak}}
    hs.free()
    bm.free()
    cm.free()
    return stats


def run_car_loop(args):
    """The race car in closed loop (N = 16384, H = 60, 60 Hz, 600 ticks, start on
    the centre line at point 0 with vx = 10, OU user input, a trial restarting
    from the start whenever the car leaves the road): host ticks through the C
    ABI (latency, e2e rate), then the loop's states replayed device-resident
    with the L2 flushed before each tick."""
    import torch
    from paper_1906_02318_gb300 import mpmi as lib
    from paper_1906_02318_gb300.screener import car_in_safe_set
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = lib.Context(dev.index)
    x, u, xn = data.transitions("car", CAR_SEED, CAR_FIT_COUNT)
    model, _ = lib.fit_model(ctx, "car", x, u, xn)
    track = data.track_polyline(CAR_TRACK_SEED)
    lib.set_safety_set(model, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.0, track,
                       data.CAR_TRACK_HALF_WIDTH)
    lo, hi = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI
    ticks, N, H = args.car_ticks, 16384, 60
    x0 = data.car_start_state(track, vx=10.0)
    uhs = data.to_f32_exact(data.ou_user_input(CAR_SEED, ticks, plants.CAR_DT, lo, hi))
    tuned = lib.tune_launch_shape(ctx, model, N, H, lo, hi, x0, uhs[0], reps=20, seed=CAR_SEED)
    sess = lib.Session(ctx, model, N, H, lo, hi, seed=CAR_SEED)
    stream = torch.cuda.current_stream(dev)

    def closed_loop(recs=None):
        xt, states, lat = x0.copy(), np.empty((ticks, 6)), []
        trials, fallback = 1, 0
        for t in range(ticks):
            states[t] = xt
            t0 = time.perf_counter()
            lib.evaluate_candidates(sess, xt, uhs[t], tick=t, stream=stream)
            r = lib.select_input(sess)
            lat.append(time.perf_counter() - t0)
            fallback += r["status"] == lib.FALLBACK
            xt = plants.bicycle_step(xt, r["u_r"])
            inside = car_in_safe_set(xt, track, data.CAR_TRACK_HALF_WIDTH, 25.0)
            if recs is not None and t >= min(20, ticks // 10):
                recs.append(metrics.tick_record(r, uhs[t], t, trials - 1, N,
                                                latency_s=lat[-1], failed=not inside))
            if not inside:
                xt = x0.copy()
                trials += 1
        return states, np.array(lat[min(20, ticks // 10):]), trials, fallback

    # launched host ticks, then the same loop with persistent host ticks
    recs_l, recs_p = [], []
    states, lat_launched, trials, fallback = closed_loop(recs_l)
    lat, mode, same = lat_launched, "launched host ticks (requested)", None
    if not args.launched_host_ticks:
        try:
            sess.set_persistent(True)
        except lib.MpmiError as e:
            mode = f"launched host ticks (persistent unavailable: {e})"
        else:
            states_p, lat, _, _ = closed_loop(recs_p)
            sess.set_persistent(False)
            mode = "persistent host ticks (resident kernel, pinned mailbox)"
            same = bool(np.array_equal(states_p, states))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    xs = torch.tensor(states, dtype=torch.float64, device=dev)
    us = torch.tensor(uhs, dtype=torch.float64, device=dev)
    res = torch.zeros((ticks, lib.RESULT_BYTES), dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(ticks)]
    for i in range(3):
        lib.evaluate_candidates_device(sess, xs[i], us[i], res[i], tick=i)
    for i in range(ticks):
        flush.zero_()
        ev[i][0].record()
        lib.evaluate_candidates_device(sess, xs[i], us[i], res[i], tick=i)
        ev[i][1].record()
    torch.cuda.synchronize()
    durs = np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3
    executed = np.array([lib.result_from_bytes(b, 2)["executed_steps"] for b in res.cpu().numpy()])
    lanes, cands, block = sess.launch_shape()
    sess.close()
    model.free()
    # the float64 oracle on the host cores, beside it: one tick of CAR_ORACLE_N
    # candidates per worker, on the loop's first states
    from oracle import fit as ofit
    K32 = ofit.round_to_f32(ofit.fit_koopman("car", x, u, xn)[0])
    workers = max(1, min(16, os.cpu_count() or 1))
    o_rate, o_steps, o_t = oracle_rate(K32, states, uhs, CAR_ORACLE_N, H, 0.0, workers,
                                       list(range(min(workers, ticks))), basis="car")
    rate = (N + 1) * H / durs.mean()
    return {"workload": "race car closed loop: N=16384 (+u_h), H=60, 60 Hz, 600 ticks",
            "shape": {"lanes": lanes, "cands_per_thread": cands, "block": block,
                      "autotuned": {"n_tried": tuned["n_tried"], "winner_us": tuned["us"],
                                    "default_shape_us": tuned["default_us"]}},
            "ticks": ticks, "trials": trials, "fallback_ticks": int(fallback),
            "paper_metrics": metrics.summarize(recs_p if recs_p else recs_l, plants.CAR_DT),
            "device_mean_us": durs.mean() * 1e6, "device_p99_us": np.percentile(durs, 99) * 1e6,
            "rollout_steps_per_s": (N + 1) * H / durs.mean(),
            "executed_steps_per_s": executed.mean() / durs.mean(),
            "host_tick_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                             "p99": float(np.percentile(lat, 99) * 1e3), "deadline_ms": 1000 / 60,
                             "misses": int(np.count_nonzero(lat > 1 / 60)), "mode": mode},
            "e2e_rollout_steps_per_s": (N + 1) * H * len(lat) / lat.sum(),
            "launched_host_tick_ms": {"p50": float(np.percentile(lat_launched, 50) * 1e3),
                                      "p99": float(np.percentile(lat_launched, 99) * 1e3)},
            "persistent_loop_identical": same,
            "cpu_oracle": {"value": o_rate, "unit": "rollout steps/s", "cores": workers,
                           "kind": "oracle", "per_core_value": oracle_rate.per_core,
                           "sample": f"FP64 numpy oracle, {o_steps // ((CAR_ORACLE_N + 1) * H)} "
                                     f"ticks of N={CAR_ORACLE_N} (H=60, track test against all "
                                     f"segments), one per spawned single-threaded worker, "
                                     f"{o_t:.1f} s"},
            "gpu_over_oracle": rate / o_rate}


def run_variants(args, bot_states):
    """The paper's variants and the factorised ablation, device-resident at the
    benchmark's sizes (L2 flushed before every tick): the balance bot (N = 16384,
    H = 50) and the race car (N = 16384, H = 60) with the full rollout (Alg. 2),
    with per-step noise z_i, with the equally spaced grid (bot, Sec. IV-B), in
    the factorised read-out form (exact in real arithmetic, not the method's own
    rollout) and, for the race car, with the rollout on the tensor cores.  Rates
    count the steps the kernel executed (early exit)."""
    import torch
    from paper_1906_02318_gb300 import mpmi as lib
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = lib.Context(dev.index)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ticks = min(args.variant_ticks, len(bot_states))
    x, u, xn = data.transitions("bot", FIT_SEED, FIT_COUNT)
    bm, _ = lib.fit_model(ctx, "bot", x, u, xn)
    lib.set_safety_set(bm, data.BOT_SAFE_LO, data.BOT_SAFE_HI)
    x, u, xn = data.transitions("car", 3, 20000)
    cm, _ = lib.fit_model(ctx, "car", x, u, xn)
    track = data.track_polyline(3)
    lib.set_safety_set(cm, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.0, track,
                       data.CAR_TRACK_HALF_WIDTH)
    x0 = data.car_start_state(track, vx=12.0)
    car_states = x0[None, :] + data.states_in_box(8, ticks, [-1.5, -1.5, -0.1, -3, -0.3, -0.2],
                                                  [1.5, 1.5, 0.1, 3, 0.3, 0.2])
    plans = {
        "bot": (bm, plants.BOT_INPUT_LO, plants.BOT_INPUT_HI, HORIZON, bot_states[:ticks],
                [0.005, 0.02, 0.005, 0.02]),
        "car": (cm, plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, 60, car_states,
                [0.03, 0.03, 0.005, 0.1, 0.02, 0.01]),
    }
    out = {"N": N_SAMPLES, "ticks": ticks, "l2": "flushed before every tick", "runs": {}}
    res = torch.zeros((ticks, lib.RESULT_BYTES), dtype=torch.uint8, device=dev)
    for name, (model, lo, hi, H, states, sigma) in plans.items():
        uhs = data.ou_user_input(9, ticks, 0.01, lo, hi)
        xs = torch.tensor(np.asarray(states), dtype=torch.float64, device=dev)
        us = torch.tensor(uhs, dtype=torch.float64, device=dev)
        variants = [("full", {}), ("noise", {"noise": sigma}), ("factored", {"rollout": "factored"})]
        if name == "bot":
            variants.insert(2, ("grid", {"sampler": "grid"}))
        else:
            variants.append(("tensor", {"rollout": "tensor"}))
        runs = {}
        for vname, opt in variants:
            sess = lib.Session(ctx, model, N_SAMPLES, H, lo, hi, seed=11,
                               sampler=opt.get("sampler", "uniform"))
            if "noise" in opt:
                sess.set_noise(opt["noise"])
            if "rollout" in opt:
                sess.set_rollout(opt["rollout"])
            for i in range(3):
                lib.evaluate_candidates_device(sess, xs[i], us[i], res[i], tick=i)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(ticks)]
            for i in range(ticks):
                flush.zero_()
                ev[i][0].record()
                lib.evaluate_candidates_device(sess, xs[i], us[i], res[i], tick=100 + i)
                ev[i][1].record()
            torch.cuda.synchronize()
            durs = np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3
            rr = [lib.result_from_bytes(r, sess.nu) for r in res.cpu().numpy()]
            executed = float(np.mean([r["executed_steps"] for r in rr]))
            runs[vname] = {"mean_us": durs.mean() * 1e6, "p99_us": np.percentile(durs, 99) * 1e6,
                           "executed_steps_per_tick": executed,
                           "executed_steps_per_s": executed / durs.mean(),
                           "nominal_steps_per_s": sess.n_slots * H / durs.mean(),
                           "safe_fraction": float(np.mean([r["n_safe"] for r in rr])) / sess.n_slots}
            sess.close()
        out["runs"][name] = dict(H=H, sigma=sigma, **runs)
    bm.free()
    cm.free()
    return out


OVER_N = (16384, 65536, 262144, 1048576)


def run_over_n(args, bot_states):
    """The plain tick's roofline fraction as N grows, one session, the library's
    default launch shape, device-resident (L2 flushed before every tick): the
    balance bot at H = 50 and the race car at H = 60.  At the benchmark's N the
    candidates fill one warp per SM sub-partition and a tick is one warp's serial
    chain plus fixed costs; with more candidates the same kernel approaches the
    FP32 pipe.  Work counted: executed prediction steps x 2 n^2 flops."""
    import torch
    from paper_1906_02318_gb300 import mpmi as lib
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * SM_FP32_LANES * 2 * sm_max * 1e6 / 1e12
    ctx = lib.Context(dev.index)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ticks = min(args.over_n_ticks, len(bot_states))
    x, u, xn = data.transitions("bot", FIT_SEED, FIT_COUNT)
    bm, _ = lib.fit_model(ctx, "bot", x, u, xn)
    lib.set_safety_set(bm, data.BOT_SAFE_LO, data.BOT_SAFE_HI)
    x, u, xn = data.transitions("car", 3, 20000)
    cm, _ = lib.fit_model(ctx, "car", x, u, xn)
    track = data.track_polyline(3)
    lib.set_safety_set(cm, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.0, track,
                       data.CAR_TRACK_HALF_WIDTH)
    x0 = data.car_start_state(track, vx=12.0)
    car_states = x0[None, :] + data.states_in_box(8, ticks, [-1.5, -1.5, -0.1, -3, -0.3, -0.2],
                                                  [1.5, 1.5, 0.1, 3, 0.3, 0.2])
    plans = {"bot": (bm, plants.BOT_INPUT_LO, plants.BOT_INPUT_HI, HORIZON, LIFTED_N,
                     bot_states[:ticks]),
             "car": (cm, plants.CAR_INPUT_LO, plants.CAR_INPUT_HI, 60, CAR_LIFTED_N, car_states)}
    out = {"ticks": ticks, "l2": "flushed before every tick", "peak_tflops": peak,
           "work": "executed prediction steps x 2 n^2 flops", "runs": {}}
    res = torch.zeros((ticks, lib.RESULT_BYTES), dtype=torch.uint8, device=dev)
    for name, (model, lo, hi, H, n, states) in plans.items():
        uhs = data.ou_user_input(9, ticks, 0.01, lo, hi)
        xs = torch.tensor(np.asarray(states), dtype=torch.float64, device=dev)
        us = torch.tensor(uhs, dtype=torch.float64, device=dev)
        rows = []
        for N in OVER_N:
            sess = lib.Session(ctx, model, N, H, lo, hi, seed=11)
            for i in range(3):
                lib.evaluate_candidates_device(sess, xs[i], us[i], res[i], tick=i)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(ticks)]
            for i in range(ticks):
                flush.zero_()
                ev[i][0].record()
                lib.evaluate_candidates_device(sess, xs[i], us[i], res[i], tick=100 + i)
                ev[i][1].record()
            torch.cuda.synchronize()
            mean = float(np.mean([a.elapsed_time(b) for a, b in ev])) * 1e-3
            rr = [lib.result_from_bytes(r, sess.nu) for r in res.cpu().numpy()]
            executed = float(np.mean([r["executed_steps"] for r in rr]))
            tflops = executed * 2 * n * n / mean / 1e12
            lanes, cands, block = sess.launch_shape()
            rows.append({"N": N, "H": H, "lanes": lanes, "cands_per_thread": cands,
                         "block": block, "mean_us": mean * 1e6,
                         "executed_steps_per_s": executed / mean,
                         "nominal_steps_per_s": sess.n_slots * H / mean,
                         "tflops": tflops, "frac": tflops / peak})
            sess.close()
        out["runs"][name] = rows
    bm.free()
    cm.free()
    return out


def max_over_ranks(values, world: int, device: str = "cpu"):
    """Element-wise maximum of per-rank timings (the slowest rank sets the job time)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(world: int, steps_per_rank: int, units_per_step: int, t_max: float) -> float:
    """Whole-job rate: every rank processed steps_per_rank steps of units_per_step units
    (weak scaling, independent replicas) within the slowest rank's time."""
    return world * steps_per_rank * units_per_step / t_max


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle work per host worker for cpu_baseline")
    ap.add_argument("--learned-ticks", type=int, default=300,
                    help="held-out ticks for the learned-vs-plain comparison (0 = skip)")
    ap.add_argument("--inflation", type=int, default=1,
                    help="run the inflated-barrier closed loops (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="wall time of the 256-session serving run (0 = skip)")
    ap.add_argument("--serve-sessions", type=int, default=256)
    ap.add_argument("--variant-ticks", type=int, default=200,
                    help="ticks per paper variant / factorised ablation (0 = skip)")
    ap.add_argument("--over-n-ticks", type=int, default=40,
                    help="ticks per N of the plain tick's roofline over N (0 = skip)")
    ap.add_argument("--car-ticks", type=int, default=600,
                    help="race-car closed-loop ticks (0 = skip)")
    ap.add_argument("--launched-host-ticks", action="store_true",
                    help="host ticks as one launch each only (no resident kernel; for runs "
                         "under a profiler, which serialises launches and would leave a "
                         "resident kernel waiting on a mailbox that cannot be written)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cfg = {"workload": "balance-bot closed loop: N=16384 (+u_h), H=50, 100 Hz, 1000 ticks",
           "N": N_SAMPLES, "H": HORIZON, "lifted_dim": LIFTED_N, "input_dim": 1,
           "ticks": TICKS, "fit_transitions": FIT_COUNT,
           "l2": "flushed before every timed tick (256 MB write)"}

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, cfg)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", rank))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    out = run_gpu(args, rank, world)

    n_step = (N_SAMPLES + 1) * HORIZON
    K = args.steps
    t_max, e2e_max = max_over_ranks([out["dev_time"], float(out["lat"].sum())], world,
                                    device="cuda")
    value = job_throughput(world, K, n_step, t_max)
    e2e_value = job_throughput(world, len(out["lat"]), n_step, e2e_max)

    if out["persistent"]:
        # the resident kernel reads the mailbox (command word + 15 words) and writes
        # the result record and the completion word
        e2e_mode = "persistent host ticks (resident kernel, pinned mailbox)"
        h2d, d2h = 16 * 8, 80 + 8
    else:
        e2e_mode = "launched host ticks (" + str(out["persist_note"]) + ")"
        h2d, d2h = 12 * 8, 80 + 8

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = out["sm_count"] * SM_FP32_LANES * 2 * sm_max * 1e6 / 1e12
    mean_dur = float(out["durs"].mean())
    flops_per_tick = (float(out["executed"].mean()) * 2 * LIFTED_N ** 2
                      + out["n_slots"] * (2 * LIFTED_N * 1 + 2))
    achieved = flops_per_tick / mean_dur / 1e12
    traffic = (TRAFFIC["bytes_per_launch"].get((out["lanes"], out["cands"], out["block"]))
               if TRAFFIC["tick_kernel_sha1"] == kernel_sha1() else None)

    line = {
        "metric": "rollout steps/s (plain path) and p99 control-tick latency at N=16384",
        "value": value, "unit": "rollout steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": t_max / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(cfg, parallelism=f"replicas{world}" if world > 1 else "single"),
        "launch": {"lanes": out["lanes"], "cands_per_thread": out["cands"],
                   "block": out["block"],
                   "autotuned": {"n_tried": out["tuned"]["n_tried"],
                                 "winner_us": out["tuned"]["us"],
                                 "default_shape_us": out["tuned"]["default_us"],
                                 "what": "warm device ticks, median of 30 per shape"}},
        "executed_steps_per_s": world * float(out["executed"].sum()) / t_max,
        "latency_ms": {"p50": float(np.percentile(out["lat"], 50) * 1e3),
                       "p99": float(np.percentile(out["lat"], 99) * 1e3),
                       "deadline_ms": 10.0,
                       "misses": int(np.count_nonzero(out["lat"] > 0.010)),
                       "what": "host-to-host C-ABI tick (evaluate_candidates + select_input), "
                               + e2e_mode},
        "learned": None,
        "e2e": {"value": e2e_value, "unit": "rollout steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "mode": e2e_mode},
        "e2e_launched": {
            "value": n_step * len(out["lat_launched"]) / float(out["lat_launched"].sum()),
            "unit": "rollout steps/s",
            "p50_ms": float(np.percentile(out["lat_launched"], 50) * 1e3),
            "p99_ms": float(np.percentile(out["lat_launched"], 99) * 1e3),
            "what": "one kernel launch per host tick; x_t/u_h read and the result written "
                    "over the host link (zero-copy)"},
        "persistent_loop_identical": out["persist_same"],
        "gpu_launches": K,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                     "peak_basis": f"{out['sm_count']} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                     "ffma_loop_tflops": out["ffma_tflops"],
                     "frac_of_ffma_loop": achieved / out["ffma_tflops"]},
        "clocks": out["clocks"],
        "fallback_ticks": out["n_fallback"], "trials": out["trials"],
        "paper_metrics": out["paper_metrics"],
        "paper_context": PAPER_CONTEXT,
    }
    if rank == 0 and args.learned_ticks > 0:
        line["learned"] = run_learned(args)
    if rank == 0 and args.inflation:
        line["closed_loop_inflated"] = run_inflation(args)
    if rank == 0 and args.serve_seconds > 0:
        line["serving"] = run_serving(args, out["states"])
    if rank == 0 and args.variant_ticks > 0:
        line["variants"] = run_variants(args, out["states"])
    if rank == 0 and args.car_ticks > 0:
        line["car_closed_loop"] = run_car_loop(args)
    if rank == 0 and args.over_n_ticks > 0:
        line["roofline_over_n"] = run_over_n(args, out["states"])
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(args):
    K32 = oracle_model()
    states, uhs = reference_states()
    workers = max(1, min(16, os.cpu_count() or 1))
    rate, steps, _ = oracle_rate(K32, states, uhs, N_SAMPLES, HORIZON, args.cpu_budget,
                                 workers, list(range(TICKS)))
    return {"value": rate, "unit": "rollout steps/s", "cores": workers, "kind": "oracle",
            "per_core_value": oracle_rate.per_core,
            "sample": f"FP64 numpy oracle, {steps // ((N_SAMPLES + 1) * HORIZON)} full ticks "
                      f"(N=16384, H=50) across {workers} spawned single-threaded workers, "
                      f"~{args.cpu_budget:.0f} s each"}


def run_reference(args, cfg):
    """The oracle as it stands, timed on the host cores, same metric and workload;
    each step is one full tick (N=16384, H=50), ticks spread over workers."""
    K32 = oracle_model()
    states, uhs = reference_states()
    workers = max(1, min(16, os.cpu_count() or 1))
    # warm-up ticks (untimed), then exactly K timed ticks
    oracle_rate(K32, states, uhs, N_SAMPLES, HORIZON, 1e9, workers,
                list(range(min(args.warmup, TICKS))))
    ids = [i % TICKS for i in range(args.steps)]
    value, steps, wall = oracle_rate(K32, states, uhs, N_SAMPLES, HORIZON, 1e9, workers, ids)
    line = {"metric": "rollout steps/s (plain path) and p99 control-tick latency at N=16384",
            "value": value, "unit": "rollout steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(cfg, parallelism=f"replicas{args.gpus}" if args.gpus > 1 else "single"),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "rollout steps/s", "cores": workers,
                             "kind": "oracle",
                             "sample": f"{args.steps} full ticks over {workers} spawned "
                                       "single-threaded workers on the host cores, no GPU "
                                       "(slowest worker's time)"},
            "e2e": {"value": value, "unit": "rollout steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
