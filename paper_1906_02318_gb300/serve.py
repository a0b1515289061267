"""Continuous-batching serving loop over mpmi servers (one per model).

Sessions tick at their own rate (100 Hz balance bot, 60 Hz race car) with a
seeded +-2 ms jitter; a tick's request is staged as soon as it is due and the
session's previous request has completed (a controller needs its last output
before its next input).  A server launches its staged requests as soon as it
has fewer than `overlap` batches on the GPU, so requests that arrive while a
batch runs start in a batch of their own that overlaps it on the device (with
overlap = 1 they wait for the running batch to be collected); finished batches
are collected in completion order.  Latency is measured from a request's
scheduled arrival to the moment its batch has been collected.  All computation
runs in libmpmi; this module keeps clocks and queues.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import mpmi as lib


@dataclass
class ServedSession:
    server: int          # index into the server list
    slot: int            # server session slot
    period: float        # seconds between ticks
    n: int
    horizon: int
    states: np.ndarray   # (T, nx) state per tick (replayed)
    user: np.ndarray     # (T, nu) user input per tick
    offset: float        # first arrival time
    jitter: np.ndarray   # (T,) seconds
    next_tick: int = 0
    outstanding: bool = False
    latencies: list = field(default_factory=list)


def run(servers, sessions, duration: float, streams=None, record=None, overlap: int = 4,
        max_batch: int | None = None):
    """Serve `sessions` for `duration` seconds of wall time with at most `overlap`
    batches per server on the GPU and, with max_batch, at most that many requests
    per batch (the rest stay due for the next one, so that sessions which all come
    due at once still spread over overlapping batches).  Returns stats; if `record`
    is a dict, every result is stored under (session index, tick)."""
    import torch
    streams = streams or [torch.cuda.Stream() for _ in servers]
    for srv in servers:
        srv.set_max_in_flight(overlap)
        srv._n_flying = srv._n_staged = 0
    by_server = [[] for _ in servers]
    for i, s in enumerate(sessions):
        by_server[s.server].append(i)
    slot_to_sess = [{sessions[i].slot: i for i in idx} for idx in by_server]
    steps = 0
    done_ticks = 0
    batches = 0
    batch_sizes = []
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        if now >= duration:
            break
        for si, srv in enumerate(servers):
            while srv._n_flying and srv.poll():
                t_done = time.perf_counter() - t0
                for slot, r in srv.collect():
                    ss = sessions[slot_to_sess[si][slot]]
                    k = int(r["tick"])
                    arrival = ss.offset + k * ss.period + ss.jitter[k % len(ss.jitter)]
                    ss.latencies.append(t_done - arrival)
                    ss.outstanding = False
                    steps += (ss.n + 1) * ss.horizon
                    done_ticks += 1
                    if record is not None:
                        record[(slot_to_sess[si][slot], k)] = r
                srv._n_flying -= 1
            # stage the due requests of this server's sessions (up to max_batch per
            # batch)
            room = None if max_batch is None else max_batch - srv._n_staged
            due = []
            for i in by_server[si]:
                if room is not None and len(due) >= room:
                    break
                ss = sessions[i]
                k = ss.next_tick
                if not ss.outstanding and ss.offset + k * ss.period + ss.jitter[k % len(ss.jitter)] <= now:
                    due.append(i)
            if due:
                srv.submit([sessions[i].slot for i in due],
                           np.stack([sessions[i].states[sessions[i].next_tick % len(sessions[i].states)] for i in due]),
                           np.stack([sessions[i].user[sessions[i].next_tick % len(sessions[i].user)] for i in due]),
                           [sessions[i].next_tick for i in due])
                for i in due:
                    sessions[i].outstanding = True
                    sessions[i].next_tick += 1
            srv._n_staged += len(due)
            if srv._n_flying < overlap and srv._n_staged:
                batch_sizes.append(srv.launch(streams[si]))
                srv._n_flying += 1
                srv._n_staged = 0
                batches += 1
    # drain: every batch in flight, then whatever is still staged, so the servers
    # end empty (a later run on them starts from no pending request)
    for si, srv in enumerate(servers):
        while srv._n_flying:
            srv.collect()
            srv._n_flying -= 1
        if srv._n_staged:
            srv.launch(streams[si])
            batches += 1
            srv.collect()
            srv._n_staged = 0
    wall = time.perf_counter() - t0
    lat = {}
    for kind in sorted({s.period for s in sessions}):
        v = np.concatenate([np.asarray(s.latencies) for s in sessions if s.period == kind]
                           or [np.zeros(0)])
        if v.size:
            lat[f"{1.0 / kind:.0f}Hz"] = dict(
                ticks=int(v.size), p50_ms=float(np.percentile(v, 50) * 1e3),
                p99_ms=float(np.percentile(v, 99) * 1e3), max_ms=float(v.max() * 1e3),
                deadline_ms=kind * 1e3, misses=int(np.count_nonzero(v > kind)))
    return dict(wall_s=wall, ticks=done_ticks, ticks_per_s=done_ticks / wall,
                rollout_steps_per_s=steps / wall, batches=batches,
                mean_batch=float(np.mean(batch_sizes)) if batch_sizes else 0.0, latency=lat)


def make_sessions(servers_meta, n_sessions, seed, state_pools, ticks=4096):
    """Seeded session mix: alternating models, N log-uniform in [1k, 64k], H uniform
    in 20..100, rates 100 Hz (model 0) and 60 Hz (model 1), +-2 ms jitter; each
    session replays its model's state pool from a random offset with its own
    Ornstein-Uhlenbeck user input."""
    from workloads import data
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_sessions):
        m = i % len(servers_meta)
        srv, lo, hi, period = servers_meta[m]
        n = int(round(np.exp(rng.uniform(np.log(1024), np.log(65536)))))
        H = int(rng.integers(20, 101))
        slot = srv.admit(n, H, lo, hi, seed=seed * 1000 + i, stream_id=i)
        pool = state_pools[m]
        start = int(rng.integers(0, len(pool)))
        states = np.roll(pool, -start, axis=0)
        user = data.ou_user_input(seed * 7919 + i, ticks, period, lo, hi)
        jitter = rng.uniform(-0.002, 0.002, ticks)
        out.append(ServedSession(server=m, slot=slot, period=period, n=n, horizon=H,
                                 states=states, user=user, offset=float(rng.uniform(0.003, 0.02)),
                                 jitter=jitter))
    return out
