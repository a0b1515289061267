"""The real-time serving loop's host-side scheduling (paper_1906_02318_gb300.serve),
on the CPU with a fake server that keeps the library server's protocol and takes
a fixed service time per batch: requests that arrive while batches run are
launched in batches of their own up to the overlap bound, finished batches are
collected, every request is answered exactly once and a session never has two
requests outstanding."""
import time

import numpy as np
import pytest

from paper_1906_02318_gb300 import serve


class FakeServer:
    """The mpmi server's host protocol with batches that finish `service_s` after
    their launch (wall clock)."""

    def __init__(self, service_s):
        self.service_s = service_s
        self.max_in_flight = 4
        self.staged = []          # [(slot, tick)]
        self.flying = []          # [(launch order, done time, [(slot, tick)])]
        self.busy = set()         # sessions with a request staged or in flight
        self.launches = 0
        self.most_in_flight = 0
        self.answered = []

    def set_max_in_flight(self, n):
        assert 1 <= n <= 4
        self.max_in_flight = n

    def submit(self, slots, x_t, u_h, ticks):
        assert len(slots) == len(x_t) == len(u_h) == len(ticks)
        for sl, t in zip(slots, ticks):
            assert sl not in self.busy, "a session with a request outstanding was submitted"
            self.busy.add(sl)
            self.staged.append((sl, int(t)))

    def launch(self, stream=None):
        if not self.staged:
            return 0
        assert len(self.flying) < self.max_in_flight, "launch beyond the in-flight bound"
        self.flying.append((self.launches, time.perf_counter() + self.service_s, self.staged))
        self.launches += 1
        self.most_in_flight = max(self.most_in_flight, len(self.flying))
        n = len(self.staged)
        self.staged = []
        return n

    def poll(self):
        now = time.perf_counter()
        return any(done <= now for _, done, _ in self.flying)

    def collect(self):
        now = time.perf_counter()
        done = [f for f in self.flying if f[1] <= now]
        pick = min(done or self.flying, key=lambda f: f[0])
        if pick[1] > now:
            time.sleep(pick[1] - now)
        self.flying.remove(pick)
        out = []
        for sl, t in pick[2]:
            self.busy.discard(sl)
            self.answered.append((sl, t))
            out.append((sl, {"tick": t}))
        return out


def _sessions(n, period, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(serve.ServedSession(
            server=0, slot=i, period=period, n=1000, horizon=20,
            states=np.zeros((8, 4)), user=np.zeros((8, 1)),
            offset=float(rng.uniform(0.0, period)), jitter=rng.uniform(-0.001, 0.001, 64)))
    return out


@pytest.mark.parametrize("overlap", [1, 4])
def test_overlap_bound_and_every_request_answered(overlap):
    # 24 sessions at 200 Hz against batches that take 6 ms: requests keep arriving
    # while batches run
    srv = FakeServer(service_s=0.006)
    sess = _sessions(24, 0.005, seed=overlap)
    stats = serve.run([srv], sess, duration=0.25, streams=[None], overlap=overlap)
    assert srv.max_in_flight == overlap
    assert srv.most_in_flight <= overlap
    if overlap > 1:
        assert srv.most_in_flight > 1          # batches did overlap
    assert not srv.flying and not srv.busy and not srv.staged  # drained, nothing left staged
    # every launched request answered once, per session in tick order from 0
    assert stats["ticks"] == sum(len(s.latencies) for s in sess)
    for i, s in enumerate(sess):
        ticks = [t for sl, t in srv.answered if sl == i]
        assert ticks == list(range(len(ticks))) and len(ticks) == s.next_tick
    assert stats["batches"] == srv.launches


def test_overlap_lowers_latency_under_load():
    lat = {}
    for overlap in (1, 4):
        srv = FakeServer(service_s=0.006)
        sess = _sessions(24, 0.005, seed=7)
        stats = serve.run([srv], sess, duration=0.3, streams=[None], overlap=overlap)
        lat[overlap] = stats["latency"]["200Hz"]["p50_ms"]
    # with one batch at a time a request waits for the running batch to finish
    assert lat[4] < lat[1]


def test_max_batch_caps_each_launch():
    """With max_batch, sessions that come due together spread over several batches
    (each at most max_batch requests) instead of one, and every request is still
    answered once and in tick order."""
    srv = FakeServer(service_s=0.004)
    sizes = []
    launch = srv.launch

    def counting_launch(stream=None):
        n = len(srv.staged)
        sizes.append(n)
        return launch(stream)
    srv.launch = counting_launch
    sess = _sessions(40, 1e-9, seed=3)           # no pacing: always due
    for s in sess:
        s.offset, s.jitter = 0.0, np.zeros_like(s.jitter)
    stats = serve.run([srv], sess, duration=0.2, streams=[None], overlap=4, max_batch=10)
    assert sizes and max(sizes) <= 10
    assert srv.most_in_flight > 1
    assert not srv.flying and not srv.busy and not srv.staged
    for i, s in enumerate(sess):
        ticks = [t for sl, t in srv.answered if sl == i]
        assert ticks == list(range(len(ticks))) and len(ticks) == s.next_tick
    assert stats["batches"] == srv.launches
