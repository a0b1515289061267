"""The continuous-batching server (through the C ABI): every served result equals
the same tick evaluated alone, admission follows slots and the memory budget, and
a short real-time serving run completes every request."""
import numpy as np
import pytest

from workloads import data, plants

from oracle import mpmi as omp
from oracle import safety as osafe
from parity import (BOUNDARY_TOL, TIE_RTOL, TRAJ_RTOL, bot_env, car_env, gpu_model,
                    oracle_samples, run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def _states(env, which, count, seed):
    if which == "bot":
        return data.states_in_box(seed, count, [-0.3, -1, -1, -1], [0.3, 1, 1, 1])
    x0 = data.car_start_state(env.track, vx=13.0)
    return x0[None, :] + data.states_in_box(seed, count, [-1.5, -1.5, -0.1, -3, -0.3, -0.2],
                                            [1.5, 1.5, 0.1, 3, 0.3, 0.2])


def _alone(lib, ctx, model, env, n, H, seed, stream, x, u, tick):
    sess = lib.Session(ctx, model, n, H, env.lo, env.hi, seed=seed, stream_id=stream)
    g = run_gpu(lib, sess, x, u, tick=tick)
    sess.close()
    return g["result"]


@pytest.mark.parametrize("which", ["bot", "car"])
def test_served_results_equal_alone(lib, ctx, which):
    env = bot_env() if which == "bot" else car_env()
    model = gpu_model(lib, ctx, env)
    srv = lib.Server(ctx, model, max_sessions=16)
    rng = np.random.default_rng(0)
    specs = [(0, 7), (1, 50), (1023, 20), (4096, 100), (20000, 60), (65535, 33), (3000, 1)]
    slots = [srv.admit(n, H, env.lo, env.hi, seed=100 + i, stream_id=i)
             for i, (n, H) in enumerate(specs)]
    for batch in range(3):          # both buffers, then the first again
        xs = _states(env, which, len(specs), 10 + batch)
        us = data.to_f32_exact(rng.uniform(env.lo, env.hi, (len(specs), len(env.lo))))
        ticks = [batch * 1000 + i for i in range(len(specs))]
        order = rng.permutation(len(specs))
        srv.submit([slots[i] for i in order], xs[order], us[order], [ticks[i] for i in order])
        assert srv.launch() == len(specs)
        got = dict(srv.collect())
        for i, (n, H) in enumerate(specs):
            a = _alone(lib, ctx, model, env, n, H, 100 + i, i, xs[i], us[i], ticks[i])
            r = got[slots[i]]
            for k in ("index", "status", "n_safe", "ttv", "executed_steps", "n_slots", "tick"):
                assert r[k] == a[k], (batch, i, k)
            assert np.array_equal(r["u_r"], a["u_r"]) and r["cost"] == a["cost"]
    srv.free()
    model.free()


@pytest.mark.parametrize("which", ["bot", "car"])
def test_served_results_match_oracle(lib, ctx, which):
    """A served batch against the float64 oracle directly (not only against the
    same tick alone): the pick is the oracle's unless the two picks tie in cost or
    one of them passes within the trajectory tolerance of a safety bound, the
    status and the pick's cost agree, and the number of safe candidates differs
    only by boundary cases (at most 0.2 % of the slots)."""
    env = bot_env() if which == "bot" else car_env()
    model = gpu_model(lib, ctx, env)
    srv = lib.Server(ctx, model, max_sessions=8)
    H = 30
    # (N, stream); the race car's oracle tests every segment of the track per step
    specs = [(500, 0), (2047, 1), (3000, 2)] if which == "bot" else [(300, 0), (1023, 1),
                                                                      (1500, 2)]
    slots = [srv.admit(n, H, env.lo, env.hi, seed=77, stream_id=sid) for n, sid in specs]
    xs = _states(env, which, len(specs), 31)
    us = data.to_f32_exact(np.random.default_rng(8).uniform(env.lo, env.hi,
                                                          (len(specs), len(env.lo))))
    ticks = [900 + i for i in range(len(specs))]
    srv.submit(slots, xs, us, ticks)
    assert srv.launch() == len(specs)
    got = dict(srv.collect())
    for i, (n, sid) in enumerate(specs):
        r = got[slots[i]]
        o = omp.tick(env.K32, env.basis, xs[i], us[i], oracle_samples(env, n, 77, sid, ticks[i]),
                     H, env.spec, record=True)
        gi, oi = r["index"], o.index
        if gi != oi:
            tie = o.ttv[gi] == o.ttv[oi] and abs(o.cost[gi] - o.cost[oi]) <= \
                TIE_RTOL * max(o.cost[gi], o.cost[oi]) + 1e-12

            def near_bound(slot):
                steps = min(int(o.ttv[slot]) + 1, H)
                zs = o.traj[slot, 1:steps + 1]
                scale = np.maximum(np.abs(zs).max(axis=1), 1.0)
                m = np.abs(osafe.margin(env.spec, zs))
                return bool(np.any(m <= (TRAJ_RTOL + BOUNDARY_TOL) * scale))
            assert tie or near_bound(gi) or near_bound(oi), (which, i, gi, oi)
        else:
            assert r["ttv"] == int(o.ttv[oi])
            assert abs(r["cost"] - o.cost[oi]) <= 1e-6 * max(o.cost[oi], 1e-12) + 1e-12
        assert r["status"] == (omp.SAFE if o.ttv[oi] == H else omp.FALLBACK) or gi != oi
        n_safe_o = int(np.count_nonzero(o.ttv == H))
        assert abs(r["n_safe"] - n_safe_o) <= max(1, 0.002 * (n + 1))
        assert r["n_slots"] == n + 1 and r["tick"] == ticks[i]
    srv.free()
    model.free()


def test_admission_by_slots_and_budget(lib):
    env = bot_env()
    big = lib.Context(0)
    model = gpu_model(lib, big, env)
    srv = lib.Server(big, model, max_sessions=4)
    slots = [srv.admit(100, 10, env.lo, env.hi) for _ in range(4)]
    with pytest.raises(lib.MpmiError) as e:
        srv.admit(100, 10, env.lo, env.hi)
    assert e.value.code == -2
    srv.release(slots[1])
    assert srv.admit(100, 10, env.lo, env.hi) == slots[1]
    srv.free()
    # a budget that holds the model, the server and exactly three sessions
    ctx0 = lib.Context(0)
    m0 = gpu_model(lib, ctx0, env)
    s0 = lib.Server(ctx0, m0, max_sessions=8)
    u1 = ctx0.memory_in_use()
    s0.admit(10, 5, env.lo, env.hi)
    per = ctx0.memory_in_use() - u1
    assert per > 0
    s0.free()
    m0.free()
    ctx4 = lib.Context(0, mem_budget=u1 + 3 * per)
    m4 = gpu_model(lib, ctx4, env)
    s4 = lib.Server(ctx4, m4, max_sessions=8)
    got = [s4.admit(10, 5, env.lo, env.hi) for _ in range(3)]
    with pytest.raises(lib.MpmiError) as e:
        s4.admit(10, 5, env.lo, env.hi)
    assert e.value.code == -2
    s4.release(got[0])
    s4.admit(10, 5, env.lo, env.hi)
    s4.free()
    m4.free()


def test_protocol_errors(lib, ctx):
    env = bot_env()
    model = gpu_model(lib, ctx, env)
    srv = lib.Server(ctx, model, max_sessions=4)
    a = srv.admit(500, 10, env.lo, env.hi)
    b = srv.admit(500, 10, env.lo, env.hi)
    with pytest.raises(lib.MpmiError):
        srv.collect()                                   # nothing in flight
    srv.submit([a], [[0.1, 0, 0, 0]], [[0.2]], [0])
    with pytest.raises(lib.MpmiError):
        srv.submit([a], [[0.1, 0, 0, 0]], [[0.2]], [1])  # one request per session
    with pytest.raises(lib.MpmiError):
        srv.release(a)                                  # staged
    with pytest.raises(lib.MpmiError) as e:
        srv.submit([b], [[np.nan, 0, 0, 0]], [[0.2]], [0])
    assert e.value.code == -3
    assert srv.launch() == 1 and srv.in_flight() == 1
    assert srv.launch() == 0                            # nothing staged
    with pytest.raises(lib.MpmiError):
        srv.submit([a], [[0.1, 0, 0, 0]], [[0.2]], [1])  # its request is on the GPU
    with pytest.raises(lib.MpmiError):
        srv.release(a)                                  # on the GPU
    # one batch at a time: the next launch waits for a collect
    srv.set_max_in_flight(1)
    srv.submit([b], [[0.0, 0.1, 0, 0]], [[0.3]], [0])
    with pytest.raises(lib.MpmiError) as e:
        srv.launch()
    assert e.value.code == -5
    assert [s for s, _ in srv.collect()] == [a]
    srv.set_max_in_flight(4)
    assert srv.launch() == 1
    srv.submit([a], [[0.1, 0, 0, 0]], [[0.2]], [1])
    assert srv.launch() == 1 and srv.in_flight() == 2   # two batches of one model
    got = [srv.collect(), srv.collect()]
    assert sorted(s for batch in got for s, _ in batch) == [a, b]
    assert srv.in_flight() == 0
    with pytest.raises(lib.MpmiError):
        srv.set_max_in_flight(5)
    srv.free()
    model.free()


@pytest.mark.parametrize("which", ["bot", "car"])
def test_overlapping_batches_equal_alone(lib, ctx, which):
    """Batches of one model launched while earlier ones are still on the GPU (up
    to four at once) run concurrently; every result is bit-identical to the same
    tick alone, whichever batch carried it and in whatever order they finish."""
    env = bot_env() if which == "bot" else car_env()
    model = gpu_model(lib, ctx, env)
    srv = lib.Server(ctx, model, max_sessions=16)
    rng = np.random.default_rng(5)
    specs = [(65535, 60), (30000, 100), (1023, 20), (7, 5), (4096, 50), (20000, 33),
             (0, 9), (12000, 80)]
    slots = [srv.admit(n, H, env.lo, env.hi, seed=300 + i, stream_id=40 + i)
             for i, (n, H) in enumerate(specs)]
    xs = _states(env, which, len(specs), 21)
    us = data.to_f32_exact(rng.uniform(env.lo, env.hi, (len(specs), len(env.lo))))
    ticks = [500 + 3 * i for i in range(len(specs))]
    groups = [[0, 1], [2, 3], [4, 5, 6], [7]]           # a big batch first, then smaller
    for g in groups:
        srv.submit([slots[i] for i in g], xs[g], us[g], [ticks[i] for i in g])
        assert srv.launch() == len(g)
    assert srv.in_flight() == len(groups)
    got = {}
    for _ in groups:
        for sl, r in srv.collect():
            got[sl] = r
    assert srv.in_flight() == 0 and len(got) == len(specs)
    for i, (n, H) in enumerate(specs):
        a = _alone(lib, ctx, model, env, n, H, 300 + i, 40 + i, xs[i], us[i], ticks[i])
        r = got[slots[i]]
        for k in ("index", "status", "n_safe", "ttv", "executed_steps", "n_slots", "tick"):
            assert r[k] == a[k], (i, k)
        assert np.array_equal(r["u_r"], a["u_r"]) and r["cost"] == a["cost"]
    srv.free()
    model.free()


def test_short_serving_run(lib, ctx):
    import torch
    from paper_1906_02318_gb300 import serve
    benv, cenv = bot_env(), car_env()
    bm, cm = gpu_model(lib, ctx, benv), gpu_model(lib, ctx, cenv)
    bs, cs = lib.Server(ctx, bm, 32), lib.Server(ctx, cm, 32)
    pools = [data.states_in_box(1, 64, [-0.1, -0.3, -0.3, -0.3], [0.1, 0.3, 0.3, 0.3]),
             _states(cenv, "car", 64, 2)]
    meta = [(bs, benv.lo, benv.hi, 0.01), (cs, cenv.lo, cenv.hi, 1 / 60)]
    sessions = serve.make_sessions(meta, 16, 3, pools)
    record = {}
    stats = serve.run([bs, cs], sessions, duration=0.5, record=record)
    assert stats["ticks"] > 100 and stats["batches"] > 0
    for key in ("100Hz", "60Hz"):
        assert stats["latency"][key]["p99_ms"] < 50.0
    # a sample of served results equals the same tick alone
    for (i, k), r in list(record.items())[:6]:
        ss = sessions[i]
        env, model = (benv, bm) if ss.server == 0 else (cenv, cm)
        a = _alone(lib, ctx, model, env, ss.n, ss.horizon, 3 * 1000 + i, i,
                   ss.states[k % len(ss.states)], ss.user[k % len(ss.user)], k)
        assert r["index"] == a["index"] and r["n_safe"] == a["n_safe"]
    bs.free()
    cs.free()


@pytest.mark.parametrize("which,n_shapes", [("bot", 4), ("car", 4)])
def test_tuned_server_results_equal_alone(lib, ctx, which, n_shapes):
    """The server's autotuner tries every compiled serve shape at three block
    sizes on a request mix, keeps the fastest, and served results stay
    bit-identical to the same ticks alone."""
    env = bot_env() if which == "bot" else car_env()
    model = gpu_model(lib, ctx, env)
    srv = lib.Server(ctx, model, max_sessions=16)
    specs = [(1023, 20), (4096, 60), (16384, 50), (2000, 100)]
    xs = _states(env, which, len(specs), 5)
    us = data.to_f32_exact(np.random.default_rng(3).uniform(env.lo, env.hi,
                                                            (len(specs), len(env.lo))))
    reqs = [(n, H, env.lo, env.hi, 200 + i, i) for i, (n, H) in enumerate(specs)]
    r = srv.tune(reqs, xs, us, reps=3)
    assert 1 <= r["n_tried"] <= 3 * n_shapes
    assert r["us"] <= r["default_us"]
    assert r["block"] in (64, 128, 256)
    slots = [srv.admit(n, H, env.lo, env.hi, seed=200 + i, stream_id=i)
             for i, (n, H) in enumerate(specs)]
    srv.submit(slots, xs, us, [7 + i for i in range(len(specs))])
    # tuning needs an empty stage
    with pytest.raises(lib.MpmiError) as e:
        srv.tune(reqs, xs, us, reps=3)
    assert e.value.code == -5
    assert srv.launch() == len(specs)
    got = dict(srv.collect())
    for i, (n, H) in enumerate(specs):
        want = _alone(lib, ctx, model, env, n, H, 200 + i, i, xs[i], us[i], 7 + i)
        res = got[slots[i]]
        for k in ("index", "status", "n_safe", "ttv", "executed_steps", "tick"):
            assert res[k] == want[k], (i, k)
        assert np.array_equal(res["u_r"], want["u_r"])
    with pytest.raises(lib.MpmiError) as e:
        srv.tune(reqs, xs, us, reps=0)
    assert e.value.code == -1
    for sl in slots:
        srv.release(sl)
    srv.free()
    model.free()
