"""Persistent host ticks (mpmi_session_set_persistent, through the C ABI): a
resident kernel fed through a pinned mailbox returns, tick for tick, exactly
the launched tick's result, and the launched tick is checked against the
oracle here too (so the chain persistent == launched ~ oracle is in one place).
Also: exit after the idle limit and relaunch on the next tick, device ticks
interleaved with host ticks, switching on and off, closing a session with the
kernel resident or a tick in flight, ticks that must not take the resident path
(noise, another rollout), the bounded staging wait, and argument checks.

A resident kernel holds the SM resources of its blocks while it waits, so other
work (another session's launched tick, a torch kernel) may have to wait for its
idle limit; the tests take the launched references before switching a session
to resident ticks, or use short idle limits where they interleave."""
import time

import numpy as np
import pytest

from oracle import mpmi as omp
from workloads import data

from parity import bot_env, car_env, compare, gpu_model, oracle_samples, run_gpu

pytestmark = pytest.mark.gpu

FIELDS = ("index", "status", "n_safe", "ttv", "cost", "n_slots", "executed_steps", "tick")


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


@pytest.fixture(scope="module")
def bot(lib, ctx):
    env = bot_env()
    return env, gpu_model(lib, ctx, env)


@pytest.fixture(scope="module")
def car(lib, ctx):
    env = car_env()
    return env, gpu_model(lib, ctx, env)


def _persistent(lib, sess, idle_ms=0.0):
    try:
        sess.set_persistent(True, idle_ms)
    except lib.MpmiError as e:
        if e.code == -6:  # UNSUPPORTED: no host-memory atomics or cooperative launch
            pytest.skip(str(e))
        raise


def _same(a, b):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), (k, a[k], b[k])
    assert np.array_equal(a["u_r"], b["u_r"])


def _inputs(env, which, k):
    rng = np.random.default_rng(100 + k)
    if which == "bot":
        x = rng.uniform([-0.4, -1.0, -1.5, -1.0], [0.4, 1.0, 1.5, 1.0])
    else:
        x = data.car_start_state(env.track, vx=8.0 + k % 10)
        x[:2] += rng.uniform(-2.0, 2.0, 2)
    u = data.to_f32_exact(data.user_input_once(200 + k, env.lo, env.hi))
    return x, u


@pytest.mark.parametrize("which,N,H", [("bot", 16384, 50), ("bot", 3000, 30),
                                       ("car", 16384, 60), ("car", 1000, 60)])
def test_resident_ticks_equal_launched_ticks(lib, ctx, bot, car, which, N, H):
    env, model = bot if which == "bot" else car
    plain = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=21, stream_id=4)
    res = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=21, stream_id=4)
    assert plain.launch_shape() == res.launch_shape()
    ticks = [1000 + 7 * k + (2**33 if k % 5 == 4 else 0) for k in range(25)]
    want = []
    for k, tick in enumerate(ticks):
        x, u = _inputs(env, which, k)
        lib.evaluate_candidates(plain, x, u, tick=tick)
        want.append(lib.select_input(plain))
    plain.close()
    _persistent(lib, res)
    for k, tick in enumerate(ticks):
        x, u = _inputs(env, which, k)
        lib.evaluate_candidates(res, x, u, tick=tick)
        _same(lib.select_input(res), want[k])
    res.close()


@pytest.mark.parametrize("which,N,H", [("bot", 16384, 50), ("car", 16384, 60)])
def test_resident_ticks_with_a_narrow_block(lib, ctx, bot, car, which, N, H):
    """A session with 64-thread blocks: the resident grid (one block per SM)
    widens its blocks until it covers every warp-tile at once; the results stay
    those of the launched ticks with 64-thread blocks."""
    env, model = bot if which == "bot" else car
    plain = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=23, block=64)
    res = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=23, block=64)
    assert plain.launch_shape()[2] == 64
    ticks = [500 + 3 * k for k in range(12)]
    want = []
    for k, tick in enumerate(ticks):
        x, u = _inputs(env, which, k)
        lib.evaluate_candidates(plain, x, u, tick=tick)
        want.append(lib.select_input(plain))
    plain.close()
    _persistent(lib, res)
    for k, tick in enumerate(ticks):
        x, u = _inputs(env, which, k)
        lib.evaluate_candidates(res, x, u, tick=tick)
        _same(lib.select_input(res), want[k])
    res.close()


@pytest.mark.parametrize("which", ["bot", "car"])
def test_resident_tick_against_the_oracle(lib, ctx, bot, car, which):
    env, model = bot if which == "bot" else car
    N, H, seed, tick = 2047, 40, 9, 31
    x, u = _inputs(env, which, 3)
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed)
    g = run_gpu(lib, sess, x, u, tick=tick, traj=True)
    o = omp.tick(env.K32, env.basis, x, u, oracle_samples(env, N, seed, 0, tick), H, env.spec,
                 include_user=True, record=True)
    compare(g, o, env, H)
    _persistent(lib, sess)
    lib.evaluate_candidates(sess, x, u, tick=tick)
    got = lib.select_input(sess)
    _same(got, g["result"])
    sess.close()


def test_idle_exit_and_relaunch(lib, ctx, bot):
    env, model = bot
    plain = lib.Session(ctx, model, 4096, 40, env.lo, env.hi, seed=5)
    want = []
    for k in range(12):
        x, u = _inputs(env, "bot", k)
        lib.evaluate_candidates(plain, x, u, tick=k)
        want.append(lib.select_input(plain))
    plain.close()
    sess = lib.Session(ctx, model, 4096, 40, env.lo, env.hi, seed=5)
    _persistent(lib, sess, idle_ms=2.0)
    for k in range(12):
        x, u = _inputs(env, "bot", k)
        lib.evaluate_candidates(sess, x, u, tick=k)
        _same(lib.select_input(sess), want[k])
        # every other tick comes after the resident kernel has given up waiting
        time.sleep(0.02 if k % 2 else 0.0)
    sess.close()


def test_device_ticks_interleaved_with_resident_host_ticks(lib, ctx, car):
    env, model = car
    sess = lib.Session(ctx, model, 5000, 60, env.lo, env.hi, seed=8)
    plain = lib.Session(ctx, model, 5000, 60, env.lo, env.hi, seed=8)
    _persistent(lib, sess, idle_ms=20.0)
    for k in range(6):
        x, u = _inputs(env, "car", k)
        lib.evaluate_candidates(sess, x, u, tick=k)
        got = lib.select_input(sess)
        dev = run_gpu(lib, sess, x, u, tick=k, traj=False)   # stops the resident kernel
        ref = run_gpu(lib, plain, x, u, tick=k, traj=False)
        _same(got, ref["result"])
        _same(dev["result"], ref["result"])
        assert np.array_equal(dev["ttv"], ref["ttv"])
    sess.close()
    plain.close()


def _launched(lib, ctx, model, env, N, H, seed, cases):
    """Results of launched host ticks on a fresh session, one per (x, u, tick)."""
    plain = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed)
    out = []
    for x, u, tick in cases:
        lib.evaluate_candidates(plain, x, u, tick=tick)
        out.append(lib.select_input(plain))
    plain.close()
    return out


def test_switching_and_closing(lib, ctx, bot):
    env, model = bot
    cases = []
    for k in range(16):
        x, u = _inputs(env, "bot", k)
        cases.append((x, u, 3 + k))
    want = _launched(lib, ctx, model, env, 8192, 50, 2, cases)
    it = iter(range(16))

    def tick(sess):
        k = next(it)
        x, u, t = cases[k]
        lib.evaluate_candidates(sess, x, u, tick=t)
        return k

    sess = lib.Session(ctx, model, 8192, 50, env.lo, env.hi, seed=2)
    _persistent(lib, sess)
    for on in (True, False, True, True, False):
        sess.set_persistent(on)
        k = tick(sess)
        _same(lib.select_input(sess), want[k])
    # a tick in flight survives switching off: it is finished and published first
    sess.set_persistent(True)
    k = tick(sess)
    sess.set_persistent(False)
    _same(lib.select_input(sess), want[k])
    # a new idle limit takes effect on the next tick
    sess.set_persistent(True, 50.0)
    k = tick(sess)
    _same(lib.select_input(sess), want[k])
    # a new tick while one is in flight waits for the first
    tick(sess)
    k = tick(sess)
    _same(lib.select_input(sess), want[k])
    # the reduction record is clean for launched ticks afterwards
    sess.set_persistent(False)
    k = tick(sess)
    _same(lib.select_input(sess), want[k])
    sess.set_persistent(True)
    k = tick(sess)
    _same(lib.select_input(sess), want[k])
    # close with the kernel resident and idle, and with a tick in flight
    sess.close()
    s2 = lib.Session(ctx, model, 8192, 50, env.lo, env.hi, seed=2)
    _persistent(lib, s2)
    tick(s2)
    t0 = time.perf_counter()
    s2.close()
    assert time.perf_counter() - t0 < 5.0
    # the device is still usable
    s3 = lib.Session(ctx, model, 8192, 50, env.lo, env.hi, seed=2)
    k = tick(s3)
    _same(lib.select_input(s3), want[k])
    s3.close()


def test_ticks_outside_the_resident_form_take_launches(lib, ctx, car):
    env, model = car
    x, u = _inputs(env, "car", 2)
    sigma = [0.05, 0.05, 0.01, 0.1]
    sess = lib.Session(ctx, model, 3000, 60, env.lo, env.hi, seed=4)
    ref = lib.Session(ctx, model, 3000, 60, env.lo, env.hi, seed=4)
    _persistent(lib, sess)
    lib.evaluate_candidates(sess, x, u, tick=9)
    lib.select_input(sess)
    for i, setup in enumerate(("noise", "tensor", "factored")):
        for s in (sess, ref):
            if setup == "noise":
                s.set_noise(sigma)
            else:
                s.set_noise([])
                s.set_rollout(setup)
        lib.evaluate_candidates(sess, x, u, tick=10 + i)
        lib.evaluate_candidates(ref, x, u, tick=10 + i)
        _same(lib.select_input(sess), lib.select_input(ref))
    for s in (sess, ref):
        s.set_rollout("full")
    lib.evaluate_candidates(ref, x, u, tick=20)
    want = lib.select_input(ref)
    lib.evaluate_candidates(sess, x, u, tick=20)
    _same(lib.select_input(sess), want)
    sess.close()
    ref.close()


def test_withheld_staging_in_the_resident_kernel(lib, ctx, car):
    env, model = car
    cases = []
    for k in range(5):
        x, u = _inputs(env, "car", 4 + k)
        cases.append((x, u, 1 + k))
    want = _launched(lib, ctx, model, env, 3000, 60, 3, cases)
    sess = lib.Session(ctx, model, 3000, 60, env.lo, env.hi, seed=3)
    _persistent(lib, sess)
    x, u, t = cases[0]
    lib.evaluate_candidates(sess, x, u, tick=t)
    _same(lib.select_input(sess), want[0])
    sess.withhold_staging(True)
    t0 = time.perf_counter()
    x, u, t = cases[1]
    lib.evaluate_candidates(sess, x, u, tick=t)
    with pytest.raises(lib.MpmiError) as e:
        lib.select_input(sess)
    assert e.value.code == -7
    assert time.perf_counter() - t0 < 30.0
    sess.withhold_staging(False)
    for k in (2, 3):
        x, u, t = cases[k]
        lib.evaluate_candidates(sess, x, u, tick=t)
        _same(lib.select_input(sess), want[k])
    # and a launched tick on the same reduction record
    sess.set_persistent(False)
    x, u, t = cases[4]
    lib.evaluate_candidates(sess, x, u, tick=t)
    _same(lib.select_input(sess), want[4])
    sess.close()


@pytest.mark.parametrize("case", ["bot_grid", "bot_no_user", "car_inflated", "linear_22",
                                  "bot_max_horizon", "car_ragged"])
def test_resident_ticks_across_session_kinds(lib, ctx, bot, car, case):
    """Samplers, the user slot, the inflated barrier, the linear bases, the longest
    horizon and ragged slot counts: resident ticks equal launched ticks."""
    models = []
    if case == "bot_grid":
        env, model = bot
        kw = dict(n=4096, H=50, sampler="grid")
    elif case == "bot_no_user":
        env, model = bot
        kw = dict(n=3000, H=40, include_user=False)
    elif case == "car_inflated":
        env = car_env(inflation=0.5)
        model = gpu_model(lib, ctx, env)
        models.append(model)
        kw = dict(n=2500, H=60)
    elif case == "linear_22":
        K = np.array([[1.0, 0.0, 0.05, 0.0], [0.0, 1.0, 0.0, 0.05],
                      [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]])
        model = lib.model_from_operator(ctx, "linear", K, nx=2, nu=2)
        lib.set_safety_set(model, [-1.0, -1.0], [1.0, 1.0])
        models.append(model)
        env = None
        kw = dict(n=5000, H=80)
    elif case == "bot_max_horizon":
        env, model = bot
        kw = dict(n=1000, H=511)
    else:
        env, model = car
        kw = dict(n=16384 + 77, H=60)
    lo = env.lo if env is not None else [-1.0, -1.0]
    hi = env.hi if env is not None else [1.0, 1.0]
    n, H = kw.pop("n"), kw.pop("H")
    rng = np.random.default_rng(7)
    cases = []
    for k in range(6):
        if env is None:
            x = rng.uniform(-0.8, 0.8, 2)
            u = data.to_f32_exact(rng.uniform(-1.0, 1.0, 2))
        else:
            x, u = _inputs(env, "bot" if env.basis == "bot" else "car", 10 + k)
        cases.append((x, u, 40 + 3 * k))
    plain = lib.Session(ctx, model, n, H, lo, hi, seed=13, **kw)
    want = []
    for x, u, t in cases:
        lib.evaluate_candidates(plain, x, u, tick=t)
        want.append(lib.select_input(plain))
    plain.close()
    sess = lib.Session(ctx, model, n, H, lo, hi, seed=13, **kw)
    _persistent(lib, sess)
    for (x, u, t), w in zip(cases, want):
        lib.evaluate_candidates(sess, x, u, tick=t)
        _same(lib.select_input(sess), w)
    sess.close()
    for m in models:
        m.free()


def test_argument_checks(lib, ctx, bot):
    env, model = bot
    sess = lib.Session(ctx, model, 100, 10, env.lo, env.hi)
    for bad in (0.5, -1.0, 60001.0, float("nan"), float("inf")):
        with pytest.raises(lib.MpmiError) as e:
            sess.set_persistent(True, bad)
        assert e.value.code == -1
    sess.set_persistent(False)   # off when never on: nothing to do
    sess.close()
