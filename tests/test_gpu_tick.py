"""Parity of the CUDA tick (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

from oracle import mpmi as omp
from oracle import safety as osafe
from oracle import sampling as osamp
from workloads import data, plants

from parity import (bot_env, car_env, compare, gpu_model, oracle_samples, run_gpu)

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


@pytest.fixture(scope="module")
def bot(lib, ctx):
    env = bot_env()
    return env, gpu_model(lib, ctx, env)


@pytest.fixture(scope="module")
def car(lib, ctx):
    env = car_env()
    return env, gpu_model(lib, ctx, env)


def _tick(lib, ctx, env, model, x_t, u_h, N, H, seed=1, stream=0, tick=0, lanes=0,
          include_user=True, sampler="uniform", block=0, traj=True, cands=0):
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, include_user=include_user,
                       sampler=sampler, seed=seed, stream_id=stream, lanes=lanes, block=block,
                       cands=cands)
    try:
        g = run_gpu(lib, sess, x_t, u_h, tick=tick, traj=traj)
    finally:
        sess.close()
    samples = oracle_samples(env, N, seed, stream, tick, sampler)
    o = omp.tick(env.K32, env.basis, x_t, u_h, samples, H, env.spec,
                 include_user=include_user, record=True)
    return g, o


# --------------------------------------------------------------- Alg. 2 first step
def test_device_philox_known_answer_vectors(lib):
    """The device generator behind every sampled candidate reproduces the
    published Philox4x32-10 known-answer vectors word for word."""
    import json
    import os
    import torch
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")) as f:
        cases = json.load(f)["cases"]
    rec = np.array([[int(w, 16) for w in c["counter"] + c["key"]] for c in cases],
                   dtype=np.uint32)
    want = np.array([[int(w, 16) for w in c["expected"]] for c in cases], dtype=np.uint32)
    rec_dev = torch.from_numpy(rec.view(np.int32)).cuda()
    out = torch.zeros((len(cases), 4), dtype=torch.int32, device="cuda")
    lib.debug_philox(rec_dev, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("which", ["bot", "car"])
@pytest.mark.parametrize("sampler", ["uniform", "grid"])
@pytest.mark.parametrize("include_user", [True, False])
def test_candidates_bit_exact(lib, ctx, bot, car, which, sampler, include_user):
    import torch
    env, model = bot if which == "bot" else car
    N = 4096 if sampler == "grid" and which == "car" else 5000
    if sampler == "grid" and which == "car":
        N = 64 * 64
    for seed, stream, tick in [(1, 0, 0), (0xDEADBEEF12345, 7, 3), (5, 2**31, 2**40 + 5)]:
        sess = lib.Session(ctx, model, N, 10, env.lo, env.hi, include_user=include_user,
                           sampler=sampler, seed=seed, stream_id=stream)
        u_h = data.to_f32_exact(data.user_input_once(seed, env.lo, env.hi))
        out = torch.zeros((sess.n_slots, sess.nu), dtype=torch.float32, device="cuda")
        uh = torch.tensor(u_h, dtype=torch.float64, device="cuda")
        lib.sample_candidates(sess, out, u_h_dev=uh, tick=tick)
        torch.cuda.synchronize()
        sess.close()
        want = omp.candidate_slots(u_h, oracle_samples(env, N, seed, stream, tick, sampler),
                                   include_user)
        got = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(got, want)


def test_external_candidates_are_used(lib, ctx, bot):
    import torch
    env, model = bot
    rng = np.random.default_rng(3)
    cand = data.to_f32_exact(rng.uniform(-1, 1, (777, 1)))
    dev = torch.tensor(cand, dtype=torch.float32, device="cuda")
    sess = lib.Session(ctx, model, 777, 30, env.lo, env.hi, sampler="external")
    x_t = np.array([0.15, 0.4, 0.5, -0.2])
    u_h = np.array([0.8125])
    g = run_gpu(lib, sess, x_t, u_h, traj=True, candidates=dev)
    sess.close()
    o = omp.tick(env.K32, "bot", x_t, u_h, cand, 30, env.spec, record=True)
    compare(g, o, env, 30)


@pytest.mark.parametrize("include_user", [True, False])
def test_exact_ties_pick_the_lowest_slot(lib, ctx, bot, include_user):
    """Caller samples drawn from four values, so every cost is one of three exact
    values and each is shared by hundreds of slots: the pick is the lowest slot
    of the least-cost safe group, as in the oracle, and u_h itself (cost 0) wins
    when it is a slot."""
    import torch
    env, model = bot
    rng = np.random.default_rng(21)
    cand = rng.choice(np.array([-0.5, -0.25, 0.25, 0.5]), size=(3001, 1))
    dev = torch.tensor(cand, dtype=torch.float32, device="cuda")
    sess = lib.Session(ctx, model, 3001, 30, env.lo, env.hi, sampler="external",
                       include_user=include_user)
    for k, x_t in enumerate([np.array([0.05, 0.0, 0.0, 0.0]), np.array([0.2, 0.4, 0.3, 0.1])]):
        u_h = np.array([0.0]) if k == 0 else np.array([0.25])
        g = run_gpu(lib, sess, x_t, u_h, traj=True, candidates=dev)
        o = omp.tick(env.K32, "bot", x_t, u_h, cand, 30, env.spec, include_user=include_user,
                     record=True)
        compare(g, o, env, 30)
        assert g["result"]["index"] == o.index
        if include_user and o.ttv[0] == 30:
            assert o.index == 0
        else:
            # the lowest slot among the safe candidates of least cost
            safe = np.nonzero(o.ttv == 30)[0]
            best = safe[o.cost[safe] == o.cost[safe].min()]
            assert o.index == int(best.min()) and len(best) > 100
    sess.close()


# ------------------------------------------------------------------ balance bot
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_bot_single_tick_paper_scale(lib, ctx, bot, lanes):
    """N = 1024, H = 20 from x_t = (0.1, 0, 0, 0), one user input from the seed."""
    env, model = bot
    u_h = data.to_f32_exact(data.user_input_once(1, env.lo, env.hi))
    g, o = _tick(lib, ctx, env, model, np.array([0.1, 0, 0, 0]), u_h, 1024, 20, lanes=lanes)
    compare(g, o, env, 20)
    assert g["result"]["index"] == o.index


@pytest.mark.parametrize("lanes,cands", [(1, 1), (1, 2), (2, 1), (4, 1)])
@pytest.mark.parametrize("N", [1, 31, 1000, 3001])
def test_bot_states_ragged(lib, ctx, bot, lanes, cands, N):
    env, model = bot
    states = data.states_in_box(11, 6, [-0.45, -1.5, -1.8, -1.5], [0.45, 1.5, 1.8, 1.5])
    excused = 0
    for k, x_t in enumerate(states):
        u_h = data.to_f32_exact(data.user_input_once(100 + k, env.lo, env.hi))
        g, o = _tick(lib, ctx, env, model, x_t, u_h, N, 50, seed=k, tick=k, lanes=lanes,
                     cands=cands)
        excused += compare(g, o, env, 50)
    assert excused <= max(2, 0.002 * N * len(states))


def test_bot_full_size(lib, ctx, bot):
    """N = 16384, H = 50 in the launch configuration the benchmark uses."""
    env, model = bot
    for k, x_t in enumerate([np.array([0.05, 0.0, 0.0, 0.0]), np.array([0.3, 0.9, 1.2, 0.6])]):
        u_h = data.to_f32_exact(data.user_input_once(200 + k, env.lo, env.hi))
        g, o = _tick(lib, ctx, env, model, x_t, u_h, 16384, 50, seed=2, tick=k)
        assert compare(g, o, env, 50) <= 0.002 * 16385


def test_bot_inflated_barrier(lib, ctx):
    import paper_1906_02318_gb300.mpmi as lib_
    env = bot_env(inflation=0.1)
    c = lib_.Context(0)
    model = gpu_model(lib_, c, env)
    x_t = np.array([0.2, 0.5, 1.0, 0.3])
    g, o = _tick(lib_, c, env, model, x_t, [0.25], 4096, 40)
    compare(g, o, env, 40)
    model.free()


# ------------------------------------------------------------------- race car
@pytest.mark.parametrize("lanes,cands", [(1, 1), (1, 2), (2, 1), (4, 1), (8, 1), (16, 1)])
def test_car_ticks(lib, ctx, car, lanes, cands):
    env, model = car
    x0 = data.car_start_state(env.track, vx=14.0)
    states = [x0, x0 + np.array([1.5, -1.0, 0.1, 4.0, 0.3, 0.2]),
              x0 + np.array([-2.0, 2.5, -0.2, -6.0, -0.2, -0.1])]
    for k, x_t in enumerate(states):
        u_h = data.to_f32_exact(data.user_input_once(300 + k, env.lo, env.hi))
        g, o = _tick(lib, ctx, env, model, x_t, u_h, 2047, 60, seed=3, tick=k, lanes=lanes,
                     cands=cands)
        assert compare(g, o, env, 60) <= 10


@pytest.mark.parametrize("lanes,cands", [(1, 1), (1, 2), (2, 1), (4, 1), (8, 1), (16, 1)])
@pytest.mark.parametrize("N", [0, 1, 33, 129])
def test_car_ragged_sizes(lib, ctx, car, lanes, cands, N):
    """Few and ragged slot counts (the user's slot alone, one sample, partial warp
    tiles and pairs) in every race-car launch shape, trajectories and all."""
    env, model = car
    x0 = data.car_start_state(env.track, vx=13.0)
    states = [x0, x0 + np.array([1.0, -1.5, 0.08, 3.0, 0.2, 0.1])]
    excused = 0
    for k, x_t in enumerate(states):
        u_h = data.to_f32_exact(data.user_input_once(400 + k, env.lo, env.hi))
        g, o = _tick(lib, ctx, env, model, x_t, u_h, N, 60, seed=4, tick=k, lanes=lanes,
                     cands=cands)
        assert g["result"]["n_slots"] == N + 1
        excused += compare(g, o, env, 60)
    assert excused <= 2


@pytest.mark.slow
def test_car_full_size(lib, ctx, car):
    """N = 16384, H = 60 in the default launch configuration."""
    env, model = car
    x_t = data.car_start_state(env.track, vx=12.0)
    u_h = data.to_f32_exact(data.user_input_once(3, env.lo, env.hi))
    g, o = _tick(lib, ctx, env, model, x_t, u_h, 16384, 60, seed=3)
    assert compare(g, o, env, 60) <= 0.002 * 16385


@pytest.mark.slow
def test_car_learned_config_full_size(lib, ctx, car):
    """N = 65536, H = 60 in the default launch configuration at that size (the
    learned-screener comparison's plain tick): the pick is the lexicographic
    minimum of the GPU's own per-candidate outputs, and sampled slots (the user's,
    the first and last 64 and 256 others) agree with the oracle except at a safety
    boundary."""
    env, model = car
    N, H, seed, tick = 65536, 60, 3, 7
    x_t = data.car_start_state(env.track, vx=12.0)
    u_h = data.to_f32_exact(data.user_input_once(4, env.lo, env.hi))
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed)
    g = run_gpu(lib, sess, x_t, u_h, tick=tick)
    sess.close()
    ttv, cost, r = g["ttv"], g["cost"], g["result"]
    slots = np.arange(N + 1)
    order = np.lexsort((slots, cost.astype(np.float64), H - ttv))
    assert r["index"] == int(order[0]) and r["n_slots"] == N + 1
    assert r["n_safe"] == int(np.count_nonzero(ttv == H))
    assert r["executed_steps"] == int(np.minimum(ttv + 1, H).sum())
    samples = oracle_samples(env, N, seed, 0, tick)
    pick = np.unique(np.concatenate([np.arange(1, 65), np.arange(N - 63, N + 1),
                                     np.random.default_rng(1).integers(1, N + 1, 256)]))
    o = omp.tick(env.K32, env.basis, x_t, u_h, samples[pick - 1], H, env.spec, record=True)
    got = np.concatenate([[0], pick])        # the oracle's slot 0 is the user's input
    assert np.allclose(cost[got], o.cost, rtol=1e-6, atol=1e-12)
    for i in np.nonzero(ttv[got] != o.ttv)[0]:  # only at a safety boundary
        s_ = int(min(ttv[got[i]], o.ttv[i])) + 1
        marg = float(osafe.margin(env.spec, o.traj[i, s_][None, :])[0])
        assert abs(marg) < 1e-4 * max(1.0, float(np.abs(o.traj[i, s_]).max()))
    assert np.count_nonzero(ttv[got] != o.ttv) <= 2


# ------------------------------------------------------------ closed forms on GPU
def test_drift_model_closed_form(lib, ctx):
    """x' = x + dt u (linear basis n = 2): ttv has a closed form per candidate."""
    dt, H, x0 = 0.05, 40, 0.3137
    K = np.array([[1.0, dt], [0.0, 1.0]])
    m = lib.model_from_operator(ctx, "linear", K, nx=1, nu=1)
    lib.set_safety_set(m, [-1.0], [1.0])
    sess = lib.Session(ctx, m, 5000, H, [-1.0], [1.0], seed=9)
    g = run_gpu(lib, sess, [x0], [0.9])
    sess.close()
    cand = omp.candidate_slots([0.9], osamp.uniform_samples(9, 0, 0, 5000, [-1], [1]), True)
    K32 = np.float32(K).astype(np.float64)
    want = []
    for c in cand[:, 0]:
        # exit step of x0 + t*dt*c in float64 with the float32 operator
        t_exit = None
        x = x0
        for t in range(1, H + 1):
            x = K32[0, 0] * x + K32[0, 1] * c
            if not (-1.0 < x < 1.0):
                t_exit = t
                break
        want.append(H if t_exit is None else t_exit - 1)
    want = np.array(want)
    close = np.abs(np.abs(x0 + np.arange(1, H + 1)[None, :] * dt * cand) - 1.0).min(axis=1) < 1e-5
    assert np.all((g["ttv"] == want) | close)
    m.free()


def test_identity_model_stays_constant(lib, ctx):
    import torch
    K = np.eye(5)
    m = lib.model_from_operator(ctx, "linear", K, nx=4, nu=1)
    lib.set_safety_set(m, [-1.0, -1, -1, -1], [1.0, 1, 1, 1])
    sess = lib.Session(ctx, m, 300, 511, [-1.0], [1.0], seed=4)
    x_t = np.array([0.5, -0.25, 0.125, 0.0])
    g = run_gpu(lib, sess, x_t, [0.0], traj=True)
    sess.close()
    assert np.all(g["ttv"] == 511) and g["result"]["status"] == lib.SAFE
    z0 = g["traj"][:, :1, :]
    assert np.array_equal(g["traj"], np.broadcast_to(z0, g["traj"].shape))
    assert g["result"]["index"] == 0 and g["result"]["u_r"][0] == 0.0
    m.free()


def test_eq2_grid_bound_on_gpu(lib, ctx):
    """Sec. IV-D, Eq. 2: with the grid and every candidate safe, the deviation
    from u_h is at most lambda / (2N) (M = 1)."""
    m = lib.model_from_operator(ctx, "linear", np.eye(2), nx=1, nu=1)
    lib.set_safety_set(m, [-np.inf], [np.inf])
    N = 10000
    sess = lib.Session(ctx, m, N, 3, [-1.0], [1.0], include_user=False, sampler="grid")
    worst = 0.0
    for k, u in enumerate(np.concatenate([np.random.default_rng(0).uniform(-1, 1, 30),
                                          [-1.0, 1.0]])):
        lib.evaluate_candidates(sess, [0.0], [u], tick=k)
        r = lib.select_input(sess)
        assert r["status"] == lib.SAFE and r["n_safe"] == N
        worst = max(worst, abs(r["u_r"][0] - u))
    sess.close()
    assert worst <= 2.0 / (2 * N) * (1 + 1e-6) + 2 ** -24
    assert worst >= 2.0 / (2 * N) * (1 - 1e-3)
    m.free()


# ------------------------------------------------------------------ edge cases
def test_only_user_slot(lib, ctx, bot):
    env, model = bot
    g, o = _tick(lib, ctx, env, model, np.array([0.1, 0, 0, 0]), [0.25], 0, 20)
    compare(g, o, env, 20)
    assert g["result"]["index"] == 0 and g["result"]["n_slots"] == 1


def test_single_step_horizon_and_no_user_slot(lib, ctx, bot):
    env, model = bot
    x_t = np.array([0.49, 0.5, 1.99, 0.5])
    g, o = _tick(lib, ctx, env, model, x_t, [0.5], 999, 1, include_user=False)
    compare(g, o, env, 1, include_user=False)


def test_all_unsafe_falls_back(lib, ctx, bot):
    env, model = bot
    x_t = np.array([0.7, 2.0, 0.0, 0.0])   # already past the barrier: every step fails
    g, o = _tick(lib, ctx, env, model, x_t, [0.5], 2048, 30)
    compare(g, o, env, 30)
    r = g["result"]
    assert r["status"] == lib.FALLBACK and r["n_safe"] == 0
    assert o.status == omp.FALLBACK


def test_safe_user_input_passes_through(lib, ctx, bot):
    env, model = bot
    sess = lib.Session(ctx, model, 4096, 20, env.lo, env.hi)
    u_h = 0.0123456789012345
    lib.evaluate_candidates(sess, [0.0, 0.0, 0.0, 0.0], [u_h])
    r = lib.select_input(sess)
    sess.close()
    assert r["index"] == 0 and r["status"] == lib.SAFE and r["u_r"][0] == u_h


def test_nonfinite_inputs(lib, ctx, bot):
    import torch
    env, model = bot
    sess = lib.Session(ctx, model, 512, 20, env.lo, env.hi)
    with pytest.raises(lib.MpmiError) as e:
        lib.evaluate_candidates(sess, [np.nan, 0, 0, 0], [0.0])
    assert e.value.code == -3
    with pytest.raises(lib.MpmiError) as e:
        lib.select_input(sess)
    assert e.value.code == -5
    # the device path treats NaN as unsafe: every candidate fails at step 1
    g = run_gpu(lib, sess, [np.nan, 0, 0, 0], [0.0])
    sess.close()
    assert np.all(g["ttv"] == 0) and g["result"]["status"] == lib.FALLBACK
    assert g["result"]["index"] == 0 and g["result"]["n_safe"] == 0


def test_host_and_device_paths_agree_and_repeat(lib, ctx, bot):
    env, model = bot
    sess = lib.Session(ctx, model, 8192, 50, env.lo, env.hi, seed=12)
    x_t, u_h = np.array([0.2, -0.3, 0.4, 0.1]), np.array([-0.625])
    outs = []
    for _ in range(3):
        lib.evaluate_candidates(sess, x_t, u_h, tick=77)
        outs.append(lib.select_input(sess))
    g = run_gpu(lib, sess, x_t, u_h, tick=77, traj=False)
    sess.close()
    for r in outs[1:] + [g["result"]]:
        for k in ("index", "status", "n_safe", "ttv", "executed_steps"):
            assert r[k] == outs[0][k]
        assert np.array_equal(r["u_r"], outs[0]["u_r"])


def test_session_argument_checks(lib, ctx, bot):
    env, model = bot
    bad = [dict(n_samples=-1, horizon=10), dict(n_samples=10, horizon=0),
           dict(n_samples=10, horizon=512), dict(n_samples=0, horizon=5, include_user=False),
           dict(n_samples=10, horizon=5, lanes=3), dict(n_samples=10, horizon=5, block=100)]
    for kw in bad:
        kw = dict(kw)
        with pytest.raises(lib.MpmiError):
            lib.Session(ctx, model, kw.pop("n_samples"), kw.pop("horizon"), env.lo, env.hi, **kw)
    with pytest.raises(lib.MpmiError):
        lib.Session(ctx, model, 10, 5, [0.5], [-0.5])     # empty input box
    with pytest.raises(lib.MpmiError):
        lib.Session(ctx, model, 10, 5, env.lo, env.hi, lanes=2, cands=2)  # not compiled


def test_grid_needs_a_perfect_power(lib, ctx, car):
    env, model = car
    with pytest.raises(lib.MpmiError):
        lib.Session(ctx, model, 10, 5, env.lo, env.hi, sampler="grid")   # 10 != G^2
    lib.Session(ctx, model, 49, 5, env.lo, env.hi, sampler="grid").close()


def test_memory_budget_admission(lib):
    env = bot_env()
    small = lib.Context(0, mem_budget=2048)
    model = gpu_model(lib, small, env)
    s1 = lib.Session(small, model, 100, 10, env.lo, env.hi)
    held = []  # open sessions keep their memory (a dropped session is closed)
    with pytest.raises(lib.MpmiError) as e:
        for _ in range(20):
            held.append(lib.Session(small, model, 100, 10, env.lo, env.hi))
    assert e.value.code == -2
    used = small.memory_in_use()
    for s in held:
        s.close()
    assert small.memory_in_use() < used
    # room again once sessions are closed
    lib.Session(small, model, 100, 10, env.lo, env.hi).close()
    s1.close()


def test_fit_model_on_device_matches_host_fit(lib, ctx):
    x, u, xn = data.transitions("bot", 1, 5000)
    m, res = lib.fit_model(ctx, "bot", x, u, xn)
    K_host, res_host = lib.fit_operator("bot", x, u, xn)
    assert np.array_equal(m.get_operator(), K_host) and res == res_host
    m.free()


# ------------------------------------------------------------- closed loop
def test_bot_closed_loop_matches_oracle(lib, ctx, bot):
    """Receding horizon (Sec. IV-C): each side drives its own plant copy from the
    same start with the same user input; the applied inputs agree tick by tick."""
    env, model = bot
    ticks, N, H = 150, 2048, 50
    u_seq = data.to_f32_exact(data.ou_user_input(2, ticks, plants.BOT_DT, env.lo, env.hi))
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=2)
    x = np.array([0.05, 0.0, 0.0, 0.0])
    gpu_u = []
    for t in range(ticks):
        lib.evaluate_candidates(sess, x, u_seq[t], tick=t)
        r = lib.select_input(sess)
        gpu_u.append(r["u_r"].copy())
        x = plants.cartpole_step(x, r["u_r"])
    sess.close()
    recs = omp.closed_loop(env.K32, "bot", env.spec, plants.cartpole_step,
                           [0.05, 0.0, 0.0, 0.0], u_seq,
                           lambda t: osamp.uniform_samples(2, 0, t, N, env.lo, env.hi), H)
    agree = 0
    for t, (_, _, o) in enumerate(recs):
        if not np.array_equal(gpu_u[t], o.u_r):
            break
        agree += 1
    assert agree >= ticks * 0.9, f"closed loops diverged at tick {agree}"


def test_car_closed_loop_matches_oracle(lib, ctx, car):
    """The race car's receding horizon (Sec. IV-C, V-B) for one second at 60 Hz:
    each side drives its own bicycle copy around the track from the same start
    with the same user input; the applied inputs agree tick by tick."""
    env, model = car
    ticks, N, H = 60, 511, 60
    u_seq = data.to_f32_exact(data.ou_user_input(4, ticks, plants.CAR_DT, env.lo, env.hi))
    x0 = data.car_start_state(env.track, vx=12.0)
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=4)
    x = x0.copy()
    gpu_u = []
    for t in range(ticks):
        lib.evaluate_candidates(sess, x, u_seq[t], tick=t)
        r = lib.select_input(sess)
        gpu_u.append(r["u_r"].copy())
        x = plants.bicycle_step(x, r["u_r"])
    sess.close()
    recs = omp.closed_loop(env.K32, "car", env.spec, plants.bicycle_step, x0, u_seq,
                           lambda t: osamp.uniform_samples(4, 0, t, N, env.lo, env.hi), H)
    agree = 0
    for t, (_, _, o) in enumerate(recs):
        if not np.array_equal(gpu_u[t], o.u_r):
            break
        agree += 1
    assert agree >= ticks * 0.9, f"closed loops diverged at tick {agree}"


@pytest.mark.parametrize("which", ["bot", "car"])
def test_all_launch_shapes_agree_bit_for_bit(lib, ctx, bot, car, which):
    """Every compiled launch shape sums each row of K z in the same order, so the
    per-candidate outcomes and the selection are identical across shapes."""
    env, model = bot if which == "bot" else car
    shapes = [(1, 1), (1, 2), (2, 1), (4, 1)] if which == "bot" else [(1, 1), (1, 2), (2, 1),
                                                                        (4, 1), (8, 1), (16, 1)]
    H = 50 if which == "bot" else 60
    x_t = (np.array([0.3, 0.9, 1.2, 0.6]) if which == "bot"
           else data.car_start_state(env.track, vx=15.0) + np.array([1.0, -0.5, 0.05, 0, 0, 0]))
    u_h = data.to_f32_exact(data.user_input_once(77, env.lo, env.hi))
    outs = []
    for lanes, cands in shapes:
        sess = lib.Session(ctx, model, 5000, H, env.lo, env.hi, seed=21, lanes=lanes,
                           cands=cands)
        outs.append(run_gpu(lib, sess, x_t, u_h, tick=4))
        sess.close()
    for o in outs[1:]:
        assert np.array_equal(o["ttv"], outs[0]["ttv"])
        assert np.array_equal(o["cost"], outs[0]["cost"])
        for k in ("index", "status", "n_safe", "executed_steps"):
            assert o["result"][k] == outs[0]["result"][k]


def test_operator_held_rows_checked_and_set_exact(lib, ctx, bot):
    """Rows of held input features (u and the constant for the balance bot) must
    be unit rows: rounding-level deviations are set exact, others refused."""
    env, _ = bot
    K = env.K32.copy()
    K[4, 2] += 1e-9
    K[11, 11] -= 1e-9
    m = lib.model_from_operator(ctx, "bot", K)
    got = m.get_operator()
    assert np.array_equal(got[4], np.eye(12)[4]) and np.array_equal(got[11], np.eye(12)[11])
    assert np.array_equal(got[:4], K[:4])
    m.free()
    K[4, 2] += 1e-3
    with pytest.raises(lib.MpmiError) as e:
        lib.model_from_operator(ctx, "bot", K)
    assert e.value.code == -1


def test_sparse_basis_model_ticks(lib, ctx):
    """A model whose basis was selected by the sparsity-promoting fit (race car,
    gamma = 1: 24 of 32 features kept) runs the same tick; parity with the
    oracle's tick of the same operator."""
    from oracle import fit as ofit
    from parity import Env
    x, u, xn = data.transitions("car", 3, 20000)
    Ko, sup, _ = ofit.fit_koopman_sparse("car", x, u, xn, 1.0)
    assert 0 < sup.sum() < 32
    base = car_env()
    env = Env("car", ofit.round_to_f32(Ko), base.spec, base.lo, base.hi, base.track)
    model = gpu_model(lib, ctx, env)
    x0 = data.car_start_state(env.track, vx=14.0)
    for k, x_t in enumerate([x0, x0 + np.array([1.5, -1.0, 0.1, 4.0, 0.3, 0.2])]):
        u_h = data.to_f32_exact(data.user_input_once(900 + k, env.lo, env.hi))
        g, o = _tick(lib, ctx, env, model, x_t, u_h, 2047, 60, seed=5, tick=k)
        assert compare(g, o, env, 60) <= 10
    model.free()


@pytest.mark.slow
def test_maximum_slot_count(lib, ctx, bot):
    """2^23 - 1 candidate slots (the key's 23-bit slot field full): the pick is the
    lexicographic minimum of the GPU's own per-candidate outputs, sampled slots
    (the last ones included) agree with the oracle, one more slot is refused."""
    import torch
    env, model = bot
    N, H = lib.MAX_SLOTS - 1, 5
    x_t = np.array([0.2, 0.6, -0.5, 0.3])
    u_h = data.to_f32_exact(data.user_input_once(13, env.lo, env.hi))
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=17, stream_id=5)
    g = run_gpu(lib, sess, x_t, u_h, tick=3)
    sess.close()
    ttv, cost, r = g["ttv"], g["cost"], g["result"]
    assert r["n_slots"] == lib.MAX_SLOTS and ttv.size == lib.MAX_SLOTS
    slots = np.arange(ttv.size)
    order = np.lexsort((slots, cost.astype(np.float64), H - ttv))
    assert r["index"] == int(order[0])
    assert r["n_safe"] == int(np.count_nonzero(ttv == H))
    assert r["executed_steps"] == int(np.minimum(ttv + 1, H).sum())
    # sampled slots against the oracle (samples are slots 1..N)
    samples = osamp.uniform_samples(17, 5, 3, N, env.lo, env.hi)
    pick = np.unique(np.concatenate([np.arange(N - 64, N + 1), np.arange(1, 65),
                                     np.random.default_rng(0).integers(1, N + 1, 256)]))
    o = omp.tick(env.K32, env.basis, x_t, u_h, samples[pick - 1], H, env.spec,
                 include_user=False, record=True)
    assert np.allclose(cost[pick], o.cost, rtol=1e-6, atol=1e-12)
    mism = np.nonzero(ttv[pick] != o.ttv)[0]
    for i in mism:                                   # only at a safety boundary
        s = int(min(ttv[pick[i]], o.ttv[i])) + 1
        marg = float(osafe.margin(env.spec, o.traj[i, s][None, :])[0])
        assert abs(marg) < 1e-4 * max(1.0, float(np.abs(o.traj[i, s]).max()))
    with pytest.raises(lib.MpmiError) as e:
        lib.Session(ctx, model, lib.MAX_SLOTS, H, env.lo, env.hi)
    assert e.value.code == -1


@pytest.mark.slow
def test_car_maximum_slot_count(lib, ctx, car):
    """The race car at 2^23 - 1 slots (the key's slot field full) in its default
    launch shape: the pick is the lexicographic minimum of the GPU's own outputs and
    sampled slots (the last ones included) agree with the oracle, track test and
    all, except at a safety boundary."""
    env, model = car
    N, H = lib.MAX_SLOTS - 1, 8
    x_t = data.car_start_state(env.track, vx=15.0)
    u_h = data.to_f32_exact(data.user_input_once(14, env.lo, env.hi))
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=19, stream_id=2)
    g = run_gpu(lib, sess, x_t, u_h, tick=5)
    sess.close()
    ttv, cost, r = g["ttv"], g["cost"], g["result"]
    assert r["n_slots"] == lib.MAX_SLOTS and ttv.size == lib.MAX_SLOTS
    slots = np.arange(ttv.size)
    order = np.lexsort((slots, cost.astype(np.float64), H - ttv))
    assert r["index"] == int(order[0])
    assert r["n_safe"] == int(np.count_nonzero(ttv == H))
    assert r["executed_steps"] == int(np.minimum(ttv + 1, H).sum())
    samples = osamp.uniform_samples(19, 2, 5, N, env.lo, env.hi)
    pick = np.unique(np.concatenate([np.arange(N - 31, N + 1), np.arange(1, 33),
                                     np.random.default_rng(2).integers(1, N + 1, 128)]))
    o = omp.tick(env.K32, env.basis, x_t, u_h, samples[pick - 1], H, env.spec,
                 include_user=False, record=True)
    assert np.allclose(cost[pick], o.cost, rtol=1e-6, atol=1e-12)
    for i in np.nonzero(ttv[pick] != o.ttv)[0]:   # only at a safety boundary
        s_ = int(min(ttv[pick[i]], o.ttv[i])) + 1
        marg = float(osafe.margin(env.spec, o.traj[i, s_][None, :])[0])
        assert abs(marg) < 1e-4 * max(1.0, float(np.abs(o.traj[i, s_]).max()))


@pytest.mark.parametrize("inflation", [0.5, 1.5])
@pytest.mark.parametrize("rollout", ["full", "tensor", "factored"])
def test_car_inflated_barrier(lib, ctx, inflation, rollout):
    """Sec. V-C.1's inflated barrier on the race car: the road narrows to w - iota
    (the grid is rebuilt for it) and the box bounds tighten by iota; every rollout
    form against the oracle."""
    env = car_env(inflation=inflation)
    model = gpu_model(lib, ctx, env)
    x0 = data.car_start_state(env.track, vx=14.0)
    for k, x_t in enumerate([x0, x0 + np.array([1.0, -0.8, 0.1, 3.0, 0.3, 0.2])]):
        u_h = data.to_f32_exact(data.user_input_once(800 + k, env.lo, env.hi))
        sess = lib.Session(ctx, model, 2047, 60, env.lo, env.hi, seed=6, stream_id=k)
        sess.set_rollout(rollout)
        g = run_gpu(lib, sess, x_t, u_h, tick=k, traj=rollout != "factored")
        sess.close()
        o = omp.tick(env.K32, "car", x_t, u_h, oracle_samples(env, 2047, 6, k, k), 60, env.spec,
                     record=True)
        assert compare(g, o, env, 60) <= 10
        free = omp.tick(env.K32, "car", x_t, u_h, oracle_samples(env, 2047, 6, k, k), 60,
                        car_env().spec)
        assert free.n_safe >= o.n_safe          # a narrower road keeps fewer candidates
    model.free()
