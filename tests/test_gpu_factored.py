"""The factorised read-out rollout (through the C ABI) against the oracle's
plain rollout of Alg. 2: the two are equal in real arithmetic, so the factorised
tick must meet the same parity bar as the full one (ttv equal except at a
boundary, the same selection except ties and boundaries)."""
import numpy as np
import pytest

from oracle import mpmi as omp
from oracle import safety as osafe
from oracle import sampling as osamp
from workloads import data

from parity import bot_env, car_env, compare, gpu_model, oracle_samples, run_gpu

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


def _factored(lib, ctx, env, model, x_t, u_h, N, H, seed, stream, tick, include_user=True):
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed, stream_id=stream,
                       include_user=include_user)
    sess.set_rollout("factored")
    try:
        g = run_gpu(lib, sess, x_t, u_h, tick=tick)
    finally:
        sess.close()
    o = omp.tick(env.K32, env.basis, x_t, u_h, oracle_samples(env, N, seed, stream, tick), H,
                 env.spec, include_user=include_user, record=True)
    return g, o


@pytest.mark.parametrize("N,H", [(1000, 50), (4097, 50), (31, 1), (2047, 200), (0, 50), (1, 50)])
def test_factored_bot_matches_oracle(lib, ctx, bot, N, H):
    env, model = bot
    states = data.states_in_box(17, 3, [-0.25, -0.6, -0.6, -0.6], [0.25, 0.6, 0.6, 0.6])
    for k, x_t in enumerate(states):
        u_h = data.to_f32_exact(data.user_input_once(40 + k, env.lo, env.hi))
        g, o = _factored(lib, ctx, env, model, x_t, u_h, N, H, 5, k, 100 + k)
        assert compare(g, o, env, H) <= max(4, 0.002 * (N + 1))


@pytest.mark.parametrize("N", [0, 1, 33])
def test_factored_car_ragged_sizes(lib, ctx, car, N):
    """The user's slot alone, one sample and a partial warp tile."""
    env, model = car
    x0 = data.car_start_state(env.track, vx=13.0)
    for k, x_t in enumerate([x0, x0 + np.array([1.0, -1.5, 0.08, 3.0, 0.2, 0.1])]):
        u_h = data.to_f32_exact(data.user_input_once(420 + k, env.lo, env.hi))
        g, o = _factored(lib, ctx, env, model, x_t, u_h, N, 60, 6, k, 40 + k)
        assert g["result"]["n_slots"] == N + 1
        assert compare(g, o, env, 60) <= 2


@pytest.mark.parametrize("include_user", [True, False])
def test_factored_car_matches_oracle(lib, ctx, car, include_user):
    env, model = car
    x0 = data.car_start_state(env.track, vx=14.0)
    states = [x0, x0 + np.array([1.5, -1.0, 0.1, 4.0, 0.3, 0.2]),
              x0 + np.array([-2.0, 2.5, -0.2, -6.0, -0.2, -0.1])]
    for k, x_t in enumerate(states):
        u_h = data.to_f32_exact(data.user_input_once(300 + k, env.lo, env.hi))
        g, o = _factored(lib, ctx, env, model, x_t, u_h, 2047, 60, 3, 0, k, include_user)
        assert compare(g, o, env, 60, include_user) <= 10


@pytest.mark.slow
def test_factored_full_size(lib, ctx, bot, car):
    env, model = bot
    x_t = np.array([0.05, 0.1, -0.2, 0.0])
    g, o = _factored(lib, ctx, env, model, x_t, [0.25], 16384, 50, 2, 0, 7)
    assert compare(g, o, env, 50) <= 0.002 * 16385
    env, model = car
    x_t = data.car_start_state(env.track, vx=12.0)
    u_h = data.to_f32_exact(data.user_input_once(3, env.lo, env.hi))
    g, o = _factored(lib, ctx, env, model, x_t, u_h, 16384, 60, 3, 0, 0)
    assert compare(g, o, env, 60) <= 0.002 * 16385


def test_factored_drift_closed_form(lib, ctx):
    """x' = x + dt u: ttv has a closed form per candidate."""
    dt, H, x0 = 0.05, 40, 0.3137
    K = np.array([[1.0, dt], [0.0, 1.0]])
    m = lib.model_from_operator(ctx, "linear", K, nx=1, nu=1)
    lib.set_safety_set(m, [-1.0], [1.0])
    sess = lib.Session(ctx, m, 5000, H, [-1.0], [1.0], seed=9)
    sess.set_rollout("factored")
    g = run_gpu(lib, sess, [x0], [0.9])
    sess.close()
    cand = omp.candidate_slots([0.9], osamp.uniform_samples(9, 0, 0, 5000, [-1], [1]), True)
    x = x0 + np.arange(1, H + 1)[None, :] * dt * cand
    inside = (x > -1.0) & (x < 1.0)
    want = np.where(inside.all(axis=1), H, np.argmin(inside, axis=1))
    close = np.abs(np.abs(x) - 1.0).min(axis=1) < 1e-5
    assert np.all((g["ttv"] == want) | close)
    m.free()


def test_factored_unbounded_coordinates_and_box_only_car(lib, ctx, car):
    """With no track the race car's read-outs are only the bounded coordinates
    (here vx alone); without any bound every candidate is safe."""
    env, _ = car
    m = lib.model_from_operator(ctx, "car", env.K32)
    lib.set_safety_set(m, [-np.inf, -np.inf, -np.inf, -np.inf, -np.inf, -np.inf],
                       [np.inf, np.inf, np.inf, 16.0, np.inf, np.inf])
    x_t = data.car_start_state(env.track, vx=15.0)
    u_h = np.array([0.0, 1.0])
    box = osafe.SafetySpec(lo=np.full(6, -np.inf),
                           hi=np.array([np.inf] * 3 + [16.0] + [np.inf] * 2))
    sess = lib.Session(ctx, m, 3000, 60, env.lo, env.hi, seed=4)
    sess.set_rollout("factored")
    g = run_gpu(lib, sess, x_t, u_h, tick=2)
    sess.close()
    o = omp.tick(env.K32, "car", x_t, u_h, oracle_samples(env, 3000, 4, 0, 2), 60, box,
                 record=True)
    envb = type(env)("car", env.K32, box, env.lo, env.hi, None)
    assert compare(g, o, envb, 60) <= 6
    assert 0 < g["result"]["n_safe"] < 3001                       # the bound matters
    lib.set_safety_set(m, [-np.inf] * 6, [np.inf] * 6)
    sess = lib.Session(ctx, m, 3000, 60, env.lo, env.hi, seed=4)
    sess.set_rollout("factored")
    g = run_gpu(lib, sess, x_t, u_h, tick=2)
    sess.close()
    assert np.all(g["ttv"] == 60) and g["result"]["index"] == 0
    m.free()


def test_factored_switch_budget_and_refusals(lib, ctx, bot):
    import torch
    env, model = bot
    x_t = np.array([0.1, -0.2, 0.3, 0.0])
    u_h = data.to_f32_exact(data.user_input_once(9, env.lo, env.hi))
    sess = lib.Session(ctx, model, 3000, 50, env.lo, env.hi, seed=2)
    plain = run_gpu(lib, sess, x_t, u_h, tick=4)
    before = ctx.memory_in_use()
    sess.set_rollout("factored")
    assert ctx.memory_in_use() - before == 50 * 4 * 12 * 4
    fact = run_gpu(lib, sess, x_t, u_h, tick=4)
    assert np.mean(fact["ttv"] == plain["ttv"]) > 0.99
    assert np.array_equal(fact["cost"], plain["cost"])
    x = torch.tensor(x_t, device="cuda")
    u = torch.tensor(u_h, device="cuda")
    r = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    tr = torch.zeros((3001, 51, 12), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.MpmiError) as e:
        lib.debug_trajectories(sess, x, u, r, tr)
    assert e.value.code == -6
    sess.set_noise([0.01])
    with pytest.raises(lib.MpmiError) as e:
        lib.evaluate_candidates_device(sess, x, u, r)
    assert e.value.code == -6
    sess.set_noise([])
    assert sess.ctx.lib.mpmi_session_set_rollout(sess.handle, 7) == -1    # unknown mode
    sess.set_rollout("full")
    assert ctx.memory_in_use() == before
    again = run_gpu(lib, sess, x_t, u_h, tick=4)
    assert np.array_equal(again["ttv"], plain["ttv"])
    for key, v in plain["result"].items():
        assert np.array_equal(again["result"][key], v), key
    sess.close()


def test_factored_budget_refusal(lib):
    env = bot_env()
    c = lib.Context(0)
    m = gpu_model(lib, c, env)
    s = lib.Session(c, m, 100, 500, env.lo, env.hi)
    tight = lib.Context(0, mem_budget=c.memory_in_use() + 1000)
    m2 = gpu_model(lib, tight, env)
    s2 = lib.Session(tight, m2, 100, 500, env.lo, env.hi)
    with pytest.raises(lib.MpmiError) as e:
        s2.set_rollout("factored")                  # 500 * 4 * 12 * 4 bytes > the budget
    assert e.value.code == -2
    s2.close()
    s.close()


def test_screened_exact_search_factored(lib, ctx, car):
    """The screened tick's exact rollout of the kept slots and its fallback run
    in the factorised form too; the exact cost-ordered search (tau = 0) still
    picks what the full factorised evaluation picks."""
    import torch
    env, model = car
    scr = lib.Screener(ctx, model, data.screener_init(3), max_batch=1024, max_slots=8000)
    x0 = data.car_start_state(env.track, vx=15.0)
    for i, x in enumerate([x0, x0 + np.array([2.0, -1.0, 0.15, 5.0, 0.2, 0.1])]):
        for u_h in (data.to_f32_exact(data.user_input_once(90 + i, env.lo, env.hi)),
                    np.array([0.375, 1.0])):
            sess = lib.Session(ctx, model, 6000, 60, env.lo, env.hi, seed=8)
            sess.set_rollout("factored")
            xd = torch.tensor(x, dtype=torch.float64, device="cuda")
            ud = torch.tensor(u_h, dtype=torch.float64, device="cuda")
            rp = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            rs = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            lib.evaluate_candidates_device(sess, xd, ud, rp, tick=i)
            lib.evaluate_screened(sess, scr, xd, ud, rs, k=128, tau=0.0, tick=i)
            torch.cuda.synchronize()
            sess.close()
            a, b = lib.result_from_bytes(rp.cpu(), 2), lib.result_from_bytes(rs.cpu(), 2)
            for key in ("index", "status", "ttv"):
                assert a[key] == b[key], key
    scr.free()
