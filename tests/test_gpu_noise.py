"""Alg. 2's per-step Gaussian noise z_i on the GPU (through the C ABI): the
noise stream itself against the oracle's Box-Muller normals, noisy ticks of
both plants against the oracle's noisy tick in every launch shape, and the
noise switch's edge cases."""
import numpy as np
import pytest

from oracle import mpmi as omp
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


def _identity_increments(lib, ctx, basis, nx, nu, x_t, sigma, N, H, seed, stream, tick,
                         n_noise=None):
    """Noisy rollout under K = I with every state safe: z_t - z_{t-1} is the noise."""
    n = {"linear": nx + nu, "car": 32}[basis]
    m = lib.model_from_operator(ctx, basis, np.eye(n), nx=nx, nu=nu)
    lib.set_safety_set(m, [-1e6] * nx, [1e6] * nx)
    lo, hi = [-1.0] * nu, [1.0] * nu
    sess = lib.Session(ctx, m, N, H, lo, hi, seed=seed, stream_id=stream)
    sess.set_noise(sigma if n_noise is None else sigma[:n_noise])
    g = run_gpu(lib, sess, x_t, [0.0] * nu, tick=tick, traj=True)
    sess.close()
    m.free()
    return g, np.diff(g["traj"], axis=1)


@pytest.mark.parametrize("tick,stream", [(0, 0), (2 ** 40 + 5, 2 ** 31 - 1), (77, 3)])
def test_noise_stream_matches_oracle_linear(lib, ctx, tick, stream):
    sigma = np.array([0.0625, 0.125, 0.25, 0.03125])
    N, H = 3000, 40
    g, d = _identity_increments(lib, ctx, "linear", 4, 1, [0.5, -0.25, 0.125, 0.0], sigma,
                                N, H, 11, stream, tick)
    assert np.all(g["ttv"] == H)
    n = osamp.gaussian_noise(11, stream, tick, N + 1, H, 4)      # (H, slots, 4)
    want = sigma[None, None, :] * np.transpose(n, (1, 0, 2))     # (slots, H, 4)
    assert np.max(np.abs(d[:, :, :4] - want)) < 1e-6
    assert np.all(d[:, :, 4] == 0.0)                             # the held input


def test_noise_stream_matches_oracle_car_second_block(lib, ctx):
    """The race car has six state coordinates: two Philox calls per step."""
    sigma = data.to_f32_exact(np.array([0.05, 0.04, 0.01, 0.2, 0.03, 0.02]))
    N, H = 1500, 25
    x_t = np.array([1.0, -2.0, 0.3, 12.0, 0.1, -0.05])
    g, d = _identity_increments(lib, ctx, "car", 6, 2, x_t, sigma, N, H, 5, 9, 123)
    n = osamp.gaussian_noise(5, 9, 123, N + 1, H, 6)
    want = sigma[None, None, :] * np.transpose(n, (1, 0, 2))
    scale = np.maximum(np.abs(g["traj"][:, 1:, :6]), 1.0)
    assert np.max(np.abs(d[:, :, :6] - want) / scale) < 2e-6
    assert np.all(d[:, :, 6:] == 0.0)                            # lifted features untouched
    # fewer coordinates: the rest stays exactly constant
    g3, d3 = _identity_increments(lib, ctx, "car", 6, 2, x_t, sigma, N, H, 5, 9, 123,
                                  n_noise=3)
    assert np.all(d3[:, :, 3:] == 0.0)
    assert np.max(np.abs(d3[:, :, :3] - want[:, :, :3]) / scale[:, :, :3]) < 2e-6


def _noisy_tick(lib, ctx, env, model, x_t, u_h, N, H, sigma, seed, stream, tick, lanes=0,
                cands=0):
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed, stream_id=stream,
                       lanes=lanes, cands=cands)
    sess.set_noise(sigma)
    try:
        g = run_gpu(lib, sess, x_t, u_h, tick=tick, traj=True)
    finally:
        sess.close()
    samples = oracle_samples(env, N, seed, stream, tick)
    noise = sigma[None, None, :] * osamp.gaussian_noise(seed, stream, tick, N + 1, H,
                                                        len(sigma))
    o = omp.tick(env.K32, env.basis, x_t, u_h, samples, H, env.spec, record=True, noise=noise)
    return g, o


@pytest.mark.parametrize("lanes,cands", [(1, 1), (1, 2), (2, 1), (4, 1)])
def test_noisy_bot_ticks(lib, ctx, bot, lanes, cands):
    env, model = bot
    sigma = data.to_f32_exact(np.array([0.004, 0.02, 0.003, 0.02]))
    states = data.states_in_box(41, 3, [-0.2, -0.5, -0.5, -0.5], [0.2, 0.5, 0.5, 0.5])
    changed = 0
    for k, x_t in enumerate(states):
        u_h = data.to_f32_exact(data.user_input_once(500 + k, env.lo, env.hi))
        g, o = _noisy_tick(lib, ctx, env, model, x_t, u_h, 2047, 50, sigma, 3, k, 10 + k,
                           lanes, cands)
        assert compare(g, o, env, 50) <= 6
        free = omp.tick(env.K32, env.basis, x_t, u_h, oracle_samples(env, 2047, 3, k, 10 + k),
                        50, env.spec)
        changed += int(np.count_nonzero(free.ttv != o.ttv))
    assert changed > 0                                  # the noise matters at this sigma


@pytest.mark.parametrize("lanes,cands", [(1, 1), (1, 2), (2, 1), (4, 1), (8, 1), (16, 1)])
def test_noisy_car_ticks(lib, ctx, car, lanes, cands):
    env, model = car
    sigma = data.to_f32_exact(np.array([0.03, 0.03, 0.005, 0.1, 0.02, 0.01]))
    x0 = data.car_start_state(env.track, vx=14.0)
    for k, x_t in enumerate([x0, x0 + np.array([1.5, -1.0, 0.1, 4.0, 0.3, 0.2])]):
        u_h = data.to_f32_exact(data.user_input_once(700 + k, env.lo, env.hi))
        g, o = _noisy_tick(lib, ctx, env, model, x_t, u_h, 1023, 60, sigma, 4, 2 + k, k,
                           lanes, cands)
        assert compare(g, o, env, 60) <= 6


def test_zero_sigma_and_noise_off_are_the_plain_tick(lib, ctx, bot):
    env, model = bot
    x_t = np.array([0.1, -0.2, 0.3, 0.0])
    u_h = data.to_f32_exact(data.user_input_once(9, env.lo, env.hi))

    def run(setting):
        sess = lib.Session(ctx, model, 4000, 50, env.lo, env.hi, seed=2)
        if setting is not None:
            sess.set_noise(setting)
        g = run_gpu(lib, sess, x_t, u_h, tick=4, traj=True)
        sess.close()
        return g

    plain = run(None)
    for setting in ([0.0, 0.0, 0.0, 0.0], []):
        g = run(setting)
        assert np.array_equal(g["ttv"], plain["ttv"])
        assert np.array_equal(g["traj"], plain["traj"], equal_nan=True)
        for key, v in plain["result"].items():
            assert np.array_equal(g["result"][key], v), key
    sess = lib.Session(ctx, model, 4000, 50, env.lo, env.hi, seed=2)
    sess.set_noise([0.01, 0.0, 0.0, 0.0])
    sess.set_noise([])                                   # switched off again
    g = run_gpu(lib, sess, x_t, u_h, tick=4, traj=True)
    sess.close()
    assert np.array_equal(g["traj"], plain["traj"], equal_nan=True)


def test_set_noise_argument_checks(lib, ctx, bot):
    import torch
    env, model = bot
    sess = lib.Session(ctx, model, 100, 10, env.lo, env.hi)
    for bad, code in (([0.1] * 5, -1), ([-0.1], -1), ([np.nan], -3), ([np.inf, 0.1], -3)):
        with pytest.raises(lib.MpmiError) as e:
            sess.set_noise(bad)
        assert e.value.code == code
    sess.set_noise([0.1])
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.MpmiError) as e:
        lib.evaluate_candidates_device(sess, x, u, r, tick=2 ** 48)
    assert e.value.code == -1
    lib.evaluate_candidates_device(sess, x, u, r, tick=2 ** 48 - 1)
    torch.cuda.synchronize()
    sess.close()


def test_screened_exact_search_with_noise(lib, ctx, car):
    """The noise is a function of (seed, stream, tick, slot): the exact screened
    search, in cost order (tau = 0) and with the network (tau > 0, whose kept
    rollout takes 16 lanes per candidate), still picks what the full noisy
    evaluation picks."""
    import torch
    env, model = car
    sigma = data.to_f32_exact(np.array([0.03, 0.03, 0.005, 0.1, 0.02, 0.01]))
    scr = lib.Screener(ctx, model, data.screener_init(3), max_batch=1024, max_slots=8000)
    x0 = data.car_start_state(env.track, vx=15.0)
    for i, x in enumerate([x0, x0 + np.array([2.0, -1.0, 0.15, 5.0, 0.2, 0.1])]):
        for u_h in (data.to_f32_exact(data.user_input_once(90 + i, env.lo, env.hi)),
                    np.array([0.375, 1.0])):
            sess = lib.Session(ctx, model, 6000, 60, env.lo, env.hi, seed=8)
            sess.set_noise(sigma)
            xd = torch.tensor(x, dtype=torch.float64, device="cuda")
            ud = torch.tensor(u_h, dtype=torch.float64, device="cuda")
            rp = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            rs = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            rn = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            lib.evaluate_candidates_device(sess, xd, ud, rp, tick=i)
            lib.evaluate_screened(sess, scr, xd, ud, rs, k=128, tau=0.0, tick=i)
            lib.evaluate_screened(sess, scr, xd, ud, rn, k=1, tau=0.05, m=4, tick=i)
            torch.cuda.synchronize()
            sess.close()
            a = lib.result_from_bytes(rp.cpu(), 2)
            for b in (lib.result_from_bytes(rs.cpu(), 2), lib.result_from_bytes(rn.cpu(), 2)):
                for key in ("index", "status", "ttv"):
                    assert a[key] == b[key], key
                assert np.array_equal(a["u_r"], b["u_r"])
    scr.free()
