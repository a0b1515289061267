"""The race car's tensor-core rollout (tcgen05, three TF32 products per term)
through the C ABI: trajectories, time-to-violation and selection against the
float64 oracle under the same tolerances as the CUDA-core rollout, ragged tiles,
noise, the exact screened search, and refusals."""
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
def car(lib, ctx):
    env = car_env()
    return env, gpu_model(lib, ctx, env)


def _tensor_tick(lib, ctx, env, model, x_t, u_h, N, H, seed, stream, tick, include_user=True,
                 sigma=None, traj=True):
    sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed, stream_id=stream,
                       include_user=include_user)
    sess.set_rollout("tensor")
    if sigma is not None:
        sess.set_noise(sigma)
    try:
        g = run_gpu(lib, sess, x_t, u_h, tick=tick, traj=traj)
    finally:
        sess.close()
    noise = None
    if sigma is not None:
        n_slots = N + int(include_user)
        noise = sigma[None, None, :] * osamp.gaussian_noise(seed, stream, tick, n_slots, H,
                                                            len(sigma))
    o = omp.tick(env.K32, env.basis, x_t, u_h, oracle_samples(env, N, seed, stream, tick), H,
                 env.spec, include_user=include_user, record=True, noise=noise)
    return g, o


def _states(env):
    x0 = data.car_start_state(env.track, vx=14.0)
    return [x0, x0 + np.array([1.5, -1.0, 0.1, 4.0, 0.3, 0.2]),
            x0 + np.array([-2.0, 2.5, -0.2, -6.0, -0.2, -0.1])]


@pytest.mark.parametrize("N,H", [(127, 60), (128, 60), (129, 60), (2047, 60), (4095, 1),
                                 (1000, 150)])
def test_tensor_rollout_matches_oracle(lib, ctx, car, N, H):
    env, model = car
    for k, x_t in enumerate(_states(env)):
        u_h = data.to_f32_exact(data.user_input_once(400 + k, env.lo, env.hi))
        g, o = _tensor_tick(lib, ctx, env, model, x_t, u_h, N, H, 3, k, 20 + k)
        assert compare(g, o, env, H) <= max(6, 0.002 * (N + 1))


@pytest.mark.parametrize("N", [0, 1, 33])
def test_tensor_rollout_ragged_sizes(lib, ctx, car, N):
    """The user's slot alone, one sample and a partial tile: one tile of 128 rows
    with nearly all of them padding, trajectories and all."""
    env, model = car
    for k, x_t in enumerate(_states(env)[:2]):
        u_h = data.to_f32_exact(data.user_input_once(410 + k, env.lo, env.hi))
        g, o = _tensor_tick(lib, ctx, env, model, x_t, u_h, N, 60, 6, k, 30 + k)
        assert g["result"]["n_slots"] == N + 1
        assert compare(g, o, env, 60) <= 2


def test_tensor_rollout_without_user_slot_and_full_size(lib, ctx, car):
    env, model = car
    x_t = _states(env)[1]
    u_h = data.to_f32_exact(data.user_input_once(3, env.lo, env.hi))
    g, o = _tensor_tick(lib, ctx, env, model, x_t, u_h, 3000, 60, 4, 1, 5, include_user=False)
    assert compare(g, o, env, 60, include_user=False) <= 8
    g, o = _tensor_tick(lib, ctx, env, model, _states(env)[0], u_h, 16384, 60, 3, 0, 0)
    assert compare(g, o, env, 60) <= 0.002 * 16385


def test_tensor_rollout_with_noise(lib, ctx, car):
    env, model = car
    sigma = data.to_f32_exact(np.array([0.03, 0.03, 0.005, 0.1, 0.02, 0.01]))
    for k, x_t in enumerate(_states(env)[:2]):
        u_h = data.to_f32_exact(data.user_input_once(700 + k, env.lo, env.hi))
        g, o = _tensor_tick(lib, ctx, env, model, x_t, u_h, 1023, 60, 4, 2 + k, k, sigma=sigma)
        assert compare(g, o, env, 60) <= 6


def test_tensor_agrees_with_cuda_core_rollout(lib, ctx, car):
    """Both approximate the same float64 rollout: per-candidate ttv agree except
    at boundary cases (each path may differ from the oracle on up to 0.2 % of
    the candidates, all at a safety boundary), and the selections agree."""
    env, model = car
    diff = total = 0
    for k, x_t in enumerate(_states(env)):
        u_h = data.to_f32_exact(data.user_input_once(50 + k, env.lo, env.hi))
        outs = []
        for mode in ("full", "tensor"):
            sess = lib.Session(ctx, model, 8191, 60, env.lo, env.hi, seed=9)
            sess.set_rollout(mode)
            outs.append(run_gpu(lib, sess, x_t, u_h, tick=k))
            sess.close()
        diff += int(np.count_nonzero(outs[0]["ttv"] != outs[1]["ttv"]))
        total += outs[0]["ttv"].size
        assert np.array_equal(outs[0]["cost"], outs[1]["cost"])
        assert outs[0]["result"]["index"] == outs[1]["result"]["index"]
    assert diff <= 0.004 * total


def test_screened_exact_search_tensor(lib, ctx, car):
    import torch
    env, model = car
    scr = lib.Screener(ctx, model, data.screener_init(3), max_batch=1024, max_slots=8000)
    for i, x in enumerate(_states(env)[:2]):
        for u_h in (data.to_f32_exact(data.user_input_once(90 + i, env.lo, env.hi)),
                    np.array([0.375, 1.0])):
            sess = lib.Session(ctx, model, 6000, 60, env.lo, env.hi, seed=8)
            sess.set_rollout("tensor")
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


def test_tensor_refusals_and_timeout(lib, ctx, car):
    env, model = car
    benv = bot_env()
    bmodel = gpu_model(lib, ctx, benv)
    s = lib.Session(ctx, bmodel, 100, 10, benv.lo, benv.hi)
    with pytest.raises(lib.MpmiError) as e:
        s.set_rollout("tensor")
    assert e.value.code == -6
    s.close()
    bmodel.free()
    x_t = _states(env)[0]
    u_h = data.to_f32_exact(data.user_input_once(5, env.lo, env.hi))
    sess = lib.Session(ctx, model, 3000, 60, env.lo, env.hi, seed=3)
    sess.set_rollout("tensor")
    want = run_gpu(lib, sess, x_t, u_h, tick=1)
    sess.withhold_staging(True)
    got = run_gpu(lib, sess, x_t, u_h, tick=1)
    assert got["result"]["status"] == lib.TIMEOUT
    sess.withhold_staging(False)
    again = run_gpu(lib, sess, x_t, u_h, tick=1)
    assert np.array_equal(again["ttv"], want["ttv"])
    sess.close()


def test_tensor_nonfinite_state_is_unsafe(lib, ctx, car):
    """A NaN state reaches the MMAs through the TF32 split as a NaN: every
    candidate fails at step 1, as in the CUDA-core rollout."""
    env, model = car
    x_t = _states(env)[0].copy()
    x_t[3] = np.nan
    sess = lib.Session(ctx, model, 1000, 60, env.lo, env.hi, seed=2)
    sess.set_rollout("tensor")
    g = run_gpu(lib, sess, x_t, [0.1, 0.2])
    sess.close()
    assert np.all(g["ttv"] == 0) and g["result"]["status"] == lib.FALLBACK
    assert g["result"]["index"] == 0 and g["result"]["n_safe"] == 0


def test_tensor_two_tiles_per_cta_sampled_oracle(lib, ctx, car):
    """80,001 slots: more tiles than resident CTAs, so both halves of every CTA
    carry tiles and CTAs take several.  Per-candidate ttv and cost of 600 slots
    spread over the range (every tile boundary region included) against the
    float64 oracle run on those candidates alone, and the whole tick against the
    CUDA-core rollout."""
    env, model = car
    N, H, seed = 80000, 60, 21
    x_t = _states(env)[1]
    u_h = data.to_f32_exact(data.user_input_once(31, env.lo, env.hi))
    outs = {}
    for mode in ("full", "tensor"):
        sess = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=seed, stream_id=2)
        sess.set_rollout(mode)
        outs[mode] = run_gpu(lib, sess, x_t, u_h, tick=4)
        sess.close()
    g, c = outs["tensor"], outs["full"]
    assert np.array_equal(g["cost"], c["cost"])
    assert np.count_nonzero(g["ttv"] != c["ttv"]) <= 0.004 * (N + 1)
    assert g["result"]["index"] == c["result"]["index"]
    samples = oracle_samples(env, N, seed, 2, 4)          # slots 1..N
    rng = np.random.default_rng(5)
    pick = np.unique(np.concatenate([rng.integers(1, N + 1, 560),
                                     np.arange(1, 41), np.arange(N - 39, N + 1)]))
    o = omp.tick(env.K32, env.basis, x_t, u_h, samples[pick - 1], H, env.spec,
                 include_user=False)
    assert np.allclose(g["cost"][pick], o.cost, rtol=1e-6, atol=0)
    assert np.count_nonzero(g["ttv"][pick] != o.ttv) <= max(3, 0.01 * pick.size)
