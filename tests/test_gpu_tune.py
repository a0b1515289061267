"""The launch-shape autotuner (mpmi_tune_launch_shape, through the C ABI): it
measures every compiled shape, the winner is at least as fast as the built-in
default in its own measurement, later sessions of the same configuration take the
winner, other configurations keep the built-in rule, and the tuned session's
results are bit-identical to the default session's (every shape sums K z in the
same order)."""
import numpy as np
import pytest

from workloads import data

from parity import bot_env, car_env, gpu_model, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


@pytest.mark.parametrize("which,N,H,n_shapes", [("bot", 16384, 50, 4), ("car", 2047, 60, 6)])
def test_tuned_shape_is_used_and_changes_nothing(lib, which, N, H, n_shapes):
    ctx = lib.Context(0)  # a fresh context: its table of tuned shapes starts empty
    env = bot_env() if which == "bot" else car_env()
    model = gpu_model(lib, ctx, env)
    x_t = (np.array([0.05, 0.0, 0.0, 0.0]) if which == "bot"
           else data.car_start_state(env.track, vx=12.0))
    u_h = data.to_f32_exact(data.user_input_once(11, env.lo, env.hi))
    default = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=5)
    default_shape = default.launch_shape()
    want = run_gpu(lib, default, x_t, u_h, tick=3)
    default.close()

    r = lib.tune_launch_shape(ctx, model, N, H, env.lo, env.hi, x_t, u_h, reps=10, seed=5)
    assert 1 <= r["n_tried"] <= 6 * n_shapes  # six block sizes per shape
    assert np.isfinite(r["us"]) and np.isfinite(r["default_us"])
    assert r["us"] <= r["default_us"]
    assert r["block"] in (64, 128, 160, 192, 224, 256)

    tuned = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=5)
    assert tuned.launch_shape() == (r["lanes"], r["cands"], r["block"])
    got = run_gpu(lib, tuned, x_t, u_h, tick=3)
    tuned.close()
    assert np.array_equal(got["ttv"], want["ttv"])
    assert np.array_equal(got["cost"], want["cost"])
    for k in ("index", "status", "n_safe", "ttv", "executed_steps"):
        assert got["result"][k] == want["result"][k]
    assert np.array_equal(got["result"]["u_r"], want["result"]["u_r"])

    # an explicit shape and another configuration are not affected
    s = lib.Session(ctx, model, N, H, env.lo, env.hi, seed=5, lanes=default_shape[0],
                    cands=default_shape[1], block=default_shape[2])
    assert s.launch_shape() == default_shape
    s.close()
    other = lib.Session(ctx, model, N + 1, H, env.lo, env.hi, seed=5)
    ctx2 = lib.Context(0)
    model2 = gpu_model(lib, ctx2, env)
    fresh = lib.Session(ctx2, model2, N + 1, H, env.lo, env.hi, seed=5)
    assert other.launch_shape() == fresh.launch_shape()
    other.close()
    fresh.close()
    model2.free()
    model.free()


def test_tuner_argument_checks(lib):
    ctx = lib.Context(0)
    env = bot_env()
    model = gpu_model(lib, ctx, env)
    x_t, u_h = np.array([0.05, 0.0, 0.0, 0.0]), np.array([0.25])
    for reps in (0, 1001):
        with pytest.raises(lib.MpmiError) as e:
            lib.tune_launch_shape(ctx, model, 1000, 20, env.lo, env.hi, x_t, u_h, reps=reps)
        assert e.value.code == -1
    with pytest.raises(lib.MpmiError) as e:
        lib.tune_launch_shape(ctx, model, 1000, 20, env.lo, env.hi, x_t, u_h,
                              sampler="external")
    assert e.value.code == -6
    with pytest.raises(lib.MpmiError) as e:
        lib.tune_launch_shape(ctx, model, 1000, 20, env.lo, env.hi, [np.nan, 0, 0, 0], u_h)
    assert e.value.code == -3
    with pytest.raises(lib.MpmiError) as e:
        lib.tune_launch_shape(ctx, model, 1000, 0, env.lo, env.hi, x_t, u_h)
    assert e.value.code == -1
    model.free()


@pytest.mark.parametrize("N,cands", [(24000, 1), (65536, 2)])
def test_car_one_lane_default_block_follows_the_sm_count(lib, N, cands):
    """The built-in rule gives the race car's one-lane shapes one block of
    ceil(warp-tiles / SMs) warps per SM where that is at most eight warps; the
    results equal those of 128-thread blocks bit for bit."""
    import math
    import torch
    ctx = lib.Context(0)
    env = car_env()
    model = gpu_model(lib, ctx, env)
    x_t = data.car_start_state(env.track, vx=12.0)
    u_h = data.to_f32_exact(data.user_input_once(12, env.lo, env.hi))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    warps = math.ceil(math.ceil((N + 1) / (32 * cands)) / sms)
    default = lib.Session(ctx, model, N, 60, env.lo, env.hi, seed=6)
    shape = default.launch_shape()
    got = run_gpu(lib, default, x_t, u_h, tick=2)
    default.close()
    assert shape == (1, cands, 32 * warps if 4 < warps <= 8 else 128)
    plain = lib.Session(ctx, model, N, 60, env.lo, env.hi, seed=6, lanes=1, cands=cands, block=128)
    want = run_gpu(lib, plain, x_t, u_h, tick=2)
    plain.close()
    assert np.array_equal(got["ttv"], want["ttv"])
    assert np.array_equal(got["cost"], want["cost"])
    for k in ("index", "status", "n_safe", "ttv", "cost", "executed_steps"):
        assert got["result"][k] == want["result"][k]
    assert np.array_equal(got["result"]["u_r"], want["result"]["u_r"])
    model.free()
