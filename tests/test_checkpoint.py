"""Checkpoint and resume (paper_1906_02318_gb300.checkpoint).

CPU: the files hold plain arrays and round-trip exactly; a file of another
format is refused.  GPU (through the C ABI): a model loaded from its file ticks
bit for bit like the saved one (race car with its track), a screener's weights
load back into the same scores, and a session saved after some ticks and
reopened continues the tick stream exactly as if it had not stopped."""
import numpy as np
import pytest

from workloads import data, plants


def test_model_file_round_trip(tmp_path):
    from paper_1906_02318_gb300 import checkpoint as ck, mpmi
    x, u, xn = data.transitions("car", 3, 2000)
    K, res = mpmi.fit_operator("car", x, u, xn)   # host-side fit, no device needed
    track = data.track_polyline(3)
    safety = dict(lo=data.CAR_SAFE_LO, hi=data.CAR_SAFE_HI, inflation=0.25, track=track,
                  half_width=data.CAR_TRACK_HALF_WIDTH)
    path = str(tmp_path / "car_model.npz")
    ck.write(path, ck.model_record("car", K, 6, 2, safety, res))
    with np.load(path, allow_pickle=False) as z:   # plain arrays only
        assert set(z.files) >= {"format", "basis", "K", "safety_lo", "track"}
    rec = ck.read(path, ck.FORMAT_MODEL)
    assert rec["basis"] == "car" and rec["nx"] == 6 and rec["nu"] == 2
    assert np.array_equal(rec["K"], K) and rec["residual"] == res
    assert np.array_equal(rec["safety_lo"], data.CAR_SAFE_LO)
    assert np.array_equal(rec["safety_hi"], data.CAR_SAFE_HI)
    assert np.array_equal(rec["track"], track) and rec["inflation"] == 0.25
    with pytest.raises(ValueError):
        ck.read(path, ck.FORMAT_SESSION)


def test_session_and_weights_records_round_trip(tmp_path):
    from paper_1906_02318_gb300 import checkpoint as ck
    cfg = dict(n_samples=4096, horizon=60, input_lo=np.array([-0.4, -1.0]),
               input_hi=np.array([0.4, 1.0]), include_user=True, sampler="grid", seed=2**40 + 3,
               stream_id=7, lanes=8, block=256, cands=1)
    path = str(tmp_path / "session.npz")
    ck.write(path, ck.session_record(cfg, 123456789012, noise=[0.1, 0.2], rollout="tensor"))
    rec = ck.read(path, ck.FORMAT_SESSION)
    assert rec["next_tick"] == 123456789012 and rec["rollout"] == "tensor"
    assert np.array_equal(rec["noise"], [0.1, 0.2])
    for key, value in cfg.items():
        assert np.array_equal(rec["cfg_" + key], value), key
    w = data.screener_init(4)
    wpath = str(tmp_path / "w.npz")
    rec = dict(format=ck.FORMAT_SCREENER)
    rec.update({f"w_{k}": np.asarray(v, dtype=np.float32) for k, v in w.items()})
    ck.write(wpath, rec)
    back = ck.load_screener_weights(wpath)
    assert set(back) == set(w)
    for k in w:
        assert np.array_equal(back[k], np.asarray(w[k], dtype=np.float32)), k


# ---------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


def _car_states(track, count):
    x0 = data.car_start_state(track, vx=11.0)
    rng = np.random.default_rng(12)
    return [x0 + np.concatenate([rng.uniform(-1.5, 1.5, 2), rng.uniform(-0.1, 0.1, 1),
                                 rng.uniform(-2, 2, 1), rng.uniform(-0.2, 0.2, 2)])
            for _ in range(count)]


def _same(a, b):
    for key in ("index", "status", "n_safe", "ttv", "cost", "executed_steps", "tick"):
        assert a[key] == b[key], key
    assert np.array_equal(a["u_r"], b["u_r"])


@pytest.mark.gpu
def test_loaded_model_and_resumed_session_tick_identically(lib, tmp_path):
    from paper_1906_02318_gb300 import checkpoint as ck
    x, u, xn = data.transitions("car", 3, 20000)
    track = data.track_polyline(3)
    ctx = lib.Context(0)
    model, res = lib.fit_model(ctx, "car", x, u, xn)
    lib.set_safety_set(model, data.CAR_SAFE_LO, data.CAR_SAFE_HI, 0.5, track,
                       data.CAR_TRACK_HALF_WIDTH)
    mpath, spath = str(tmp_path / "model.npz"), str(tmp_path / "session.npz")
    ck.save_model(mpath, model, res)
    lo, hi = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI
    states = _car_states(track, 10)
    uhs = [data.to_f32_exact(data.user_input_once(300 + t, lo, hi)) for t in range(10)]
    # the uninterrupted stream on the original model
    ref = lib.Session(ctx, model, 4096, 60, lo, hi, seed=31, stream_id=5)
    want = []
    for t in range(10):
        lib.evaluate_candidates(ref, states[t], uhs[t], tick=1000 + t)
        want.append(lib.select_input(ref))
    ref.close()
    # a session on the model loaded in another context: ticks 0..4, saved, reopened
    ctx2 = lib.Context(0)
    loaded = ck.load_model(ctx2, mpath)
    assert np.array_equal(loaded.get_operator(), model.get_operator())
    first = lib.Session(ctx2, loaded, 4096, 60, lo, hi, seed=31, stream_id=5)
    for t in range(5):
        lib.evaluate_candidates(first, states[t], uhs[t], tick=1000 + t)
        _same(lib.select_input(first), want[t])
    ck.save_session(spath, first, next_tick=1005)
    first.close()
    resumed, tick = ck.open_session(ctx2, loaded, spath)
    assert tick == 1005
    for t in range(5, 10):
        lib.evaluate_candidates(resumed, states[t], uhs[t], tick=tick + t - 5)
        _same(lib.select_input(resumed), want[t])
    resumed.close()
    loaded.free()
    model.free()


@pytest.mark.gpu
def test_saved_screener_weights_score_identically(lib, tmp_path):
    import torch
    from paper_1906_02318_gb300 import checkpoint as ck
    from parity import car_env, gpu_model
    ctx = lib.Context(0)
    env = car_env()
    model = gpu_model(lib, ctx, env)
    w = data.screener_init(9)
    w["b1"] = np.random.default_rng(1).normal(0, 0.2, 128)
    a = lib.Screener(ctx, model, w, max_batch=1024, max_slots=2048)
    path = str(tmp_path / "screener.npz")
    ck.save_screener(path, a)
    b = lib.Screener(ctx, model, ck.load_screener_weights(path), max_batch=1024, max_slots=2048)
    rng = np.random.default_rng(2)
    f = torch.tensor(rng.uniform(-1, 1, (1000, 12)), dtype=torch.float32, device="cuda")
    ya = torch.zeros(1000, dtype=torch.float32, device="cuda")
    yb = torch.zeros(1000, dtype=torch.float32, device="cuda")
    a.score(f, ya)
    b.score(f, yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    a.free()
    b.free()
    model.free()
