"""Parity of the learned screener's CUDA kernels with the float64 reference, and
the invariants of the screened tick (through the C ABI)."""
import numpy as np
import pytest

from oracle import screener as osc
from oracle import sampling as osamp
from workloads import data, plants

from parity import car_env, gpu_model

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
def setup(lib):
    ctx = lib.Context(0)
    env = car_env()
    model = gpu_model(lib, ctx, env)
    w0 = data.screener_init(11)
    scr = lib.Screener(ctx, model, w0, max_batch=4096, max_slots=20000)
    return ctx, env, model, scr, w0


def _states(env, count, seed):
    x0 = data.car_start_state(env.track, vx=12.0)
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        v = env.track[(37 * i + 5) % len(env.track)]
        nxt = env.track[((37 * i + 5) + 1) % len(env.track)]
        head = np.arctan2(*(nxt - v)[::-1])
        out.append(np.array([v[0] + rng.uniform(-2.5, 2.5), v[1] + rng.uniform(-2.5, 2.5),
                             head + rng.uniform(-0.3, 0.3), rng.uniform(5, 22),
                             rng.uniform(-1, 1), rng.uniform(-0.5, 0.5)]))
    return [x0] + out


def test_tick_features_match_reference(lib, setup):
    import torch
    ctx, env, model, scr, _ = setup
    out = torch.zeros(12, dtype=torch.float32, device="cuda")
    for x in _states(env, 12, 0):
        scr.tick_features(torch.tensor(x, dtype=torch.float64, device="cuda"), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        want = osc.tick_features(env.track, env.spec.half_width, x)
        # nearest segment as the reference finds it (float64, lowest index on ties)
        a = env.track
        d = np.roll(a, -1, axis=0) - a
        t = np.clip(np.sum((x[:2] - a) * d, axis=1) / np.sum(d * d, axis=1), 0, 1)
        dist = np.linalg.norm(x[:2] - a - t[:, None] * d, axis=1)
        i_ref = int(np.argmin(dist))
        if int(got[10]) != i_ref:
            # only a float32 near-tie may pick a neighbouring segment
            assert abs(dist[int(got[10])] - dist[i_ref]) < 1e-4
            continue
        assert abs(got[11] - dist[i_ref]) < 1e-4
        assert np.allclose(got[:10], want, atol=2e-4, rtol=0)


def test_slot_features_match_candidates(lib, setup):
    import torch
    ctx, env, model, scr, _ = setup
    N = 3000
    sess = lib.Session(ctx, model, N, 60, env.lo, env.hi, seed=5)
    x = _states(env, 1, 3)[1]
    u_h = data.to_f32_exact(data.user_input_once(4, env.lo, env.hi))
    feats = torch.zeros((N + 1, 12), dtype=torch.float32, device="cuda")
    tf = torch.zeros(12, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    scr.features(sess, xd, torch.tensor(u_h, dtype=torch.float64, device="cuda"), feats, tick=9)
    scr.tick_features(xd, tf)
    torch.cuda.synchronize()
    sess.close()
    f = feats.cpu().numpy().astype(np.float64)
    cands = np.vstack([u_h, osamp.uniform_samples(5, 0, 9, N, env.lo, env.hi)])
    assert np.array_equal(f[:, :10], np.broadcast_to(tf.cpu().numpy()[:10], (N + 1, 10)))
    assert np.allclose(f[:, 10], cands[:, 0] / 0.4, rtol=1e-6, atol=1e-7)
    assert np.array_equal(f[:, 11], cands[:, 1])


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    f = np.column_stack([rng.uniform(-1, 1, B), rng.uniform(-1, 1, B), rng.uniform(0.5, 1, B),
                         rng.uniform(0, 1, B), rng.uniform(-0.3, 0.3, B), rng.uniform(-0.3, 0.3, B),
                         rng.uniform(-0.5, 0.5, (B, 4)), rng.uniform(-1, 1, B),
                         rng.uniform(-1, 1, B)])
    f = data.to_f32_exact(f)
    t = data.to_f32_exact(rng.uniform(0, 1, B))
    return f, t


def test_gradients_match_reference(lib, setup):
    import torch
    ctx, env, model, scr, w0 = setup
    scr.set_weights(w0)
    f, t = _batch(1, 512)
    g = torch.zeros(lib.SCREENER_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    scr.gradients(torch.tensor(f, dtype=torch.float32, device="cuda"),
                  torch.tensor(t, dtype=torch.float32, device="cuda"), g, loss)
    torch.cuda.synchronize()
    cache = osc.forward(w0, f)
    ref = osc.backward(w0, cache, t)
    got = lib.unpack_weights(g.cpu().numpy())
    assert float(loss.item()) == pytest.approx(osc.loss(cache["y"], t), rel=1e-5)
    for k in ref:
        scale = float(np.max(np.abs(ref[k])))
        assert np.max(np.abs(np.asarray(got[k]) - ref[k])) <= 1e-4 * scale + 1e-9, k


def test_adam_step_matches_reference(lib, setup):
    import torch
    ctx, env, model, scr, w0 = setup
    scr.set_weights(w0)
    p = {k: v.copy() for k, v in w0.items()}
    state = {}
    for step in (1, 2, 3):
        f, t = _batch(10 + step, 256)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        scr.train_step(torch.tensor(f, dtype=torch.float32, device="cuda"),
                       torch.tensor(t, dtype=torch.float32, device="cuda"), loss, lr=1e-3)
        g = osc.backward(p, osc.forward(p, f), t)
        osc.adam_step(p, g, state, step, lr=1e-3)
    got = scr.get_weights()
    for k in p:
        assert np.max(np.abs(np.asarray(got[k]) - p[k])) <= 2e-6, k


def test_tensor_core_scores_within_bf16_tolerance(lib, setup):
    import torch
    ctx, env, model, scr, w0 = setup
    w = {k: v.copy() for k, v in w0.items()}
    w["b1"] = np.random.default_rng(2).normal(0, 0.1, 128)
    w["b3"] = np.array(0.2)
    scr.set_weights(w)
    f, _ = _batch(3, 4099)
    out = torch.zeros(4099, dtype=torch.float32, device="cuda")
    scr.score(torch.tensor(f, dtype=torch.float32, device="cuda"), out)
    torch.cuda.synchronize()
    want = osc.forward({k: data.to_f32_exact(v) for k, v in w.items()}, f)["y"]
    err = np.abs(out.cpu().numpy() - want)
    assert err.max() < 0.02 and err.mean() < 0.004


def _plain_and_screened(lib, ctx, env, model, scr, x, u_h, N, k, tau, tick, m=8):
    import torch
    sess = lib.Session(ctx, model, N, 60, env.lo, env.hi, seed=7)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ud = torch.tensor(u_h, dtype=torch.float64, device="cuda")
    rp = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rs = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ttv = torch.zeros(N + 1, dtype=torch.int32, device="cuda")
    cost = torch.zeros(N + 1, dtype=torch.float32, device="cuda")
    lst = torch.full((N + 1,), -1, dtype=torch.int32, device="cuda")
    nl = torch.zeros(1, dtype=torch.int32, device="cuda")
    feats = torch.zeros((N + 1, 12), dtype=torch.float32, device="cuda")
    scores = torch.zeros(N + 1, dtype=torch.float32, device="cuda")
    lib.evaluate_candidates_device(sess, xd, ud, rp, tick=tick, ttv_dev=ttv, cost_dev=cost)
    lib.evaluate_screened(sess, scr, xd, ud, rs, k=k, tau=tau, m=m, tick=tick, list_dev=lst,
                          n_list_dev=nl)
    # the same network on the same slot inputs (the tensor-core path of the tick)
    scr.features(sess, xd, ud, feats, tick=tick)
    scr.score(feats, scores)
    torch.cuda.synchronize()
    sess.close()
    n = int(nl.item())
    return (lib.result_from_bytes(rp.cpu(), 2), lib.result_from_bytes(rs.cpu(), 2),
            ttv.cpu().numpy(), cost.cpu().numpy(), np.sort(lst.cpu().numpy()[:n]),
            scores.cpu().numpy())


def test_screening_everything_equals_plain(lib, setup):
    ctx, env, model, scr, w0 = setup
    scr.set_weights(w0)
    for i, x in enumerate(_states(env, 3, 4)):
        u_h = data.to_f32_exact(data.user_input_once(20 + i, env.lo, env.hi))
        a, b, ttv, cost, lst, _ = _plain_and_screened(lib, ctx, env, model, scr, x, u_h, 5000,
                                                      5001, 0.0, i)
        assert lst.tolist() == list(range(5001))
        for key in ("index", "status", "n_safe", "ttv", "executed_steps"):
            assert a[key] == b[key], key
        # every slot was evaluated: no second launch even when none is safe
        assert b["flags"] == 1


@pytest.mark.parametrize("k,tau,m", [(64, 0.5, 1), (512, 0.9, 8), (2048, 0.3, 4), (1, 0.6, 32),
                                     (300, 0.0, 1)])
def test_screened_tick_invariants(lib, setup, k, tau, m):
    """The kept slots are exactly the oracle's rule applied to the device's own
    costs and network scores (a cost-order prefix holding >= k slots and, with the
    network, >= m predicted-safe ones), and the selection is the exhaustive one."""
    ctx, env, model, scr, w0 = setup
    w = {key: v.copy() for key, v in w0.items()}
    w["w3"] = 4.0 * w["w3"]  # spread the scores so that tau splits the slots
    scr.set_weights(w)
    H, N = 60, 8000
    for i, x in enumerate(_states(env, 4, 5 + k)):
        u_h = data.to_f32_exact(data.user_input_once(40 + i, env.lo, env.hi))
        a, b, ttv, cost, lst, y = _plain_and_screened(lib, ctx, env, model, scr, x, u_h, N, k,
                                                      tau, 100 + i, m=m)
        want = osc.screen(y, cost, k, np.float32(tau), m)
        assert lst.tolist() == want.tolist()
        assert 0 in lst and len(lst) >= min(k, N + 1)
        out = np.setdiff1d(np.arange(N + 1), lst)
        if len(out):
            assert cost[lst].max() < cost[out].min()
        # the selection is the exhaustive one, whatever the screen kept
        for key in ("index", "status", "ttv"):
            assert a[key] == b[key], key
        assert np.array_equal(a["u_r"], b["u_r"]) and a["cost"] == b["cost"]
        assert b["index"] == osc.screened_selection(ttv, cost.astype(np.float64), lst, H)
        kept_steps = int(np.minimum(ttv[lst] + 1, H).sum())
        if b["flags"] & 2:
            # nothing safe among the kept slots: the full evaluation ran; the
            # reported steps are both launches'
            assert not np.any(ttv[lst] == H) and len(lst) < N + 1
            assert b["n_safe"] == a["n_safe"]
            assert b["executed_steps"] == a["executed_steps"] + kept_steps
        else:
            assert b["status"] == lib.SAFE or len(lst) == N + 1
            assert b["executed_steps"] == kept_steps and b["n_slots"] == len(lst)



@pytest.mark.slow
def test_screened_tick_full_size(lib, setup):
    """N = 65536, the learned-screener configuration's size: the kept slots are the
    oracle's rule on the device's own costs and scores, and the cost-ordered and
    network-set screens select exactly what the exhaustive evaluation selects."""
    ctx, env, model, _, w0 = setup
    scr = lib.Screener(ctx, model, w0, max_batch=256, max_slots=65537)
    try:
        for i, x in enumerate(_states(env, 2, 21)):
            u_h = data.to_f32_exact(data.user_input_once(80 + i, env.lo, env.hi))
            for k, tau, m in ((4096, 0.0, 1), (1, 0.5, 16)):
                a, b, ttv, cost, lst, y = _plain_and_screened(lib, ctx, env, model, scr, x, u_h,
                                                              65536, k, tau, 500 + i, m=m)
                assert lst.tolist() == osc.screen(y, cost, k, np.float32(tau), m).tolist()
                for key in ("index", "status", "ttv"):
                    assert a[key] == b[key], (i, k, key)
                assert np.array_equal(a["u_r"], b["u_r"]) and a["cost"] == b["cost"]
    finally:
        scr.free()


def test_host_screened_tick_equals_device(lib, setup):
    """The screened tick from host buffers, collected with select_input, gives the
    device-resident screened tick's result field for field, over consecutive ticks
    of one session interleaved with plain host ticks; a state off the road (every
    kept slot unsafe) takes the on-device fallback, whose launch then completes
    the tick."""
    import torch
    ctx, env, model, scr, w0 = setup
    scr.set_weights(w0)
    sess = lib.Session(ctx, model, 6000, 60, env.lo, env.hi, seed=7)
    res = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    states = _states(env, 3, 31)
    off_road = states[1].copy()
    off_road[:2] += 60.0                 # far outside the track band: nothing is safe
    flags = []
    try:
        for i, x in enumerate(states + [off_road]):
            u_h = data.to_f32_exact(data.user_input_once(90 + i, env.lo, env.hi))
            for k, tau, m in ((256, 0.0, 1), (1, 0.0, 1), (1, 0.5, 8)):
                tick = 600 + 10 * i + k
                lib.evaluate_screened(sess, scr, torch.tensor(x, dtype=torch.float64,
                                                              device="cuda"),
                                      torch.tensor(u_h, dtype=torch.float64, device="cuda"),
                                      res, k=k, tau=tau, m=m, tick=tick)
                torch.cuda.synchronize()
                want = lib.result_from_bytes(res.cpu(), 2)
                lib.evaluate_screened_host(sess, scr, x, u_h, k=k, tau=tau, m=m, tick=tick)
                got = lib.select_input(sess)
                for key in ("index", "status", "n_safe", "ttv", "cost", "n_slots",
                            "executed_steps", "tick", "flags"):
                    assert got[key] == want[key], (i, k, key)
                assert np.array_equal(got["u_r"], want["u_r"])
                flags.append(got["flags"])
            lib.evaluate_candidates(sess, x, u_h, tick=900 + i)   # a plain host tick between
            assert lib.select_input(sess)["tick"] == 900 + i
    finally:
        sess.close()
    assert any(f & 2 for f in flags) and any(not f & 2 for f in flags)

def test_screen_score_network_matches_reference(lib, setup):
    """The network inside the screened tick (tensor cores) against the float64
    network on the same slot inputs: with tau at the median reference score, the
    kept prefix lies between the prefixes the reference network gives with tau
    moved by +-0.05 (the bfloat16 inference's margin)."""
    import torch
    ctx, env, model, scr, w0 = setup
    w = {key: v.copy() for key, v in w0.items()}
    w["b1"] = np.random.default_rng(4).normal(0, 0.3, 128)
    w["w3"] = 4.0 * w["w3"]  # spread the outputs (reference std ~0.09)
    scr.set_weights(w)
    N, k, m, tick = 8000, 1, 64, 77
    x = _states(env, 2, 9)[2]
    u_h = data.to_f32_exact(data.user_input_once(61, env.lo, env.hi))
    sess = lib.Session(ctx, model, N, 60, env.lo, env.hi, seed=7)
    feats = torch.zeros((N + 1, 12), dtype=torch.float32, device="cuda")
    scr.features(sess, torch.tensor(x, dtype=torch.float64, device="cuda"),
                 torch.tensor(u_h, dtype=torch.float64, device="cuda"), feats, tick=tick)
    torch.cuda.synchronize()
    sess.close()
    y = osc.forward({key: data.to_f32_exact(v) for key, v in w.items()},
                    feats.cpu().numpy().astype(np.float64))["y"]
    tau = float(np.median(y[1:]))
    a, b, ttv, cost, lst, yg = _plain_and_screened(lib, ctx, env, model, scr, x, u_h, N, k, tau,
                                                   tick, m=m)
    assert np.abs(yg - y).max() < 0.02
    inner = osc.screen(y, cost, k, tau - 0.05, m)   # more predicted safe: shorter
    outer = osc.screen(y, cost, k, tau + 0.05, m)
    assert set(inner.tolist()) <= set(lst.tolist()) <= set(outer.tolist())


def test_training_reduces_loss(lib, setup):
    from paper_1906_02318_gb300 import screener as drv
    ctx, env, model, scr, w0 = setup
    scr.set_weights(w0)
    sess = lib.Session(ctx, model, 1023, 60, env.lo, env.hi, seed=3)
    x0 = data.car_start_state(env.track, vx=12.0)
    uhs = data.ou_user_input(3, 40, plants.CAR_DT, env.lo, env.hi)
    feats, targets, _ = drv.collect_labels(sess, scr, plants.bicycle_step, x0, uhs, env.track,
                                           env.spec.half_width)
    sess.close()
    losses = drv.train(scr, feats, targets, epochs=6, batch=1024, lr=2e-3)
    assert losses[-1] < 0.7 * losses[0]


def test_cost_ordered_search_is_exact(lib, setup):
    """tau = 0 keeps the k cheapest slots: either the least-cost safe candidate is
    among them or every kept slot is cheaper, hence unsafe, and the full
    evaluation runs -- the selection always equals the exhaustive one."""
    ctx, env, model, scr, w0 = setup
    for i, x in enumerate(_states(env, 8, 9)):
        for u_h in (data.to_f32_exact(data.user_input_once(60 + i, env.lo, env.hi)),
                    np.array([0.375, 1.0]), np.array([-0.4, -1.0])):
            a, b, ttv, cost, lst, _ = _plain_and_screened(lib, ctx, env, model, scr, x, u_h,
                                                          6000, 128, 0.0, 200 + i)
            for key in ("index", "status", "ttv"):
                assert a[key] == b[key], key
            assert np.array_equal(a["u_r"], b["u_r"])


def test_learned_screen_does_less_work_than_cost_order(lib, setup):
    """What the trained network gains over the method without it: on held-out
    closed-loop ticks the network-set prefix selects exactly what the exhaustive
    evaluation selects (agreement 1, no safety miss) and executes fewer rollout
    steps per tick than the exact cost-ordered search with a fixed k.  tau and m
    are calibrated on other held-out ticks (fewest executed steps)."""
    from paper_1906_02318_gb300 import screener as drv
    ctx, env, model, scr, w0 = setup
    scr.set_weights(w0)
    x0 = data.car_start_state(env.track, vx=12.0)
    sess = lib.Session(ctx, model, 8192, 60, env.lo, env.hi, seed=13)
    feats, targets, _ = drv.collect_labels(
        sess, scr, plants.bicycle_step, x0,
        data.ou_user_input(13, 60, plants.CAR_DT, env.lo, env.hi), env.track,
        env.spec.half_width)
    drv.train(scr, feats, targets, epochs=8, batch=4096, lr=2e-3)
    del feats, targets

    def held_out(seed, ticks, tick0):
        u = data.ou_user_input(seed, ticks, plants.CAR_DT, env.lo, env.hi)
        _, _, xs = drv.collect_labels(sess, scr, plants.bicycle_step, x0, u, env.track,
                                      env.spec.half_width, tick0=tick0)
        return xs, u

    xc, uc = held_out(14, 30, 5000)
    xe, ue = held_out(15, 60, 9000)
    cal = drv.calibrate(sess, scr, xc, uc, taus=(0.5, 0.8, 0.9, 0.95), ms=(1, 4, 16),
                        tick0=5000)
    learned = drv.compare(sess, scr, xe, ue, k=1, tau=cal["tau"], m=cal["m"], tick0=9000)
    ordered = drv.compare(sess, scr, xe, ue, k=512, tau=0.0, tick0=9000)
    sess.close()
    assert learned["agreement"] == 1.0 and ordered["agreement"] == 1.0
    assert learned["safety_misses"] == 0 and ordered["safety_misses"] == 0
    assert learned["mean_executed_steps"] < ordered["mean_executed_steps"]
    assert learned["mean_executed_steps"] < learned["plain_executed_steps"]
