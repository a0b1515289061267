"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
values of Eq. 2, closed forms (linear plants, matrix powers, drift models with
analytic exit times), textbook special cases (circle/segment distances),
invariants stated by the paper (a safe user input passes through unchanged,
Sec. III-C) and brute force on tiny inputs (pure-Python scalar loops).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import basis, fit, mpmi, philox, safety, sampling
from workloads import data, plants

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def test_mulhilo_matches_python_integers():
    rng = np.random.default_rng(0)
    b = rng.integers(0, 2 ** 32, 5000, dtype=np.uint64).astype(np.uint32)
    b[:3] = [0, 1, 0xFFFFFFFF]
    for a in (philox.M0, philox.M1, 0xFFFFFFFF):
        hi, lo = philox.mulhilo32(a, b)
        for bi, h, l in zip(b[:200].tolist(), hi[:200].tolist(), lo[:200].tolist()):
            p = a * bi
            assert h == p >> 32 and l == p & 0xFFFFFFFF


def _philox_kat():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.json")) as f:
        cases = json.load(f)["cases"]
    return [([int(w, 16) for w in c["counter"]], [int(w, 16) for w in c["key"]],
             [int(w, 16) for w in c["expected"]]) for c in cases]


def test_philox_known_answer_vectors():
    # The published known answers fix the whole generator: the multipliers, the
    # round function's word order, the Weyl key schedule and the round count.
    for ctr, key, want in _philox_kat():
        got = philox.philox4x32(*ctr, *key)
        assert [int(v) for v in got] == want
    # nine or eleven rounds miss every vector
    for rounds in (9, 11):
        for ctr, key, want in _philox_kat():
            assert [int(v) for v in philox.philox4x32(*ctr, *key, rounds=rounds)] != want


def test_philox_single_round_zero_counter_is_key_placement():
    # With a zero counter both products vanish, so one round leaves only the key
    # words in positions 0 and 2 (definition of the round function).
    out = philox.philox4x32(0, 0, 0, 0, 0x12345678, 0x9ABCDEF0, rounds=1)
    assert [int(v) for v in out] == [0x12345678, 0, 0x9ABCDEF0, 0]


def test_philox_second_round_uses_bumped_key():
    k0, k1 = 0x01020304, 0x05060708
    out = philox.philox4x32(0, 0, 0, 0, k0, k1, rounds=2)
    # the second round sees (k0, 0, k1, 0) with the key bumped by the Weyl constants
    p0, p1 = philox.M0 * k0, philox.M1 * k1
    kb0, kb1 = (k0 + philox.W0) & 0xFFFFFFFF, (k1 + philox.W1) & 0xFFFFFFFF
    want = [(p1 >> 32) ^ kb0, p1 & 0xFFFFFFFF, (p0 >> 32) ^ kb1, p0 & 0xFFFFFFFF]
    assert [int(v) for v in out] == want


def test_philox_words_uniform_and_uncorrelated():
    n = 1 << 17
    c = np.arange(n, dtype=np.uint32)
    w = philox.philox4x32(c, 7, 0, 3, 0xDEADBEEF, 42)
    for word in w:
        top = (word >> np.uint32(24)).astype(np.int64)
        counts = np.bincount(top, minlength=256)
        chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-4
    u = [word.astype(np.float64) / 2 ** 32 for word in w]
    for i in range(4):
        for j in range(i + 1, 4):
            assert abs(np.corrcoef(u[i], u[j])[0, 1]) < 0.02


@pytest.mark.parametrize("which", ["counter", "key"])
def test_philox_avalanche(which):
    rng = np.random.default_rng(1)
    flips = []
    for _ in range(400):
        c = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2 ** 32, 2, dtype=np.uint64)
        base = np.array([int(v) for v in philox.philox4x32(*c, int(k[0]), int(k[1]))])
        bit = int(rng.integers(0, 32))
        if which == "counter":
            c2 = c.copy()
            pos = int(rng.integers(0, 4))
            c2[pos] ^= np.uint32(1 << bit)
            o = philox.philox4x32(*c2, int(k[0]), int(k[1]))
        else:
            o = philox.philox4x32(*c, int(k[0]) ^ (1 << bit), int(k[1]))
        o = np.array([int(v) for v in o])
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, o)))
    assert abs(np.mean(flips) - 64.0) < 1.5


# --------------------------------------------------------------------------- sampling
def test_uniform_samples_binary32_in_box_and_uniform():
    lo, hi = [-0.4, -1.0], [0.4, 1.0]
    s = sampling.uniform_samples(5, 2, 11, 50000, lo, hi)
    assert s.shape == (50000, 2)
    assert np.array_equal(s, s.astype(np.float32).astype(np.float64))
    for j in range(2):
        assert s[:, j].min() >= lo[j] and s[:, j].max() <= hi[j]
        ks = stats.kstest((s[:, j] - lo[j]) / (hi[j] - lo[j]), "uniform")
        assert ks.pvalue > 1e-3
    assert abs(np.corrcoef(s[:, 0], s[:, 1])[0, 1]) < 0.02


def test_uniform_samples_counter_layout():
    a = sampling.uniform_samples(9, 1, 3, 4096, [-1], [1])
    assert np.array_equal(a[:1000], sampling.uniform_samples(9, 1, 3, 1000, [-1], [1]))
    for other in (sampling.uniform_samples(9, 1, 4, 4096, [-1], [1]),
                  sampling.uniform_samples(9, 2, 3, 4096, [-1], [1]),
                  sampling.uniform_samples(10, 1, 3, 4096, [-1], [1])):
        assert np.mean(a == other) < 0.01


def test_grid_samples_are_midpoints():
    g = sampling.grid_samples(8, [-1.0], [1.0])
    assert np.allclose(g[:, 0], -1.0 + (np.arange(8) + 0.5) * 0.25, atol=0)
    g2 = sampling.grid_samples(9, [0.0, -1.0], [3.0, 2.0])
    assert sorted(set(g2[:, 0])) == [0.5, 1.5, 2.5]
    assert sorted(set(g2[:, 1])) == [-0.5, 0.5, 1.5]
    with pytest.raises(ValueError):
        sampling.grid_samples(10, [0.0, 0.0], [1.0, 1.0])


# --------------------------------------------------------------------------- Eq. 2
def _all_safe_linear_spec(nx):
    return safety.SafetySpec(lo=np.full(nx, -np.inf), hi=np.full(nx, np.inf))


def test_eq2_worked_values_and_grid_bound():
    g = json.load(open(os.path.join(GOLDEN, "eq2_deviation.json")))
    for case in g["cases"]:
        lam, n = case["lambda"], case["N"]
        bound = lam / (2 * n)
        # the printed value is Eq. 2 rounded to the printed precision
        assert float(f"{bound:.{case['printed_sig_digits']}g}") == case["printed"]
        # the grid of Sec. IV-B with all candidates safe meets the bound (M = 1)
        lo, hi = -lam / 2, lam / 2
        samples = sampling.grid_samples(n, [lo], [hi])
        K = np.eye(2)                       # linear basis [x, u], identity model
        spec = _all_safe_linear_spec(1)
        rng = np.random.default_rng(int(n))
        u_hs = np.concatenate([rng.uniform(lo, hi, 40), [lo, hi, 0.0]])
        worst = 0.0
        for u_h in u_hs:
            r = mpmi.tick(K, "linear", [0.0], [u_h], samples, 3, spec, include_user=False)
            assert r.status == mpmi.SAFE and r.n_safe == n
            dev = mpmi.deviation(r.u_r, [u_h])
            assert dev <= bound * (1 + 1e-6) + 2.0 ** -23 * abs(hi)
            worst = max(worst, dev)
        # the edges of the input box attain the bound
        assert worst >= bound * (1 - 1e-3)


# --------------------------------------------------------------------------- basis
def test_bot_features_special_point():
    z = basis.lift("bot", np.array([0.0, 2.0, 1.5, -3.0]), np.array([0.25]))
    want = [0.0, 2.0, 1.5, -3.0, 0.25, 0.0, 1.0, 4.0, 0.5, 0.0, 0.25, 1.0]
    assert np.array_equal(z, want)
    z = basis.lift("bot", np.array([np.pi / 2, 1.0, 0.0, 0.0]), np.array([2.0]))
    assert np.allclose(z[[5, 6, 9, 10]], [1.0, 0.0, 1.0, 0.0], atol=1e-15)


def test_car_features_special_point():
    x = np.array([3.0, -4.0, 0.0, 10.0, 0.5, 0.2])
    z = basis.lift("car", x, np.array([0.1, -0.5]))
    assert z.shape == (32,)
    vx, vy, om, d, a = 10.0, 0.5, 0.2, 0.1, -0.5
    want = [3.0, -4.0, 0.0, vx, vy, om, d, a, 0.0, 1.0,
            vx, 0.0, vy, 0.0, om * vx, om * vy, vx * vx, vy * vy, om * om,
            d * vx, d * vy, d * om, a * vx, d, 0.0, a, 0.0, om, 0.0, vx * vy, d * d, 1.0]
    assert np.allclose(z, want, rtol=0, atol=1e-15)


def test_lift_broadcasts_state_over_candidates():
    u = np.linspace(-1, 1, 7)[:, None]
    z = basis.lift("bot", np.array([[0.1, 0.2, 0.3, 0.4]]), u)
    assert z.shape == (7, 12)
    for i in range(7):
        assert np.array_equal(z[i], basis.lift("bot", np.array([0.1, 0.2, 0.3, 0.4]), u[i]))


# --------------------------------------------------------------------------- fit
def _linear_plant(seed, nx, nu):
    rng = np.random.default_rng(seed)
    A = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx))
    B = rng.standard_normal((nx, nu))
    return A, B


def test_fit_linear_plant_closed_form():
    A, B = _linear_plant(0, 4, 2)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((500, 4))
    u = rng.uniform(-1, 1, (500, 2))
    xn = plants.linear_step(A, B, x, u)
    K, res = fit.fit_koopman("linear", x, u, xn)
    want = np.block([[A, B], [np.zeros((2, 4)), np.eye(2)]])
    assert np.abs(K - want).max() < 1e-10
    assert res < 1e-12


@pytest.mark.parametrize("kind,held", [("bot", (4, 11)), ("car", (6, 7, 30, 31))])
def test_fit_held_input_rows_are_unit_rows(kind, held):
    x, u, xn = data.transitions(kind, 1 if kind == "bot" else 3, 3000)
    K, res = fit.fit_koopman(kind, x, u, xn)
    n = K.shape[0]
    assert basis.held_features(kind) == held
    for r in held:
        assert np.array_equal(K[r], np.eye(n)[r])          # set exactly
    # the unconstrained least-squares solution (normal equations, another
    # routine) is the unit row up to rounding, and the other rows agree
    X, Y = basis.lift(kind, x, u), basis.lift(kind, xn, u)
    K_ne = np.linalg.solve(X.T @ X, X.T @ Y).T
    for r in held:
        assert np.abs(K_ne[r] - np.eye(n)[r]).max() < 1e-8
    others = [r for r in range(n) if r not in held]
    assert np.abs(K_ne[others] - K[others]).max() < 1e-6 * max(1.0, np.abs(K).max())
    res_ne = np.linalg.norm(X @ K_ne.T - Y) / np.linalg.norm(Y)
    assert abs(res - res_ne) < 1e-9
    assert 0 < res < 0.2


# --------------------------------------------------------------------------- rollout
def test_rollout_matches_matrix_powers():
    rng = np.random.default_rng(2)
    n = 5
    K = np.eye(n) + 0.05 * rng.standard_normal((n, n))   # non-symmetric
    spec = _all_safe_linear_spec(4)
    x_t = rng.standard_normal(4)
    samples = rng.uniform(-1, 1, (6, 1))
    H = 25
    r = mpmi.tick(K, "linear", x_t, [0.2], samples, H, spec, record=True)
    z0 = basis.lift("linear", x_t[None, :], r.candidates)
    for t in (1, 2, 7, 25):
        want = z0 @ np.linalg.matrix_power(K, t).T
        assert np.allclose(r.traj[:, t], want, rtol=1e-12, atol=1e-12)
    assert np.all(r.ttv == H) and r.executed_steps == H * 7


def test_rollout_reproduces_linear_plant():
    A, B = _linear_plant(3, 4, 1)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((200, 4))
    u = rng.uniform(-1, 1, (200, 1))
    K, _ = fit.fit_koopman("linear", x, u, plants.linear_step(A, B, x, u))
    x_t = np.array([0.1, -0.2, 0.3, 0.05])
    samples = np.array([[0.5], [-0.25]])
    r = mpmi.tick(K, "linear", x_t, [0.0], samples, 10, _all_safe_linear_spec(4),
                  record=True)
    for i, c in enumerate(r.candidates):
        xs = x_t.copy()
        for t in range(1, 11):
            xs = plants.linear_step(A, B, xs, c)
            assert np.allclose(r.traj[i, t, :4], xs, rtol=1e-9, atol=1e-10)


def test_identity_model_constant_trajectory():
    spec = safety.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
    x_t = np.array([0.1, 0.3, -0.5, 0.2])
    r = mpmi.tick(np.eye(12), "bot", x_t, [0.0], np.zeros((4, 1)), 30, spec, record=True)
    for t in range(31):
        assert np.array_equal(r.traj[:, t], r.traj[:, 0])
    assert np.all(r.ttv == 30) and r.index == 0 and r.status == mpmi.SAFE


# --------------------------------------------------------------------------- safety
def test_box_bounds_are_strict_and_inflated():
    spec = safety.SafetySpec(lo=np.array([-0.5, -np.inf]), hi=np.array([0.5, np.inf]))
    z = np.array([[0.5, 0.0], [-0.5, 0.0], [0.4999999, 1e300], [np.nan, 0.0],
                  [0.0, np.nan], [np.inf, 0.0]])
    assert safety.is_safe(spec, z).tolist() == [False, False, True, False, False, False]
    spec.inflation = 0.1
    z = np.array([[0.39, 0.0], [0.41, 0.0], [-0.41, 0.0]])
    assert safety.is_safe(spec, z).tolist() == [True, False, False]


def test_distance_circle_and_segment_closed_forms():
    tr = data.track_polyline(0, circular=True)
    S = len(tr)
    R = data.TRACK_RADIUS
    ang = 2 * np.pi * np.arange(0, S, 17) / S
    # on a vertex ray: outside the circle the vertex is nearest (distance r - R);
    # inside, the two adjacent chords are, at (R - r) cos(pi / S)
    for r in (R + 2.5, R + 0.001):
        p = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
        assert np.allclose(safety.distance_to_polyline(tr, p), r - R, atol=1e-9)
    for r in (R - 3.0, R - 0.5):
        p = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
        assert np.allclose(safety.distance_to_polyline(tr, p),
                           (R - r) * np.cos(np.pi / S), atol=1e-9)
    # on the bisector of a chord the nearest point is the chord's midpoint
    mid = ang + np.pi / S
    r = R + 1.0
    p = np.stack([r * np.cos(mid), r * np.sin(mid)], axis=1)
    want = r - R * np.cos(np.pi / S)
    assert np.allclose(safety.distance_to_polyline(tr, p), want, atol=1e-9)
    # a single segment: perpendicular distance inside, endpoint distance outside
    a, b = np.array([0.0, 0.0]), np.array([4.0, 0.0])
    p = np.array([[1.0, 3.0], [6.0, 0.0], [-3.0, -4.0]])
    assert np.allclose(safety.point_segment_distance(p, a, b), [3.0, 2.0, 5.0])


def test_track_spec_unsafe_off_road_and_fast():
    tr = data.track_polyline(0, circular=True)
    spec = safety.SafetySpec(lo=data.CAR_SAFE_LO, hi=data.CAR_SAFE_HI, track=tr,
                             half_width=4.0)
    R = data.TRACK_RADIUS
    z = np.zeros((4, 32))
    z[:, 0] = [R + 3.9, R - 4.1, R, R]
    z[:, 3] = [10, 10, 24.9, 25.0]
    assert safety.is_safe(spec, z).tolist() == [True, False, True, False]
    # the inflated barrier narrows the road to w - iota and the speed bound to 25 - iota
    spec.inflation = 0.5
    z[:, 0] = [R + 3.4, R + 3.7, R, R]
    z[:, 3] = [10, 10, 24.4, 24.6]
    assert safety.is_safe(spec, z).tolist() == [True, False, True, False]


# --------------------------------------------------------------------------- Alg. 2
def _drift(dt):
    return np.array([[1.0, dt], [0.0, 1.0]])  # x' = x + dt u, u held


def _drift_ttv(x0, dt, xi, H, lo=-1.0, hi=1.0):
    """Analytic steps passed before x0 + t dt xi leaves (lo, hi)."""
    if xi > 0:
        t_exit = math.ceil((hi - x0) / (dt * xi))
    elif xi < 0:
        t_exit = math.ceil((lo - x0) / (dt * xi))
    else:
        return H
    return min(max(t_exit - 1, 0), H)


def test_drift_model_ttv_and_selection_closed_form():
    dt, H, x0 = 0.05, 40, 0.3
    rng = np.random.default_rng(5)
    samples = rng.uniform(-1, 1, (300, 1))
    spec = safety.SafetySpec(lo=np.array([-1.0]), hi=np.array([1.0]))
    u_h = 0.9                                            # unsafe: exits at t ~ 16
    r = mpmi.tick(_drift(dt), "linear", [x0], [u_h], samples, H, spec)
    want = [_drift_ttv(x0, dt, c, H) for c in r.candidates[:, 0]]
    assert r.ttv.tolist() == want
    # safe iff x0 + H dt xi stays inside: xi in ((-1 - x0)/(H dt), (1 - x0)/(H dt))
    ok = (samples[:, 0] > (-1 - x0) / (H * dt)) & (samples[:, 0] < (1 - x0) / (H * dt))
    assert r.n_safe == int(ok.sum())
    best = samples[ok][np.argmin(np.abs(samples[ok, 0] - u_h))]
    assert r.status == mpmi.SAFE and r.u_r[0] == best[0]
    assert r.executed_steps == sum(min(t + 1, H) for t in want)


def test_all_unsafe_falls_back_to_longest_survivor():
    # values chosen off the lattice so no trajectory lands exactly on a bound
    dt, H, x0, u_h = 0.1, 200, 0.9513, 0.4871
    samples = np.array([[0.8137], [-0.1531], [0.0217], [-0.6], [0.0191]])
    spec = safety.SafetySpec(lo=np.array([-1.0]), hi=np.array([1.0]))
    r = mpmi.tick(_drift(dt), "linear", [x0], [u_h], samples, H, spec)
    ttv = [_drift_ttv(x0, dt, c, H) for c in r.candidates[:, 0]]
    assert r.ttv.tolist() == ttv and max(ttv) < H
    assert r.status == mpmi.FALLBACK and r.n_safe == 0
    # xi = -0.1531 leaves the lower bound last: 1.9513 / 0.01531 -> step 128
    assert r.index == 2 and r.ttv[2] == 127 and r.u_r[0] == -0.1531


def test_safe_user_input_passes_through_unchanged():
    x, u, xn = data.transitions("bot", 1, 3000)
    K, _ = fit.fit_koopman("bot", x, u, xn)
    spec = safety.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
    u_h = 0.01234567890123
    r = mpmi.tick(fit.round_to_f32(K), "bot", np.zeros(4), [u_h],
                  sampling.uniform_samples(1, 0, 0, 256, [-1], [1]), 20, spec)
    assert r.ttv[0] == 20 and r.index == 0 and r.status == mpmi.SAFE
    assert r.u_r[0] == u_h and mpmi.deviation(r.u_r, [u_h]) == 0.0


def test_monotone_in_horizon_and_nested_prefixes():
    x, u, xn = data.transitions("bot", 1, 3000)
    K = fit.round_to_f32(fit.fit_koopman("bot", x, u, xn)[0])
    spec = safety.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
    x_t = np.array([0.2, 0.5, 0.5, 0.0])
    s = sampling.uniform_samples(3, 0, 0, 2048, [-1], [1])
    r50 = mpmi.tick(K, "bot", x_t, [0.9], s, 50, spec)
    for h in (10, 30, 49):
        rh = mpmi.tick(K, "bot", x_t, [0.9], s, h, spec)
        assert np.array_equal(rh.ttv, np.minimum(r50.ttv, h))
    prev = np.inf
    for n in (64, 256, 1024, 2048):
        r = mpmi.tick(K, "bot", x_t, [0.9], s[:n], 30, spec, include_user=False)
        c = r.cost[r.index] if r.status == mpmi.SAFE else np.inf
        assert c <= prev
        prev = c


def test_selection_invariant_to_candidate_order():
    x, u, xn = data.transitions("bot", 1, 3000)
    K = fit.round_to_f32(fit.fit_koopman("bot", x, u, xn)[0])
    spec = safety.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
    x_t = np.array([0.25, 0.8, 0.0, 0.0])
    s = sampling.uniform_samples(4, 0, 0, 1024, [-1], [1])
    r = mpmi.tick(K, "bot", x_t, [0.7], s, 40, spec, include_user=False)
    perm = np.random.default_rng(6).permutation(1024)
    rp = mpmi.tick(K, "bot", x_t, [0.7], s[perm], 40, spec, include_user=False)
    assert rp.u_r[0] == r.u_r[0] and rp.status == r.status and rp.n_safe == r.n_safe
    assert np.array_equal(rp.ttv, r.ttv[perm])


# ------------------------------------------------------------ brute force, tiny N
def _bf_lift(kind, x, u):
    if kind == "bot":
        th, thd, p, v = x
        uu = u[0]
        return [th, thd, p, v, uu, math.sin(th), math.cos(th), thd * thd, thd * uu,
                thd * thd * math.sin(th), uu * math.cos(th), 1.0]
    px, py, psi, vx, vy, om = x
    d, a = u
    s, c = math.sin(psi), math.cos(psi)
    return [px, py, psi, vx, vy, om, d, a, s, c, vx * c, vx * s, vy * c, vy * s,
            om * vx, om * vy, vx * vx, vy * vy, om * om, d * vx, d * vy, d * om, a * vx,
            d * c, d * s, a * c, a * s, om * c, om * s, vx * vy, d * d, 1.0]


def _bf_dist(track, px, py):
    best = math.inf
    S = len(track)
    for i in range(S):
        ax, ay = track[i]
        bx, by = track[(i + 1) % S]
        dx, dy = bx - ax, by - ay
        t = ((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy)
        t = min(1.0, max(0.0, t))
        best = min(best, math.hypot(px - ax - t * dx, py - ay - t * dy))
    return best


def _bf_tick(kind, K, x_t, u_h, samples, H, lo, hi, track=None, w=0.0):
    cands = [list(u_h)] + [list(s) for s in samples]
    n = len(K)
    rows = []
    for slot, c in enumerate(cands):
        z = _bf_lift(kind, list(x_t), c)
        ttv = 0
        for t in range(1, H + 1):
            z = [sum(K[i][k] * z[k] for k in range(n)) for i in range(n)]
            ok = all(lo[j] < z[j] < hi[j] for j in range(len(lo)))
            if ok and track is not None:
                ok = _bf_dist(track, z[0], z[1]) < w
            if not ok:
                break
            ttv = t
        cost = sum((a - b) ** 2 for a, b in zip(c, u_h))
        rows.append((H - ttv, cost, slot, ttv))
    rows_sorted = sorted(rows)
    return rows, rows_sorted[0]


@pytest.mark.parametrize("kind", ["bot", "car"])
def test_brute_force_tiny(kind):
    if kind == "bot":
        x, u, xn = data.transitions("bot", 1, 2000)
        spec = safety.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
        x_t, H, lo, hi = np.array([0.3, 0.6, 1.2, 0.5]), 40, [-1.0], [1.0]
        track, w = None, 0.0
    else:
        x, u, xn = data.transitions("car", 3, 4000)
        track = data.track_polyline(3)
        spec = safety.SafetySpec(lo=data.CAR_SAFE_LO, hi=data.CAR_SAFE_HI, track=track,
                                 half_width=4.0)
        x_t, H = data.car_start_state(track, vx=14.0), 30
        lo, hi = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI
        w = 4.0
    K = fit.round_to_f32(fit.fit_koopman(kind, x, u, xn)[0])
    for seed in range(3):
        s = sampling.uniform_samples(seed, 0, 0, 63, lo, hi)
        u_h = data.to_f32_exact(data.user_input_once(seed, lo, hi))
        r = mpmi.tick(K, kind, x_t, u_h, s, H, spec)
        rows, best = _bf_tick(kind, K.tolist(), x_t.tolist(), u_h.tolist(), s.tolist(), H,
                              spec.lo.tolist(), spec.hi.tolist(),
                              None if track is None else track.tolist(), w)
        assert r.ttv.tolist() == [row[3] for row in rows]
        assert np.allclose(r.cost, [row[1] for row in rows], rtol=1e-15, atol=0)
        assert r.index == best[2]


def test_exact_ties_go_to_the_lowest_slot():
    """Brute force on candidates drawn from four values: every cost is shared by
    a dozen slots, and the pick is the lowest slot of the least-cost group that
    survives longest (the lexicographic minimum of (H - ttv, cost, slot))."""
    x, u, xn = data.transitions("bot", 1, 2000)
    K = fit.round_to_f32(fit.fit_koopman("bot", x, u, xn)[0])
    spec = safety.SafetySpec(lo=data.BOT_SAFE_LO, hi=data.BOT_SAFE_HI)
    rng = np.random.default_rng(13)
    s = rng.choice(np.array([-0.5, -0.25, 0.25, 0.5]), size=(47, 1))
    for x_t, u_h in ((np.array([0.05, 0.0, 0.0, 0.0]), [-0.25]),
                     (np.array([0.2, 0.4, 0.3, 0.1]), [0.25]),
                     (np.array([0.45, 1.5, 1.8, 1.0]), [0.5])):
        for include_user in (True, False):
            r = mpmi.tick(K, "bot", x_t, u_h, s, 30, spec, include_user=include_user)
            rows, best = _bf_tick("bot", K.tolist(), x_t.tolist(), list(u_h), s.tolist(), 30,
                                  spec.lo.tolist(), spec.hi.tolist())
            if not include_user:  # the brute force puts u_h in slot 0: drop it
                rows = [(a, b, c - 1, d) for a, b, c, d in rows[1:]]
                best = sorted(rows)[0]
            group = [row[2] for row in rows if row[:2] == best[:2]]
            assert len(group) > 1
            assert r.index == best[2] == min(group)

