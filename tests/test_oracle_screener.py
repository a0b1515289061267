"""Pins of the screener reference (oracle/screener.py): GELU identities, the
chain-rule backward against central finite differences, Adam's first step in
closed form, track features on a circle in closed form, the screening order."""
import math

import numpy as np
import pytest

from oracle import screener as sc
from workloads import data


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    assert sc.gelu(np.array(0.0)) == 0.0
    # tanh is odd, so gelu(x) - gelu(-x) = x
    assert np.allclose(sc.gelu(x) - sc.gelu(-x), x, atol=1e-15)
    assert np.allclose(sc.gelu(np.array([30.0, -30.0])), [30.0, 0.0], atol=1e-12)
    # close to the exact erf form (the approximation's published accuracy)
    from scipy.special import erf
    exact = 0.5 * x * (1 + erf(x / math.sqrt(2)))
    assert np.max(np.abs(sc.gelu(x) - exact)) < 1e-3
    h = 1e-6
    fd = (sc.gelu(x + h) - sc.gelu(x - h)) / (2 * h)
    assert np.allclose(sc.gelu_grad(x), fd, atol=1e-8)


def _small_problem(seed=0, B=6):
    rng = np.random.default_rng(seed)
    p = data.screener_init(seed, hidden=9, n_in=12)
    p["b1"] = rng.normal(0, 0.1, 9)
    p["b2"] = rng.normal(0, 0.1, 9)
    p["b3"] = np.array(0.3)
    f = rng.normal(0, 1, (B, 12))
    t = rng.uniform(0, 1, B)
    return p, f, t


def test_backward_matches_finite_differences():
    p, f, t = _small_problem()
    g = sc.backward(p, sc.forward(p, f), t)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k].reshape(-1)[idx] += h
            lp = sc.loss(sc.forward(q, f)["y"], t)
            q[k].reshape(-1)[idx] -= 2 * h
            lm = sc.loss(sc.forward(q, f)["y"], t)
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 + 1e-5 * abs(fd), (k, idx, fd, an)


def test_adam_first_step_is_signed_learning_rate():
    p, f, t = _small_problem(2)
    g = sc.backward(p, sc.forward(p, f), t)
    q = {k: v.copy() for k, v in p.items()}
    sc.adam_step(q, g, {}, step=1, lr=1e-3, eps=0.0)
    for k in p:
        nz = g[k] != 0
        assert np.allclose((q[k] - p[k])[nz], -1e-3 * np.sign(g[k][nz]), rtol=1e-12)


def test_circle_curvature_and_lookahead():
    tr = data.track_polyline(0, circular=True)
    kappa = sc.vertex_curvature(tr)
    assert np.allclose(kappa, 1.0 / data.TRACK_RADIUS, rtol=1e-12)   # counter-clockwise: left
    assert np.allclose(sc.lookahead_table(tr), 1.0 / data.TRACK_RADIUS, rtol=1e-12)
    assert np.allclose(sc.vertex_curvature(tr[::-1]), -1.0 / data.TRACK_RADIUS, rtol=1e-12)


def test_lookahead_walks_arc_length():
    # a square-ish closed track with unit spacing: the vertex 5 m ahead is 5 vertices on
    pts = [(x, 0.0) for x in range(20)] + [(20.0, y) for y in range(20)] + \
          [(x, 20.0) for x in range(20, 0, -1)] + [(0.0, y) for y in range(20, 0, -1)]
    tr = np.array(pts, dtype=float)
    kappa = sc.vertex_curvature(tr)
    look = sc.lookahead_table(tr)
    for i in (0, 7, 33, 79):
        for m, ell in enumerate(sc.LOOKAHEAD_M):
            assert look[i, m] == kappa[(i + int(ell)) % len(tr)]


def test_features_on_circle_chord_bisector():
    tr = data.track_polyline(0, circular=True)
    S, R, w = len(tr), data.TRACK_RADIUS, 4.0
    i = 17
    mid = 2 * np.pi * (i + 0.5) / S
    r = R * np.cos(np.pi / S) - 1.5            # 1.5 m inside the chord, left of the track
    x = np.array([r * np.cos(mid), r * np.sin(mid), mid + np.pi / 2, 12.5, -0.5, 0.4])
    f = sc.tick_features(tr, w, x)
    assert f[0] == pytest.approx(1.5 / w, abs=1e-9)
    assert f[1] == pytest.approx(0.0, abs=1e-9) and f[2] == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(f[3:6], [0.5, -0.1, 0.2])
    assert np.allclose(f[6:], 10.0 / R, rtol=1e-9)
    c = sc.candidate_features(f, np.array([[0.2, -0.5], [-0.4, 1.0]]))
    assert c.shape == (2, 12) and np.allclose(c[:, 10:], [[0.5, -0.5], [-1.0, 1.0]])
    # heading 0.3 rad to the left of the chord's direction: heading error +0.3
    x[2] += 0.3
    f = sc.tick_features(tr, w, x)
    assert f[1] == pytest.approx(math.sin(0.3), abs=1e-9)
    assert f[2] == pytest.approx(math.cos(0.3), abs=1e-9)


def test_cost_bins_follow_the_cost_order():
    c = np.array([0.0, 1e-30, 0.125, 0.5, 0.51, 0.5625, 1.0, 4.64], dtype=np.float32)
    b = sc.cost_bin(c)
    assert np.all(np.diff(b) >= 0) and b[0] == 0
    # 0.5 and 0.51 share the bin [0.5, 0.5625) (three mantissa bits); 0.5625 opens the next
    assert b[3] == b[4] and b[5] == b[4] + 1
    assert b.max() < 2048  # the device histograms have 2048 bins


def test_screen_keeps_the_cost_prefix_the_scores_ask_for():
    # costs in distinct bins; order by cost: 0, 5, 2, 1, 3, 4
    cost = np.array([0.0, 0.5, 0.25, 1.0, 2.0, 0.125])
    scores = np.array([0.1, 0.95, 0.2, 0.99, 0.97, 0.3])
    assert sc.screen(scores, cost, 3, 0.0).tolist() == [0, 2, 5]
    assert sc.screen(scores, cost, 1, 0.9, m=1).tolist() == [0, 1, 2, 5]
    assert sc.screen(scores, cost, 1, 0.9, m=2).tolist() == [0, 1, 2, 3, 5]
    assert sc.screen(scores, cost, 5, 0.9, m=1).tolist() == [0, 1, 2, 3, 5]
    assert sc.screen(scores, cost, 1, 0.9, m=4).tolist() == [0, 1, 2, 3, 4, 5]  # only 3
    assert sc.screen(scores, cost, 1, 0.05, m=1).tolist() == [0]
    # a shared bin is kept whole
    cost2 = np.array([0.0, 0.5, 0.51, 1.0])
    assert sc.screen(np.zeros(4), cost2, 2, 0.0).tolist() == [0, 1, 2]


def test_screened_selection_is_exhaustive_for_any_scores():
    """Brute force over random ticks (random safety, random and adversarial
    scores): the kept prefix either holds the least-cost safe slot or only unsafe
    slots, so the screened selection equals the exhaustive one."""
    rng = np.random.default_rng(11)
    H = 7
    for trial in range(3000):
        n = int(rng.integers(1, 40))
        cost = rng.choice([0.0, 0.01, 0.02, 0.1, 0.3, 0.31, 1.0, 2.5], n)
        cost = (cost + rng.uniform(0, 0.05, n) * rng.integers(0, 2, n)).astype(np.float32)
        ttv = np.where(rng.random(n) < rng.random(), H, rng.integers(0, H, n))
        kind = trial % 3
        scores = (rng.random(n) if kind == 0 else
                  (ttv == H) * 1.0 if kind == 1 else (ttv != H) * 1.0)
        k = int(rng.integers(1, n + 1))
        tau = float(rng.choice([0.0, 0.5, 0.9]))
        m = int(rng.integers(1, 6))
        kept = sc.screen(scores, cost, k, tau, m)
        got = sc.screened_selection(ttv, cost.astype(np.float64), kept, H)
        # exhaustive by scalar loops: max ttv, then min cost, then min slot
        best = 0
        for i in range(1, n):
            if (H - ttv[i], cost[i], i) < (H - ttv[best], cost[best], best):
                best = i
        assert got == best
