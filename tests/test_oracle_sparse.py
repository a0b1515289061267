"""Pins of the oracle's sparsity-promoting basis selection (Sec. IV-A, V-C.3):
exact support recovery and exact polishing on matrices with known zero rows,
the group-lasso optimality conditions at the ADMM solution, and the two limits
of the penalty on plant data."""
import numpy as np
import pytest

from oracle import basis, fit
from workloads import data


def _planted(seed=0, m=800, n=10, p=6, zero=(2, 5, 7)):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, n)) * rng.uniform(0.1, 10.0, n)
    W = rng.standard_normal((n, p))
    W[list(zero)] = 0.0
    return X, W, X @ W


@pytest.mark.parametrize("gamma", [1e-3, 1e-2, 0.05])
def test_planted_support_and_exact_polish(gamma):
    X, W, Y = _planted()
    Wh, support = fit.select_columns(X, Y, range(1, 10), gamma)
    assert support.tolist() == [w.any() for w in W]
    assert np.abs(Wh - W).max() < 1e-10


def test_zero_penalty_keeps_everything_and_equals_least_squares():
    X, _, _ = _planted(zero=())
    rng = np.random.default_rng(3)
    Y = X @ rng.standard_normal((10, 6)) + 0.1 * rng.standard_normal((800, 6))
    Wh, support = fit.select_columns(X, Y, range(10), 0.0)
    assert support.all()
    W_ne = np.linalg.solve(X.T @ X, X.T @ Y)                   # normal equations
    assert np.abs(Wh - W_ne).max() < 1e-8


@pytest.mark.parametrize("gamma", [0.02, 0.2])
def test_group_lasso_optimality_conditions(gamma):
    """Stage (1) solves min (1/m)||A V - B||^2 + gamma sum_j ||V_j||: at the
    solution the gradient row g_j = (2/m) A_j^T (B - A V) equals gamma V_j/||V_j||
    on kept groups and has norm <= gamma on dropped ones (penalised rows only)."""
    rng = np.random.default_rng(7)
    X, _, Y0 = _planted(seed=7, zero=(2, 5, 7))
    Y = Y0 + 0.5 * rng.standard_normal(Y0.shape)
    A = X / fit.rms_scale(X)[None, :]
    B = Y / fit.rms_scale(Y)[None, :]
    cand = list(range(1, 10))
    Z = fit.group_lasso(A, B, cand, gamma, iters=3000)
    grad = 2.0 / A.shape[0] * A.T @ (B - A @ Z)
    assert np.abs(grad[0]).max() < 1e-6                         # unpenalised row
    dropped = 0
    for j in cand:
        nz = np.linalg.norm(Z[j])
        if nz > 0:
            assert np.abs(grad[j] - gamma * Z[j] / nz).max() < 1e-5
        else:
            dropped += 1
            assert np.linalg.norm(grad[j]) <= gamma * (1 + 1e-6)
    assert dropped >= 3


def test_plant_limits_of_the_penalty():
    x, u, xn = data.transitions("bot", 1, 3000)
    K0, s0, r0 = fit.fit_koopman_sparse("bot", x, u, xn, 0.0)
    K, _ = fit.fit_koopman("bot", x, u, xn)
    assert s0.all() and np.abs(K0 - K).max() < 1e-8 and r0 > 0
    # a huge penalty keeps only the state and held features
    Kb, sb, _ = fit.fit_koopman_sparse("bot", x, u, xn, 1e6)
    held = basis.held_features("bot")
    assert np.nonzero(sb)[0].tolist() == sorted([0, 1, 2, 3] + list(held))
    X, Y = basis.lift("bot", x, u), basis.lift("bot", xn, u)
    cols = np.nonzero(sb)[0]
    Wk = np.linalg.solve(X[:, cols].T @ X[:, cols], X[:, cols].T @ Y[:, :4])
    assert np.abs(Kb[:4][:, cols] - Wk.T).max() < 1e-8          # polished state rows
    assert not Kb[:, ~sb].any() and not Kb[~sb].any()            # dropped: no column, no row
    for j in held:
        assert np.array_equal(Kb[j], np.eye(12)[j])
