"""Least-squares fit of the lifted linear operator K (Sec. IV-A).

The paper learns K from data with the EDMD family of methods (it cites
Williams et al. 2015 and sparsity-promoting DMD, Jovanovic et al. 2014).  With
the basis fixed (see ``basis``), EDMD reduces to ordinary least squares over the
lifted transition pairs:

    K = argmin_K  sum_m || Psi(x_{m+1}, u_m) - K Psi(x_m, u_m) ||^2

i.e. with the lifted snapshots stacked as rows, X K^T ~= Y, solved here with the
library least-squares routine in float64.  No regularisation, no sparsity
selection (readings stated in the design notes).  Because the input is held over
the horizon, each pure-input feature (u, delta, a, delta^2) and the constant
appear unchanged in Y: their column of Y is a column of X, so the exact
least-squares solution for their rows of K is the unit row (zero residual,
unique when X has full column rank).  The routine returns it up to rounding
(~1e-15); those rows are set to the exact unit rows, so a rollout carries the
held features unchanged.
"""
from __future__ import annotations

import numpy as np

from .basis import held_features, lift


def fit_koopman(basis: str, x: np.ndarray, u: np.ndarray, x_next: np.ndarray):
    """Return (K float64 n x n, relative residual ||X K^T - Y||_F / ||Y||_F)."""
    X = lift(basis, x, u)
    Y = lift(basis, x_next, u)
    kt, *_ = np.linalg.lstsq(X, Y, rcond=None)
    K = kt.T.copy()
    n = K.shape[0]
    nx = np.atleast_2d(x).shape[1]
    nu = np.atleast_2d(u).shape[1] if np.ndim(u) > 1 else 1
    for j in held_features(basis, nx, nu):
        K[j] = np.eye(n)[j]
    res = np.linalg.norm(X @ K.T - Y) / np.linalg.norm(Y)
    return K, float(res)


def round_to_f32(K: np.ndarray) -> np.ndarray:
    """K rounded to binary32 and promoted back: the operator a binary32 rollout holds."""
    return np.asarray(K, dtype=np.float32).astype(np.float64)


# ---- sparsity-promoting basis selection (Sec. IV-A, Sec. V-C.3) ----------------
#
# The paper selects its basis functions from random candidates with
# sparsity-promoting DMD (Jovanovic, Schmid & Nichols 2014), whose two stages are
# (1) a least-squares fit with an l1-type penalty, solved by ADMM, that zeroes
# whole terms, and (2) "polishing": an unpenalised least-squares refit on the
# terms that survived.  Reading (the paper's code is not available): the same two
# stages applied to the lifted regression X W ~= Y (W = K^T), with one penalty
# group per candidate feature -- the row W[j, :], i.e. feature j's influence on
# every predicted feature -- so a dropped feature leaves the model entirely.
# Columns of X and of Y are scaled to unit root-mean-square first, so one
# dimensionless gamma treats all features alike.  With A = X D^-1 and B = Y E^-1
# (D, E = diagonals of the column RMS values), V = D W E^-1:
#
#   minimise  (1/m) ||A V - B||_F^2 + gamma * sum_{j in C} ||V[j, :]||_2
#
# ADMM with the split V = Z, penalty parameter rho, scaled dual U (Boyd et al.
# 2011, group lasso):
#   V <- (2/m A^T A + rho I)^-1 (2/m A^T B + rho (Z - U))
#   Z[j] <- max(0, 1 - (gamma / rho) / ||(V + U)[j]||) (V + U)[j]   (j in C)
#   Z[j] <- (V + U)[j]                                              (j not in C)
#   U <- U + V - Z
# for a fixed number of iterations; the support is {j : Z[j] != 0} plus every
# feature outside C.  Polishing refits W by least squares on the support's
# columns of X; rows of W for dropped features are zero.

def group_lasso(A: np.ndarray, B: np.ndarray, candidates, gamma: float, rho: float = 1.0,
                iters: int = 400) -> np.ndarray:
    """Stage (1): the ADMM iterations above on already scaled A, B; returns Z."""
    m, n = A.shape
    cand = np.zeros(n, dtype=bool)
    cand[list(candidates)] = True
    G = 2.0 / m * (A.T @ A) + rho * np.eye(n)
    AtB = 2.0 / m * (A.T @ B)
    Z = np.zeros((n, B.shape[1]))
    U = np.zeros_like(Z)
    for _ in range(iters):
        V = np.linalg.solve(G, AtB + rho * (Z - U))
        P = V + U
        Z = P.copy()
        norms = np.linalg.norm(P, axis=1)
        for j in np.nonzero(cand)[0]:
            shrink = 1.0 - (gamma / rho) / norms[j] if norms[j] > 0 else 0.0
            Z[j] = max(0.0, shrink) * P[j]
        U = U + V - Z
    return Z


def rms_scale(M: np.ndarray) -> np.ndarray:
    """Column root-mean-square values (1 for an all-zero column)."""
    s = np.sqrt(np.mean(M * M, axis=0))
    s[s == 0] = 1.0
    return s


def select_columns(X: np.ndarray, Y: np.ndarray, candidates, gamma: float,
                   rho: float = 1.0, iters: int = 400):
    """Stages (1) and (2) on raw matrices.  Returns (W (n x p) with zero rows for
    dropped columns, support: boolean mask over the n columns of X)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[1]
    A = X / rms_scale(X)[None, :]
    B = Y / rms_scale(Y)[None, :]
    Z = group_lasso(A, B, candidates, gamma, rho, iters)
    cand = np.zeros(n, dtype=bool)
    cand[list(candidates)] = True
    support = ~cand | (np.linalg.norm(Z, axis=1) > 0)
    W = np.zeros((n, Y.shape[1]))
    cols = np.nonzero(support)[0]
    Ws, *_ = np.linalg.lstsq(X[:, cols], Y, rcond=None)
    W[cols] = Ws
    return W, support


def fit_koopman_sparse(basis: str, x: np.ndarray, u: np.ndarray, x_next: np.ndarray,
                       gamma: float, rho: float = 1.0, iters: int = 400):
    """K with a data-selected subset of the basis: the state features and the held
    features are always kept; the others compete under the group penalty.  A
    dropped feature has a zero column (no prediction reads it) and a zero row;
    held rows are the exact unit rows.  Returns (K, support mask, residual), the
    residual taken over the kept features (the ones the model predicts)."""
    X = lift(basis, x, u)
    Y = lift(basis, x_next, u)
    n = X.shape[1]
    nx = np.atleast_2d(x).shape[1]
    nu = np.atleast_2d(u).shape[1] if np.ndim(u) > 1 else 1
    held = set(held_features(basis, nx, nu))
    cand = [j for j in range(nx, n) if j not in held]
    W, support = select_columns(X, Y, cand, gamma, rho, iters)
    K = W.T.copy()
    for j in range(n):
        if not support[j]:
            K[j] = 0.0
    for j in held:
        K[j] = np.eye(n)[j]
    keep = np.nonzero(support)[0]
    res = np.linalg.norm((X @ K.T - Y)[:, keep]) / np.linalg.norm(Y[:, keep])
    return K, support, float(res)
