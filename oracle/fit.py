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
