"""Pins of the oracle's per-fold ridge / OLS models (oracle.ridge, oracle.press).

Each pin comes from outside the oracle's own arithmetic:
- the normal-equation solution against numpy.linalg.solve (a library routine)
  and the one-column closed form b = c / (a + lambda);
- the leave-one-out identity of ordinary least squares: with P = N folds,
  PRESS = sum_n (e_n / (1 - h_nn))^2, where e are the residuals and h the
  leverages of the fit on ALL rows.  Without preprocessing the design is X;
  with X and Y centered on the training rows the per-fold fit equals OLS with
  an intercept, so the design is [1 | X];
- invariances of OLS predictions: rescaling X's or Y's columns (the scale
  flags) changes no prediction, so PRESS does not change;
- brute force: the model fitted directly on each fold's explicitly
  preprocessed training rows, predicting its validation rows.
"""
import numpy as np
import pytest

import oracle

CX, SX, CY, SY = 1, 2, 4, 8


def _data(seed, N, K, M, mu=3.0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, K)) * rng.uniform(0.5, 2.0, K) + rng.uniform(-mu, mu, K)
    Bt = rng.standard_normal((K, M))
    Y = X @ Bt + 0.3 * rng.standard_normal((N, M)) + rng.uniform(-mu, mu, M)
    return X, Y


def _folds(seed, N, P):
    rng = np.random.default_rng(seed)
    f = np.arange(N) % P
    return rng.permutation(f).astype(np.int32)


@pytest.mark.parametrize("lam", [0.0, 0.5, 10.0])
@pytest.mark.parametrize("flags", [0, 5, 15])
def test_ridge_matches_library_solve(lam, flags):
    X, Y = _data(1, 60, 5, 3)
    folds = _folds(2, 60, 4)
    xtx, xty, _, _ = oracle.naive(X, Y, folds, 4, flags, 1)
    B, info = oracle.ridge(xtx, xty, lam)
    assert (info == 0).all()
    for p in range(4):
        ref = np.linalg.solve(xtx[p] + lam * np.eye(5), xty[p])
        np.testing.assert_allclose(B[p], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_ridge_one_column_closed_form():
    a = np.array([[[4.0]], [[0.25]]])
    c = np.array([[[2.0, -1.0]], [[1.0, 3.0]]])
    B, info = oracle.ridge(a, c, 0.75)
    assert (info == 0).all()
    np.testing.assert_allclose(B[:, 0, :], c[:, 0, :] / (a[:, 0, :] + 0.75), rtol=1e-15)


def test_ridge_reports_the_failing_pivot():
    A = np.stack([np.eye(4), np.eye(4)])
    A[1, 2, 2] = -1.0   # fold 1: the pivot of column 2 is negative
    C = np.ones((2, 4, 2))
    B, info = oracle.ridge(A, C, 0.0)
    assert list(info) == [0, 3]
    np.testing.assert_allclose(B[0], C[0])
    assert np.isnan(B[1]).all()
    B, info = oracle.ridge(A, C, -2.0)   # every fold fails at column 0
    assert list(info) == [1, 1]


def _loo_press_closed_form(D, Y):
    """PRESS of OLS on design D by the leave-one-out identity."""
    G = np.linalg.inv(D.T @ D)
    beta = G @ D.T @ Y
    e = Y - D @ beta
    h = np.einsum("ij,jk,ik->i", D, G, D)
    return ((e / (1.0 - h)[:, None]) ** 2).sum(axis=0)


@pytest.mark.parametrize("flags, intercept", [(0, False), (CX | CY, True)])
def test_press_leave_one_out_identity(flags, intercept):
    N, K, M = 30, 3, 2
    X, Y = _data(3, N, K, M)
    folds = np.arange(N, dtype=np.int32)   # P = N: leave-one-out
    xtx, xty, mean, std = oracle.naive(X, Y, folds, N, flags, 1)
    B, info = oracle.ridge(xtx, xty, 0.0)
    assert (info == 0).all()
    got = oracle.press(X, Y, folds, N, flags, mean, std, B).sum(axis=0)
    D = np.hstack([np.ones((N, 1)), X]) if intercept else X
    np.testing.assert_allclose(got, _loo_press_closed_form(D, Y), rtol=1e-9)


def test_press_ols_invariant_to_scaling():
    X, Y = _data(4, 80, 4, 3)
    folds = _folds(5, 80, 5)
    out = {}
    for flags in (CX | CY, CX | SX | CY, CX | CY | SY, 15):
        xtx, xty, mean, std = oracle.naive(X, Y, folds, 5, flags, 1)
        B, _ = oracle.ridge(xtx, xty, 0.0)
        out[flags] = oracle.press(X, Y, folds, 5, flags, mean, std, B)
    for flags, v in out.items():
        np.testing.assert_allclose(v, out[CX | CY], rtol=1e-9, err_msg=str(flags))


@pytest.mark.parametrize("flags", [0, 3, 5, 12, 15])
@pytest.mark.parametrize("ddof", [0, 1])
def test_press_brute_force(flags, ddof):
    """Fit each fold's ridge model on its explicitly preprocessed training rows
    and predict its validation rows."""
    N, K, M, P, lam = 50, 4, 2, 5, 2.0
    X, Y = _data(6, N, K, M)
    folds = _folds(7, N, P)
    xtx, xty, mean, std = oracle.naive(X, Y, folds, P, flags, ddof)
    B, _ = oracle.ridge(xtx, xty, lam)
    got = oracle.press(X, Y, folds, P, flags, mean, std, B)
    for p in range(P):
        tr, va = folds != p, folds == p
        mx, my = X[tr].mean(axis=0), Y[tr].mean(axis=0)
        sx, sy = X[tr].std(axis=0, ddof=ddof), Y[tr].std(axis=0, ddof=ddof)

        def prep(A, m, s, c, sc):
            return (A - (m if c else 0.0)) / (s if sc else 1.0)

        Xt = prep(X[tr], mx, sx, flags & CX, flags & SX)
        Yt = prep(Y[tr], my, sy, flags & CY, flags & SY)
        beta = np.linalg.solve(Xt.T @ Xt + lam * np.eye(K), Xt.T @ Yt)
        pred = prep(X[va], mx, sx, flags & CX, flags & SX) @ beta
        yhat = pred * (sy if flags & SY else 1.0) + (my if flags & CY else 0.0)
        np.testing.assert_allclose(got[p], ((Y[va] - yhat) ** 2).sum(axis=0), rtol=1e-9)
