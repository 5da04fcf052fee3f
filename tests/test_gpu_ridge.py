"""Per-fold ridge / OLS models on the products (cv_ridge, cv_ridge_press)
against the oracle.

Each stage is checked on its own inputs: cv_ridge against the oracle's
Cholesky solve of the SAME products (error bound: a backward-stable solve
gives a relative error below about cond(A) * K * eps, so the tolerance is
1e3 * cond * eps), and cv_ridge_press against the oracle's validation error
for the SAME coefficients and statistics (FP64 sums in another order:
1e-10 relative).  End to end, the FP64 path is compared with the oracle's
products, models and errors.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _run(pr, flags, ddof, lam, prec, in_dtype):
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X.astype(in_dtype)).to(dev)
    Y = torch.from_numpy(pr.Y.astype(in_dtype)).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, X.dtype, torch.float64, prec)
    XTX = torch.empty((pr.P, pr.K, pr.K), dtype=torch.float64, device=dev)
    XTY = torch.empty((pr.P, pr.K, pr.M), dtype=torch.float64, device=dev)
    mean = torch.empty((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev)
    std = torch.empty_like(mean)
    cvx.cv_products(plan, X, Y, flags, ddof, XTX, XTY, mean, std)
    B, info = cvx.cv_ridge(XTX, XTY, lam)
    press = cvx.cv_ridge_press(plan, X, Y, flags, mean, std, B)
    torch.cuda.synchronize()
    assert cvx.cv_plan_status(plan) == 0
    return tuple(t.cpu().numpy() for t in (XTX, XTY, mean, std, B, info, press))


def _check_stages(pr, flags, xtx, xty, mean, std, B, info, press, lam):
    assert (info == 0).all()
    Bo, info_o = oracle.ridge(xtx, xty, lam)
    assert (info_o == 0).all()
    for p in range(pr.P):
        cond = np.linalg.cond(xtx[p] + lam * np.eye(pr.K))
        err = np.abs(B[p] - Bo[p]).max() / np.abs(Bo[p]).max()
        assert err <= max(1e-13, 1e3 * cond * EPS), (p, err, cond)
    po = oracle.press(pr.X, pr.Y, pr.folds, pr.P, flags, mean, std, B)
    np.testing.assert_allclose(press, po, rtol=1e-10)


@pytest.mark.parametrize("flags", [0, 5, 15])
@pytest.mark.parametrize("lam", [0.0, 3.0])
def test_fp64_end_to_end(flags, lam):
    pr = workloads.small_case(dtype=np.float64)
    xtx, xty, mean, std, B, info, press = _run(pr, flags, 1, lam, "fp64", np.float64)
    _check_stages(pr, flags, xtx, xty, mean, std, B, info, press, lam)
    ox, oy, om, osd = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, 1)
    Bo, _ = oracle.ridge(ox, oy, lam)
    po = oracle.press(pr.X, pr.Y, pr.folds, pr.P, flags, om, osd, Bo)
    conds = [np.linalg.cond(ox[p] + lam * np.eye(pr.K)) for p in range(pr.P)]
    np.testing.assert_allclose(press, po, rtol=max(1e-9, 1e-12 * max(conds)))


@pytest.mark.parametrize("N,K,M,P,scheme,prec", [
    (3001, 130, 3, 7, "venetian", "fp16x3"),   # FP32 inputs, split precision products
    (2000, 300, 20, 4, "random", "fp64"),       # K > block size, M > responses per pass
    (900, 17, 9, 3, "unbalanced", "bf16x3"),
])
def test_shapes(N, K, M, P, scheme, prec):
    pr = workloads.random_case(300 + K, N, K, M, P, dtype=np.float32, scheme=scheme)
    for flags in (5, 15):
        xtx, xty, mean, std, B, info, press = _run(pr, flags, 1, 1.0, prec, np.float32)
        _check_stages(pr, flags, xtx, xty, mean, std, B, info, press, 1.0)


def test_leave_one_out_identity():
    """P = N, OLS on X and Y centered per fold: the leave-one-out identity of
    OLS with an intercept gives the total error from one fit on all rows."""
    pr = workloads.random_case(77, 64, 4, 2, 64, dtype=np.float64, scheme="venetian")
    _, _, _, _, B, info, press = _run(pr, 5, 1, 0.0, "fp64", np.float64)
    assert (info == 0).all()
    D = np.hstack([np.ones((pr.N, 1)), pr.X])
    G = np.linalg.inv(D.T @ D)
    e = pr.Y - D @ (G @ D.T @ pr.Y)
    h = np.einsum("ij,jk,ik->i", D, G, D)
    np.testing.assert_allclose(press.sum(axis=0), ((e / (1.0 - h)[:, None]) ** 2).sum(axis=0), rtol=1e-9)


def test_not_positive_definite_is_reported():
    dev = torch.device("cuda:0")
    pr = workloads.random_case(5, 500, 6, 2, 3, dtype=np.float64)
    xtx, xty, _, _ = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, 15, 1)
    A = torch.from_numpy(xtx).to(dev)
    C = torch.from_numpy(xty).to(dev)
    lam = -(float(np.max(np.diagonal(xtx, axis1=1, axis2=2))) + 1.0)
    B, info = cvx.cv_ridge(A, C, lam)
    assert (info.cpu().numpy() == 1).all()
    assert torch.isnan(B).all()
    # fold 1 fails at column 2 only
    xtx2 = np.stack([np.eye(6)] * 3)
    xtx2[1, 2, 2] = -1.0
    B, info = cvx.cv_ridge(torch.from_numpy(xtx2).to(dev), C, 0.0)
    assert list(info.cpu().numpy()) == [0, 3, 0]
    np.testing.assert_allclose(B[0].cpu().numpy(), xty[0], rtol=1e-15)


@pytest.mark.parametrize("K,M", [(1, 1), (31, 1), (32, 8), (33, 9), (65, 17), (100, 3), (161, 0)])
def test_blocked_factor_at_block_edges(K, M):
    """The factor is built in 32 x 32 blocks and the solve takes up to 8
    responses per block: sizes on both sides of those edges, against the
    oracle's solve (B) and NumPy's Cholesky factor (L, row-major, zero above
    the diagonal)."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(1000 + K + M)
    P, lam = 3, 0.25
    Z = rng.standard_normal((P, 3 * K + 4, K))
    xtx = np.einsum("pnk,pnj->pkj", Z, Z)
    xty = rng.standard_normal((P, K, M))
    L = torch.full((P, K, K), 7.0, dtype=torch.float64, device=dev)   # the factor overwrites every entry
    B, info = cvx.cv_ridge(torch.from_numpy(xtx).to(dev), torch.from_numpy(xty).to(dev), lam, L=L)
    assert (info.cpu().numpy() == 0).all()
    Lh = L.cpu().numpy()
    for p in range(P):
        A = xtx[p] + lam * np.eye(K)
        Lo = np.linalg.cholesky(A)
        assert np.abs(Lh[p] - Lo).max() <= 1e-12 * np.abs(Lo).max(), p
        assert not np.triu(Lh[p], 1).any()
    if M > 0:
        Bo, _ = oracle.ridge(xtx, xty, lam)
        for p in range(P):
            cond = np.linalg.cond(xtx[p] + lam * np.eye(K))
            err = np.abs(B[p].cpu().numpy() - Bo[p]).max() / np.abs(Bo[p]).max()
            assert err <= max(1e-13, 1e3 * cond * EPS), (p, err, cond)


def test_failure_in_a_later_block():
    """A pivot that fails in the second block column stops that fold only:
    info is the failing column + 1, its B is NaN, the other folds solve."""
    dev = torch.device("cuda:0")
    K, M = 70, 9
    xtx = np.stack([np.eye(K) * 2.0] * 3)
    xtx[1, 45, 45] = -1.0
    xty = np.random.default_rng(3).standard_normal((3, K, M))
    B, info = cvx.cv_ridge(torch.from_numpy(xtx).to(dev), torch.from_numpy(xty).to(dev), 0.0)
    assert list(info.cpu().numpy()) == [0, 46, 0]
    Bh = B.cpu().numpy()
    assert np.isnan(Bh[1]).all()
    np.testing.assert_allclose(Bh[[0, 2]], xty[[0, 2]] / 2.0, rtol=1e-15)


def test_argument_errors():
    dev = torch.device("cuda:0")
    A = torch.eye(3, dtype=torch.float64, device=dev)[None]
    C = torch.ones((1, 3, 1), dtype=torch.float64, device=dev)
    with pytest.raises(cvx.CVError):
        cvx.cv_ridge(A, C, float("nan"))
    with pytest.raises(ValueError):
        cvx.cv_ridge(A.float(), C, 0.0)
