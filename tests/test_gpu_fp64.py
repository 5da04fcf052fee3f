"""Parity of the FP64 CUDA path (CV_PREC_FP64) with the CPU oracle.

Tolerance: relative Frobenius error <= 1e-12 per fold and per product (the
FP64 target), plus the same bound on the correlation-scale error of X^T X.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import corr_scale_error, rel_fro_per_fold, run_library

pytestmark = pytest.mark.gpu
TOL = 1e-12


def xty_reference_flags(flags):
    """Lemma 9: X^T Y centered on either side equals the product with both sides
    centered.  The oracle's literal one-sided form sums (x - mean) * y with y
    uncentered and loses digits to cancellation when |mean(y)| >> std(y), so the
    X^T Y reference for one-sided centering is the both-sides form."""
    return flags | (cvx.CV_CENTER_X | cvx.CV_CENTER_Y) if flags & (cvx.CV_CENTER_X | cvx.CV_CENTER_Y) else flags


def _check(pr, flags, ddof, out_dtype=torch.float64, tol=TOL, **kw):
    xtx, xty, mean, std = run_library(pr, flags, ddof, "fp64", out_dtype, **kw)
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
    oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), ddof)[1] if pr.M else None
    e1 = rel_fro_per_fold(xtx, o[0])
    e2 = rel_fro_per_fold(xty, oy) if pr.M else 0.0
    e3 = corr_scale_error(xtx, o[0])
    assert e1 <= tol and e2 <= tol and e3 <= tol, (pr.name, flags, ddof, e1, e2, e3)
    np.testing.assert_allclose(mean, o[2], rtol=1e-12, atol=1e-12 * np.abs(o[2]).max())
    np.testing.assert_allclose(std, o[3], rtol=1e-11)
    assert np.array_equal(xtx, np.transpose(xtx, (0, 2, 1)))
    return e1, e2


@pytest.mark.parametrize("ddof", [0, 1])
def test_small_config_all_flags(ddof):
    pr = workloads.small_case()
    for flags in range(16):
        _check(pr, flags, ddof)


@pytest.mark.parametrize("N,K,M,P,scheme", [
    (700, 9, 3, 2, "random"),           # P = 2
    (150, 7, 2, 150, "venetian"),       # leave-one-out, P = N
    (2000, 30, 4, 9, "unbalanced"),
    (1500, 127, 0, 4, "random"),        # M = 0, D = 128 exactly
    (1300, 127, 1, 5, "contiguous"),    # D = 129: a second tile column
    (3001, 128, 3, 7, "venetian"),      # ragged segments, D crosses a tile
    (900, 1, 0, 3, "random"),           # one column
    (5000, 200, 9, 13, "unbalanced"),   # several tiles, several segments per fold
])
def test_shapes_and_partitionings(N, K, M, P, scheme):
    pr = workloads.random_case(101 + K, N, K, M, P, scheme=scheme)
    for flags in (0, 1, 4, 5, 10, 15):
        _check(pr, flags, 1)


@pytest.mark.parametrize("in_dtype,out_dtype", [(np.float32, torch.float64), (np.float64, torch.float32),
                                                (np.float32, torch.float32)])
def test_dtypes(in_dtype, out_dtype):
    pr = workloads.random_case(5, 1200, 40, 3, 6, dtype=in_dtype, offset=30.0)
    tol = TOL if out_dtype == torch.float64 else 2e-7
    for flags in (0, 5, 15):
        _check(pr, flags, 1, out_dtype=out_dtype, tol=tol)


def test_large_offsets_fp32():
    """mu = 1e3, sigma ~ 1: centered products must not lose digits."""
    pr = workloads.offset_case(N=20000, K=64, M=4, P=5)
    for flags in (1, 5, 15, 0):
        _check(pr, flags, 1)


def test_constant_and_integer_columns():
    pr = workloads.random_case(9, 600, 6, 2, 4)
    X = pr.X.copy()
    X[:, 1] = 7.0        # constant: sigma = 0 -> replaced by 1
    X[:, 4] = -3.0
    pr.X = X
    pr.Y = pr.Y.copy()
    pr.Y[:, 0] = 2.0
    for flags in range(16):
        _check(pr, flags, 1)


def test_host_fold_ids_and_sort_matches_algorithm1():
    for N, P, scheme in [(5000, 7, "random"), (20000, 300, "unbalanced"), (70000, 700, "venetian"),
                         (3000, 2, "contiguous")]:
        pr = workloads.random_case(3, N, 2, 1, P, scheme=scheme)
        for on_dev in (True, False):
            folds = torch.from_numpy(pr.folds).cuda() if on_dev else pr.folds
            plan = cvx.cv_plan(N, 2, 1, P, folds, torch.float64, torch.float64, "fp64")
            off, rows = oracle.validation_partitions(pr.folds, P)
            assert np.array_equal(cvx.cv_plan_fold_offsets(plan), off)
            assert np.array_equal(cvx.cv_plan_permutation(plan).astype(np.int64), rows)


def test_errors():
    X = torch.randn(10, 3, device="cuda", dtype=torch.float64)
    Y = torch.randn(10, 1, device="cuda", dtype=torch.float64)
    bad = torch.tensor([0, 1, 2, 3, 0, 1, 2, 3, 0, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_plan(10, 3, 1, 4, bad, torch.float64, torch.float64, "fp64")
    assert e.value.name == "CV_ERR_FOLD_RANGE"
    neg = torch.tensor([0, 1, 2, -1, 0, 1, 2, 3, 0, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_plan(10, 3, 1, 4, neg, torch.float64, torch.float64, "fp64")
    assert e.value.name == "CV_ERR_FOLD_RANGE"
    empty = torch.tensor([0, 1, 0, 1, 0, 1, 3, 3, 0, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_plan(10, 3, 1, 4, empty, torch.float64, torch.float64, "fp64")
    assert e.value.name == "CV_ERR_EMPTY_FOLD"
    # fold 0 holds 9 of 10 rows: its training partition has one row
    lone = torch.tensor([0] * 9 + [1], dtype=torch.int32, device="cuda")
    plan = cvx.cv_plan(10, 3, 1, 2, lone, torch.float64, torch.float64, "fp64")
    with pytest.raises(cvx.CVError) as e:
        cvx.products(X, Y, lone, 2, cvx.CV_SCALE_X, 1, plan=plan)
    assert e.value.name == "CV_ERR_NOT_SCALABLE"
    cvx.products(X, Y, lone, 2, cvx.CV_SCALE_X, 0, plan=plan)      # ddof 0: fine
    cvx.products(X, Y, lone, 2, cvx.CV_CENTER_X, 1, plan=plan)     # no scaling: fine
    with pytest.raises(cvx.CVError):
        cvx.products(X, Y, lone, 2, 16, 1, plan=plan)
    with pytest.raises(cvx.CVError):
        cvx.products(X, Y, lone, 2, 1, 2, plan=plan)


def test_deterministic():
    pr = workloads.random_case(17, 4000, 70, 5, 6, scheme="random")
    a = run_library(pr, 15, 1, "fp64")
    b = run_library(pr, 15, 1, "fp64")
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_wide_range_full_size_sampled():
    """N=1e5, K=500, M=10, P=10 contiguous folds (the benchmark workload), FP64
    inputs: sampled entries against the oracle computed one by one, plus
    properties that hold at any size."""
    pr = workloads.wide_range_case(dtype=np.float64)
    flags, ddof = 15, 1
    xtx, xty, mean, std = run_library(pr, flags, ddof, "fp64")
    rng = np.random.default_rng(0)
    samples = [(int(rng.integers(pr.P)), 0, int(rng.integers(pr.K)), int(rng.integers(pr.K)))
               for _ in range(60)]
    samples += [(int(rng.integers(pr.P)), 1, int(rng.integers(pr.K)), int(rng.integers(pr.M)))
                for _ in range(40)]
    samples += [(p, 0, pr.K - 1, pr.K - 1) for p in range(pr.P)]
    ref = oracle.naive_entries(pr.X, pr.Y, pr.folds, pr.P, flags, ddof, samples)
    counts = np.bincount(pr.folds, minlength=pr.P)
    for (p, w, i, j), r in zip(samples, ref):
        got = (xtx if w == 0 else xty)[p, i, j]
        scale = pr.N - counts[p] - ddof          # centered-scaled diagonal
        assert abs(got - r) <= TOL * scale, (p, w, i, j, got, r)
    for p in range(pr.P):
        np.testing.assert_allclose(np.diag(xtx[p]), pr.N - counts[p] - ddof, rtol=1e-12)
