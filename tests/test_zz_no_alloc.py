"""cv_products_f64_static: the allocation-free entry point.

It serves callers that cannot allocate device memory (a process whose GPU
memory another framework's allocator owns under a fixed budget, or a loop
where a cudaMalloc's device synchronization and possible failure are not
acceptable).  This file runs last so that, if it fails, every other test has
already run.  Through the C ABI it checks that calls in a row, each reusing
the scratch array the previous one left behind (a larger problem after a
smaller one, then a smaller one after a larger one), give the products of
the plan-based cv_products within the FP64 path's tolerance and match the
CPU oracle element by element; that the limits themselves work; and that
bad fold ids and oversized problems are refused with the documented codes.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import corr_scale_error, rel_fro_per_fold

pytestmark = pytest.mark.gpu
TOL = 1e-12          # FP64 outputs: the FP64 path's bound against the oracle
TOL_F32_OUT = 1e-6   # FP32 outputs: one FP32 rounding of each output entry (2^-24) plus the FP64 path's error


def _dev_inputs(pr):
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev) if pr.M > 0 else None
    f = torch.from_numpy(pr.folds).to(dev)
    return X, Y, f


def _plan_based(pr, flags, ddof, out_dtype):
    X, Y, f = _dev_inputs(pr)
    return cvx.products(X, Y, f, pr.P, flags, ddof, "fp64", out_dtype, with_stats=True)


def _static(pr, flags, ddof, out_dtype):
    X, Y, f = _dev_inputs(pr)
    dev = X.device
    xtx = torch.full((pr.P, pr.K, pr.K), float("nan"), dtype=out_dtype, device=dev)
    xty = torch.full((pr.P, pr.K, pr.M), float("nan"), dtype=out_dtype, device=dev) if pr.M > 0 else None
    mean = torch.empty((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev)
    std = torch.empty((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev)
    cvx.cv_products_f64_static(X, Y, f, pr.P, flags, ddof, xtx, xty, mean, std)
    torch.cuda.synchronize()
    return xtx, xty, mean, std


def _np(t, pr):
    return t.double().cpu().numpy() if t is not None else np.zeros((pr.P, pr.K, 0))


def _check_case(pr, flags, ddof, out_dtype):
    tol = TOL if out_dtype == torch.float64 else TOL_F32_OUT
    got = _static(pr, flags, ddof, out_dtype)
    ref = _plan_based(pr, flags, ddof, out_dtype)
    xtx, xty = _np(got[0], pr), _np(got[1], pr)
    # against the plan-based entry point
    assert rel_fro_per_fold(xtx, _np(ref[0], pr)) <= tol
    if pr.M > 0:
        assert rel_fro_per_fold(xty, _np(ref[1], pr)) <= tol
    # against the oracle (Algorithms 2/4/6), element by element
    o = oracle.naive(pr.X, pr.Y if pr.M > 0 else None, pr.folds, pr.P, flags, ddof)
    assert rel_fro_per_fold(xtx, o[0]) <= tol
    assert corr_scale_error(xtx, o[0]) <= tol
    if pr.M > 0:
        assert rel_fro_per_fold(xty, o[1]) <= tol
    np.testing.assert_allclose(got[2].cpu().numpy(), o[2], rtol=1e-12, atol=1e-12 * np.abs(o[2]).max())
    np.testing.assert_allclose(got[3].cpu().numpy(), o[3], rtol=1e-12)


def test_two_calls_match_plan_based_products():
    prev = oracle.set_threads(0)
    try:
        # smaller, then larger (more folds, wider), then smaller again with
        # fewer folds, a narrower W, no Y, ddof 0 and FP32 outputs: every call
        # must overwrite what the previous one left in the scratch array
        first = workloads.random_case(31, 3000, 40, 3, 7, dtype=np.float32, scheme="random", offset=25.0)
        second = workloads.random_case(32, 20000, 100, 5, 16, dtype=np.float64, scheme="unbalanced")
        third = workloads.random_case(33, 1500, 10, 0, 3, dtype=np.float32, scheme="contiguous", offset=-4.0)
        _check_case(first, 15, 1, torch.float64)
        _check_case(second, 5, 1, torch.float64)
        _check_case(third, 3, 0, torch.float32)
        _check_case(first, 10, 0, torch.float64)
    finally:
        oracle.set_threads(prev)


def test_at_the_limits():
    """N = 32768 rows, P = 16 folds and K + M + 1 = 128 columns: the largest
    problem the fixed scratch array holds."""
    prev = oracle.set_threads(0)
    try:
        pr = workloads.random_case(34, 32768, 120, 7, 16, dtype=np.float32, scheme="random", offset=10.0)
        _check_case(pr, 15, 1, torch.float64)
    finally:
        oracle.set_threads(prev)


def test_bad_fold_ids_are_rejected():
    pr = workloads.random_case(35, 2000, 12, 2, 5, dtype=np.float32)
    X, Y, f = _dev_inputs(pr)
    out = torch.empty((5, 12, 12), dtype=torch.float64, device=X.device)
    bad = f.clone()
    bad[17] = 5                      # outside [0, P)
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_products_f64_static(X, Y, bad, 5, 15, 1, out, None)
    assert e.value.name == "CV_ERR_FOLD_RANGE"
    empty = torch.where(f == 3, torch.zeros_like(f), f)   # fold 3 has no row
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_products_f64_static(X, Y, empty, 5, 15, 1, out, None)
    assert e.value.name == "CV_ERR_EMPTY_FOLD"
    # the next valid call is unaffected
    _check_case(pr, 15, 1, torch.float64)


def test_sizes_beyond_the_limit_are_rejected():
    pr = workloads.random_case(3, 40000, 8, 1, 4)
    X, Y, f = _dev_inputs(pr)
    out = torch.empty((4, 8, 8), dtype=torch.float64, device=X.device)
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_products_f64_static(X, Y, f, 4, 15, 1, out, None)
    assert e.value.name == "CV_ERR_UNSUPPORTED"
    pr = workloads.random_case(4, 1000, 120, 8, 4)       # K + M + 1 = 129
    X, Y, f = _dev_inputs(pr)
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_products_f64_static(X, Y, f, 4, 15, 1, None, None)
    assert e.value.name == "CV_ERR_UNSUPPORTED"
