"""cv_products_f64_static: the allocation-free entry point.

It serves callers that cannot allocate device memory (a process whose GPU
memory another framework's allocator owns under a fixed budget, or a loop
where a cudaMalloc's device synchronization and possible failure are not
acceptable).  This file runs last so that, if it fails, every other test has
already run.  It checks, through the C ABI, that two calls in a row (the
second one reusing the scratch array the first left behind) give the
products of the plan-based cv_products within the FP64 path's tolerance.
"""
import numpy as np
import pytest
import torch

import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import rel_fro_per_fold

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _plan_based(pr, flags, ddof):
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    xtx, xty, mean, std = cvx.products(X, Y, f, pr.P, flags, ddof, "fp64", torch.float64, with_stats=True)
    return xtx, xty, mean, std


def _static(pr, flags, ddof):
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    xtx = torch.full((pr.P, pr.K, pr.K), float("nan"), dtype=torch.float64, device=dev)
    xty = torch.full((pr.P, pr.K, pr.M), float("nan"), dtype=torch.float64, device=dev)
    mean = torch.empty((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev)
    std = torch.empty((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev)
    cvx.cv_products_f64_static(X, Y, f, pr.P, flags, ddof, xtx, xty, mean, std)
    torch.cuda.synchronize()
    return xtx, xty, mean, std


def test_two_calls_match_plan_based_products():
    first = workloads.random_case(31, 3000, 40, 3, 7, dtype=np.float32, scheme="random", offset=25.0)
    second = workloads.random_case(32, 20000, 100, 5, 16, dtype=np.float64, scheme="unbalanced")
    for pr, flags in ((first, 15), (second, 5)):
        got = _static(pr, flags, 1)
        ref = _plan_based(pr, flags, 1)
        xtx, xty = got[0].cpu().numpy(), got[1].cpu().numpy()
        assert rel_fro_per_fold(xtx, ref[0].cpu().numpy()) <= TOL
        assert rel_fro_per_fold(xty, ref[1].cpu().numpy()) <= TOL
        np.testing.assert_allclose(got[2].cpu().numpy(), ref[2].cpu().numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got[3].cpu().numpy(), ref[3].cpu().numpy(), rtol=1e-12)


def test_sizes_beyond_the_limit_are_rejected():
    pr = workloads.random_case(3, 40000, 8, 1, 4)
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    out = torch.empty((4, 8, 8), dtype=torch.float64, device=dev)
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_products_f64_static(X, Y, f, 4, 15, 1, out, None)
    assert e.value.name == "CV_ERR_UNSUPPORTED"
