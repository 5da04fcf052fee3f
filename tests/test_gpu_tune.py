"""cv_plan_tune on the GPU: it measures the candidate plan options of a
problem, returns the fastest and records it in the cache, a second call takes
the cached entry without measuring, and a plan made with the chosen options
(or with the explicit small-fold strategy on folds larger than its automatic
threshold) matches the oracle (Algorithms 2/4/6)."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import rel_fro_per_fold

pytestmark = pytest.mark.gpu
TOLS = {"fp64": 1e-12, "fp16x3": 2e-6}


def _inputs(pr):
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    return X, Y, f


def test_tune_measures_caches_and_reuses(tmp_path):
    pr = workloads.random_case(601, 20000, 100, 3, 200, dtype=np.float32, scheme="random", offset=10.0)
    X, Y, f = _inputs(pr)
    path = str(tmp_path / "tune.json")
    key = cvx.cv_tune_key(pr.N, pr.K, pr.M, pr.P, torch.float32, torch.float64, "fp16x3")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert key == f"sm{sms}/prec4/in0/out1/K100/M3/N2^14/rows2^6"
    best, ms = cvx.cv_plan_tune(pr.N, pr.K, pr.M, pr.P, f, X, Y, 15, 1, torch.float32, torch.float64, "fp16x3",
                                cache_path=path)
    assert ms > 0 and best.strategy in (0, 1, 2) and best.ctas >= 0
    cached = cvx.cv_tune_cache_get(path, key)
    assert cached is not None
    assert (cached[0].strategy, cached[0].ctas) == (best.strategy, best.ctas)
    # the second call returns the cached entry, time included, without measuring
    cvx.cv_tune_cache_put(path, key, (best.strategy, best.ctas), 12345.0)
    best2, ms2 = cvx.cv_plan_tune(pr.N, pr.K, pr.M, pr.P, f, X, Y, 15, 1, torch.float32, torch.float64, "fp16x3",
                                  cache_path=path)
    assert (best2.strategy, best2.ctas, ms2) == (best.strategy, best.ctas, 12345.0)
    plan = cvx.cv_plan_ex(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, "fp16x3", best)
    out = cvx.products(X, Y, f, pr.P, 15, 1, "fp16x3", torch.float64, plan=plan, with_stats=True)
    assert cvx.cv_plan_status(plan) == 0
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, 15, 1)
    assert rel_fro_per_fold(out[0].cpu().numpy(), o[0]) <= TOLS["fp16x3"]
    assert rel_fro_per_fold(out[1].cpu().numpy(), o[1]) <= TOLS["fp16x3"]


@pytest.mark.parametrize("prec", ["fp16x3", "fp64"])
def test_explicit_small_fold_strategy_on_larger_folds(prec):
    """Folds of about 300 rows (above the automatic 64-row threshold) through
    the small-fold strategy: each fold spans several staged row blocks of the
    recomputing epilogue."""
    pr = workloads.random_case(602, 6000, 70, 2, 20, dtype=np.float32, scheme="unbalanced", offset=10.0)
    X, Y, f = _inputs(pr)
    for strategy in (cvx.CV_STRATEGY_SMALL_FOLDS, cvx.CV_STRATEGY_FOLD_GROUPED):
        plan = cvx.cv_plan_ex(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, prec, (strategy, 0))
        for flags in (15, 0):
            out = cvx.products(X, Y, f, pr.P, flags, 1, prec, torch.float64, plan=plan, with_stats=True)
            assert cvx.cv_plan_status(plan) == 0
            o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, 1)
            assert rel_fro_per_fold(out[0].cpu().numpy(), o[0]) <= TOLS[prec], (strategy, flags)
            assert rel_fro_per_fold(out[1].cpu().numpy(), o[1]) <= TOLS[prec], (strategy, flags)
