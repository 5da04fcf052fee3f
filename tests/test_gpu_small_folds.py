"""Parity of the small-fold strategy (folds averaging at most 64 rows: each
fold's part of H recomputed from its rows in the epilogue) with the oracle,
on both precisions.  Tolerances are those of the fold-grouped strategy: 1e-12
relative Frobenius for FP64, 2e-6 for the split FP16 path."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import corr_scale_error, rel_fro_per_fold, run_library
from test_gpu_fp64 import xty_reference_flags

pytestmark = pytest.mark.gpu
TOLS = {"fp64": 1e-12, "fp16x3": 2e-6}


def _compare(pr, flags, ddof, prec, out_dtype=torch.float64, which=None):
    xtx, xty, mean, std = run_library(pr, flags, ddof, prec, out_dtype)
    if which is None:
        o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
        oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), ddof)[1] if pr.M else None
        sel = np.arange(pr.P)
    else:
        o = oracle.naive_subset(pr.X, pr.Y, pr.folds, pr.P, flags, ddof, which)
        oy = oracle.naive_subset(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), ddof, which)[1] \
            if pr.M else None
        sel = np.asarray(which)
    tol = TOLS[prec] if out_dtype == torch.float64 else max(TOLS[prec], 2e-7)
    e1 = rel_fro_per_fold(xtx[sel], o[0][sel])
    e2 = rel_fro_per_fold(xty[sel], oy[sel]) if pr.M else 0.0
    e3 = corr_scale_error(xtx[sel], o[0][sel])
    assert e1 <= tol and e2 <= tol and e3 <= tol, (pr.name, prec, flags, ddof, e1, e2, e3)
    np.testing.assert_allclose(mean[sel], o[2][sel], rtol=1e-7, atol=1e-7 * np.abs(o[2]).max())
    np.testing.assert_allclose(std[sel], o[3][sel], rtol=1e-6)
    assert np.array_equal(xtx, np.transpose(xtx, (0, 2, 1)))


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_small_folds_all_flags(prec):
    """2000 rows in 200 random folds of 10 rows, every flag combination."""
    pr = workloads.random_case(41, 2000, 40, 3, 200, dtype=np.float32, scheme="random")
    for flags in range(16):
        _compare(pr, flags, 1, prec)
    for flags in (0, 5, 15):
        _compare(pr, flags, 0, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
@pytest.mark.parametrize("N,K,M,P,scheme", [
    (300, 20, 2, 300, "venetian"),      # leave-one-out
    (3000, 70, 5, 100, "unbalanced"),   # some folds longer than one staging pass
    (2600, 150, 4, 130, "random"),      # two tile rows, ragged
    (1000, 127, 0, 50, "contiguous"),   # M = 0, D = 128
    (1500, 128, 1, 500, "random"),      # D = 130, three rows per fold
])
def test_small_folds_shapes(prec, N, K, M, P, scheme):
    pr = workloads.random_case(300 + K, N, K, M, P, dtype=np.float32, scheme=scheme)
    for flags in (0, 1, 5, 10, 15):
        _compare(pr, flags, 1, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_small_folds_dtypes_and_offsets(prec):
    """FP64 storage with a large common offset, and FP32 outputs."""
    pr = workloads.random_case(57, 1800, 33, 2, 90, dtype=np.float64, scheme="random", offset=1e3)
    for flags in (0, 5, 15):
        _compare(pr, flags, 1, prec)
    pr32 = workloads.random_case(58, 1800, 33, 2, 90, dtype=np.float32, scheme="unbalanced")
    _compare(pr32, 15, 1, prec, out_dtype=torch.float32)


def test_small_fold_plan_layout():
    """The strategy is picked by fold size: its plan holds no per-fold tiles."""
    dev = torch.device("cuda:0")
    for P, small in ((200, True), (20, False)):
        pr = workloads.random_case(5, 4000, 64, 2, P, dtype=np.float32)
        f = torch.from_numpy(pr.folds).to(dev)
        plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, "fp16x3")
        ws = cvx.cv_plan_workspace_bytes(plan)
        per_fold_tiles = P * 16384 * 12   # int64 + float per element of one tile, every fold
        assert (ws < per_fold_tiles) == small, (P, ws)


@pytest.mark.parametrize("prec", ["fp16x3", "fp64"])
def test_many_folds_full_size_sampled(prec):
    """N=5e4, K=256, M=4, P=5000 random folds of 10 rows, X ~ N(0,1) + 50:
    whole folds checked against the naive oracle on a sample of folds."""
    pr = workloads.many_folds_case()
    which = [0, 1234, 4999]
    for flags in (1, 5):
        _compare(pr, flags, 1, prec, which=which)
