"""Parity of the other tensor-core precisions with the CPU oracle:
CV_PREC_BF16X3, CV_PREC_TF32X3 and CV_PREC_TF32 (CV_PREC_FP16X3 is covered by
test_gpu_split.py).

Tolerances, from the arithmetic of each split (the contraction works on the
shifted, power-of-two scaled values v of every column):
  BF16X3  v = hi + lo + d with hi = bf16(v), lo = bf16(v - hi), so
          |d| <= 2^-9 |v - hi| <= 2^-18 |v|; the dropped lo*lo is <= 2^-18 v^2.
          A row's product is off by at most ~3 x 2^-18 = 1.1e-5 of |v_i v_j|,
          and the FP32 accumulator adds at most one rounding (2^-24 of the
          running sum) per MMA step, L / 16 steps for a segment of L rows, so
          with the segments of these tests (L <= 1500) the bound is
          1.1e-5 + 94 x 6e-8 ~ 1.7e-5: tolerance 5e-5.
  TF32X3  v = hi + lo + d with hi = tf32(v), lo = tf32(v - hi) (round to
          nearest), so |d| <= 2^-11 |v - hi| <= 2^-22 |v|; the dropped lo*lo
          is <= 2^-22 v^2: a row's product is off by at most ~3 x 2^-22 =
          7e-7 of |v_i v_j|.  hi*hi accumulates in FP32 as in BF16X3, one
          rounding per MMA step, L / 8 steps of K = 8 for a segment of L rows
          (L <= 1500 here): 7e-7 + 188 x 6e-8 ~ 1.2e-5: tolerance 5e-5.
  TF32    one product of tf32(v) (10 explicit mantissa bits, round to
          nearest): |tf32(v) - v| <= 2^-11 |v|, so a row's product is off by at
          most 2^-10 |v_i v_j| ~ 9.8e-4 and, by Cauchy-Schwarz, an entry by at
          most 9.8e-4 sqrt(O_ii O_jj) plus the same accumulator rounding:
          tolerance 2e-3 for the relative Frobenius and correlation-scale
          errors.
Means and standard deviations come from the ones column and the diagonal of
the same contraction, so they carry the same relative error, measured against
the column's standard deviation.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import corr_scale_error, rel_fro_per_fold, run_library
from test_gpu_fp64 import xty_reference_flags

pytestmark = pytest.mark.gpu
TOLS = {"bf16x3": 5e-5, "tf32x3": 5e-5, "tf32": 2e-3}


def _check(pr, flags, ddof, prec):
    tol = TOLS[prec]
    xtx, xty, mean, std = run_library(pr, flags, ddof, prec)
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
    oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), ddof)[1] if pr.M else None
    e1 = rel_fro_per_fold(xtx, o[0])
    e2 = rel_fro_per_fold(xty, oy) if pr.M else 0.0
    e3 = corr_scale_error(xtx, o[0])
    assert e1 <= tol and e2 <= tol and e3 <= tol, (prec, pr.name, flags, ddof, e1, e2, e3)
    # statistics, on the scale of each column's standard deviation
    o_std = np.maximum(o[3], 1e-300)
    assert np.max(np.abs(mean - o[2]) / o_std) <= tol, (prec, "mean")
    assert np.max(np.abs(std - o[3]) / o_std) <= tol, (prec, "std")
    assert np.array_equal(xtx, np.transpose(xtx, (0, 2, 1)))
    return e1, e2, e3


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
@pytest.mark.parametrize("ddof", [0, 1])
def test_small_config_all_flags(prec, ddof):
    pr = workloads.small_case(dtype=np.float32)
    for flags in range(16):
        _check(pr, flags, ddof, prec)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
@pytest.mark.parametrize("N,K,M,P,scheme", [
    (700, 9, 3, 2, "random"),
    (2000, 30, 4, 9, "unbalanced"),
    (1300, 127, 1, 5, "contiguous"),    # D = 129: a second column block
    (3001, 128, 3, 7, "venetian"),
    (6000, 260, 9, 13, "unbalanced"),   # three tile rows, ragged segments
])
def test_shapes_and_partitionings(prec, N, K, M, P, scheme):
    pr = workloads.random_case(101 + K, N, K, M, P, dtype=np.float32, scheme=scheme)
    for flags in (0, 5, 10, 15):
        _check(pr, flags, 1, prec)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
@pytest.mark.parametrize("in_dtype", [np.float32, np.float64])
def test_large_offsets(prec, in_dtype):
    """Columns with mean 1e3 and standard deviation about 1: the per-column
    shift keeps the cancellation in X^T X - N mu mu^T out of the contraction."""
    pr = workloads.offset_case(N=20000, K=64, M=4, P=5, dtype=in_dtype)
    for flags in (0, 1, 5, 15):
        _check(pr, flags, 1, prec)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
def test_ragged_load_path(prec):
    """Unaligned leading dimension: the register-gather conversion instead of
    the tensor-memory-accelerator one, same operand image."""
    pr = workloads.random_case(23, 2500, 130, 3, 6, dtype=np.float32, scheme="random")
    dev = torch.device("cuda:0")
    big = torch.zeros((pr.N, pr.K + 3), dtype=torch.float32, device=dev)
    big[:, :pr.K].copy_(torch.from_numpy(pr.X))
    import paper_2401_13185_gb300 as cvx
    Xv = big[:, :pr.K]
    Yd = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, prec)
    xtx, xty = cvx.products(Xv, Yd, f, pr.P, 15, 1, plan=plan)
    assert cvx.cv_plan_status(plan) == 0
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, 15, 1)
    assert rel_fro_per_fold(xtx.cpu().numpy(), o[0]) <= TOLS[prec]
    assert rel_fro_per_fold(xty.cpu().numpy(), o[1]) <= TOLS[prec]
