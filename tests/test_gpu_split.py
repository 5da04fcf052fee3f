"""Parity of the tcgen05 split-FP16 path (CV_PREC_FP16X3) with the CPU oracle.

Tolerance: relative Frobenius error <= 2e-6 per fold and per product, and the
same bound on the correlation-scale error of X^T X.  Derivation: each operand
is carried as FP16 hi + lo, about 22 significant bits (relative representation
error <= 2^-22 ~ 2.4e-7 per element, so <= ~5e-7 per product); the FP32
tensor-memory accumulator adds one rounding (2^-24 relative to the running
sum) per K=16 MMA step over a segment of at most a few thousand rows; the
segment partials and everything after them are FP64.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import corr_scale_error, rel_fro_per_fold, run_library
from test_gpu_fp64 import xty_reference_flags

pytestmark = pytest.mark.gpu
TOL = 2e-6


def _check(pr, flags, ddof, out_dtype=torch.float64, tol=TOL):
    xtx, xty, mean, std = run_library(pr, flags, ddof, "fp16x3", out_dtype)
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
    oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), ddof)[1] if pr.M else None
    e1 = rel_fro_per_fold(xtx, o[0])
    e2 = rel_fro_per_fold(xty, oy) if pr.M else 0.0
    e3 = corr_scale_error(xtx, o[0])
    assert e1 <= tol and e2 <= tol and e3 <= tol, (pr.name, flags, ddof, e1, e2, e3)
    np.testing.assert_allclose(mean, o[2], rtol=1e-7, atol=1e-7 * np.abs(o[2]).max())
    np.testing.assert_allclose(std, o[3], rtol=1e-6)
    assert np.array_equal(xtx, np.transpose(xtx, (0, 2, 1)))
    return e1, e2, e3


@pytest.mark.parametrize("ddof", [0, 1])
def test_small_config_all_flags(ddof):
    pr = workloads.small_case(dtype=np.float32)
    for flags in range(16):
        _check(pr, flags, ddof)


@pytest.mark.parametrize("N,K,M,P,scheme", [
    (700, 9, 3, 2, "random"),
    (150, 7, 2, 150, "venetian"),       # leave-one-out
    (2000, 30, 4, 9, "unbalanced"),
    (1500, 127, 0, 4, "random"),        # M = 0, D = 128
    (1300, 127, 1, 5, "contiguous"),    # D = 129
    (3001, 128, 3, 7, "venetian"),
    (900, 1, 0, 3, "random"),
    (6000, 260, 9, 13, "unbalanced"),   # three tile rows, ragged segments
    (4000, 200, 5, 6, "random"),        # last block of 78 used columns: 80 computed
])
def test_shapes_and_partitionings(N, K, M, P, scheme):
    pr = workloads.random_case(101 + K, N, K, M, P, dtype=np.float32, scheme=scheme)
    for flags in (0, 1, 4, 5, 10, 15):
        _check(pr, flags, 1)


@pytest.mark.parametrize("in_dtype", [np.float32, np.float64])
def test_large_offsets(in_dtype):
    pr = workloads.offset_case(N=20000, K=64, M=4, P=5, dtype=in_dtype)
    for flags in (0, 1, 5, 15):
        _check(pr, flags, 1)


def test_constant_columns():
    pr = workloads.random_case(9, 600, 6, 2, 4, dtype=np.float32)
    pr.X = pr.X.copy()
    pr.X[:, 1] = 7.0
    pr.Y = pr.Y.copy()
    pr.Y[:, 0] = -2.5
    for flags in range(16):
        _check(pr, flags, 1)


def test_float32_output():
    pr = workloads.random_case(5, 1200, 40, 3, 6, dtype=np.float32, offset=30.0)
    for flags in (0, 5, 15):
        _check(pr, flags, 1, out_dtype=torch.float32, tol=TOL)


def test_deterministic():
    pr = workloads.random_case(17, 4000, 70, 5, 6, dtype=np.float32)
    a = run_library(pr, 15, 1, "fp16x3")
    b = run_library(pr, 15, 1, "fp16x3")
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_out_of_range_operand_is_reported():
    """A value far outside the sampled range overflows FP16 after scaling; the
    plan reports CV_ERR_RANGE instead of returning silently wrong numbers."""
    pr = workloads.random_case(4, 8192, 8, 1, 4, dtype=np.float32)
    X = pr.X.copy()
    X[4097, 3] = 1e9          # not in the strided shift sample (rows k * N / 4096)
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, "fp16x3")
    cvx.products(Xd, Yd, f, pr.P, 15, 1, plan=plan)
    assert cvx.cv_status_string(cvx.cv_plan_status(plan)) == "CV_ERR_RANGE"
    # cleared after reading; a clean call reports CV_OK
    Xd.copy_(torch.from_numpy(pr.X))
    cvx.products(Xd, Yd, f, pr.P, 15, 1, plan=plan)
    assert cvx.cv_plan_status(plan) == 0


def test_wide_range_full_size_sampled():
    """N=1e5, K=500, M=10, P=10 contiguous folds, FP32 storage, all flags
    centered and scaled: sampled entries against the oracle."""
    pr = workloads.wide_range_case()
    flags, ddof = 15, 1
    xtx, xty, mean, std = run_library(pr, flags, ddof, "fp16x3")
    rng = np.random.default_rng(1)
    samples = [(int(rng.integers(pr.P)), 0, int(rng.integers(pr.K)), int(rng.integers(pr.K)))
               for _ in range(60)]
    samples += [(int(rng.integers(pr.P)), 1, int(rng.integers(pr.K)), int(rng.integers(pr.M)))
                for _ in range(40)]
    ref = oracle.naive_entries(pr.X, pr.Y, pr.folds, pr.P, flags, ddof, samples)
    counts = np.bincount(pr.folds, minlength=pr.P)
    for (p, w, i, j), r in zip(samples, ref):
        got = (xtx if w == 0 else xty)[p, i, j]
        scale = pr.N - counts[p] - ddof
        assert abs(got - r) <= TOL * scale, (p, w, i, j, got, r)
    for p in range(pr.P):
        np.testing.assert_allclose(np.diag(xtx[p]), pr.N - counts[p] - ddof, rtol=TOL)


@pytest.mark.parametrize("case", ["ld_pad_aligned", "ld_pad_unaligned", "x_misaligned", "m31", "m32"])
def test_layouts_and_load_paths(case):
    """Padded and unaligned leading dimensions, a base address off the 16-byte
    boundary, and the widest Y the TMA-fed path takes (M = 31) next to the first
    that falls back to the register-gather path (M = 32)."""
    M = 31 if case == "m31" else (32 if case == "m32" else 3)
    pr = workloads.random_case(23, 2500, 132, M, 6, dtype=np.float32, scheme="random")
    dev = torch.device("cuda:0")
    pad = {"ld_pad_aligned": 4, "ld_pad_unaligned": 3}.get(case, 0)
    big = torch.zeros((pr.N, pr.K + pad + 1), dtype=torch.float32, device=dev)
    off = 1 if case == "x_misaligned" else 0
    Xv = big[:, off:off + pr.K]
    Xv.copy_(torch.from_numpy(pr.X))
    if pad:
        Xv = big[:, :pr.K]
    Yd = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    for flags in (0, 5, 15):
        plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, "fp16x3")
        xtx, xty = cvx.products(Xv, Yd, f, pr.P, flags, 1, plan=plan)
        assert cvx.cv_plan_status(plan) == 0
        o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, 1)
        oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), 1)[1]
        assert rel_fro_per_fold(xtx.cpu().numpy(), o[0]) <= TOL
        assert rel_fro_per_fold(xty.cpu().numpy(), oy) <= TOL


def test_launch_count_and_phase_profile():
    """cv_plan_launches counts the kernels each cv_products call enqueues, and
    the phase profile reports all six phases (operand conversion only on the
    split path)."""
    pr = workloads.random_case(7, 4096, 96, 4, 6, dtype=np.float32, scheme="contiguous")
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    folds = torch.from_numpy(pr.folds).to(dev)
    XTX = torch.empty((pr.P, pr.K, pr.K), dtype=torch.float64, device=dev)
    XTY = torch.empty((pr.P, pr.K, pr.M), dtype=torch.float64, device=dev)
    # split, 6 folds: shift estimate with Y packing (1), TMA-fed conversion (1),
    # Gram (1), statistics from the segment partials (1), fold sums with the
    # epilogue (1); FP64: shift (1), Gram (1), fold sums and total (2), stats
    # (1), epilogue (1)
    for prec, per_call in (("fp16x3", 5), ("fp64", 6)):
        plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, folds, X.dtype, torch.float64, prec)
        assert cvx.cv_plan_launches(plan) == 0
        cvx.cv_plan_profile(plan, True)
        for _ in range(3):
            cvx.cv_products(plan, X, Y, 15, 1, XTX, XTY)
        assert cvx.cv_plan_launches(plan) == 3 * per_call
        ms, calls = cvx.cv_plan_phase_ms(plan)
        assert calls == 3 and tuple(ms) == cvx.PHASES
        assert all(v >= 0.0 for v in ms.values())
        assert ms["gram"] > 0.0 and ms["epilogue"] > 0.0
        if prec == "fp64":
            assert ms["convert"] < 0.01
        cvx.cv_plan_profile(plan, False)
        assert cvx.cv_plan_status(plan) == 0
