"""The seeded input generators: deterministic, every fold non-empty, the
partitioning schemes as stated, and the batched draw's prefix property that
bench.py --batched-count relies on."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("N,P", [(10, 3), (1000, 7), (64, 64), (100_000, 10)])
def test_schemes(N, P):
    rng = np.random.default_rng(0)
    v = workloads.folds_venetian(N, P)
    assert np.array_equal(v, np.arange(N) % P)
    c = workloads.folds_contiguous(N, P)
    assert np.all(np.diff(c) >= 0) and c[0] == 0 and c[-1] == P - 1
    for f in (v, c, workloads.folds_balanced_random(N, P, rng), workloads.folds_unbalanced_random(N, P, rng)):
        assert f.dtype == np.int32 and f.shape == (N,)
        counts = np.bincount(f, minlength=P)
        assert counts.min() >= 1 and counts.sum() == N and f.max() < P
    b = np.bincount(workloads.folds_balanced_random(N, P, rng), minlength=P)
    # the first N mod P folds hold one extra row
    assert np.all(b[: N % P] == N // P + 1) and np.all(b[N % P:] == N // P)


def test_generators_are_deterministic():
    a, b = workloads.small_case(), workloads.small_case()
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Y, b.Y) and np.array_equal(a.folds, b.folds)
    r1 = workloads.random_case(5, 300, 7, 2, 4, scheme="unbalanced")
    r2 = workloads.random_case(5, 300, 7, 2, 4, scheme="unbalanced")
    assert np.array_equal(r1.X, r2.X) and np.array_equal(r1.folds, r2.folds)


def test_batched_draw_prefix():
    few = workloads.batched_cases(count=5)
    many = workloads.batched_cases(count=12)
    for a, b in zip(few, many):
        assert (a.N, a.K, a.M, a.P, a.flags) == (b.N, b.K, b.M, b.P, b.flags)
        assert np.array_equal(a.X, b.X) and np.array_equal(a.folds, b.folds)
    for pr in many:
        assert 500 <= pr.N <= 20000 and 16 <= pr.K <= 512 and 1 <= pr.M <= 8 and pr.P in (5, 10, 20)
        assert 0 <= pr.flags < 16 and pr.X.dtype == np.float32


def test_bench_shapes():
    pr = workloads.wide_range_case()
    assert (pr.N, pr.K, pr.M, pr.P) == (100_000, 500, 10, 10)
    assert np.array_equal(pr.folds, workloads.folds_contiguous(100_000, 10))
