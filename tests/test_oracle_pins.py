"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself.  The pins are:
  * a hand-worked example (tests/golden/hand_n6_k2_m1_p2.json);
  * brute force in exact rational / 50-digit decimal arithmetic on tiny
    integer data (Definitions 2-5, Algorithm 6);
  * special cases that reduce to numpy's covariance, correlation, standard
    deviation and plain matrix product;
  * invariants (symmetry, positive semi-definiteness, the diagonal of a
    correlation, Lemma 2 summed over folds, shift / scale / permutation
    invariance);
  * Table 1's coincidences among the 16 flag combinations;
  * the leakage counterexample after Lemma 11;
  * agreement of the two independent CPU algorithms (Proposition 17).
"""
import itertools
import json
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
CX, SX, CY, SY = 1, 2, 4, 8
ALL_FLAGS = list(range(16))


def _eval(expr):
    return float(eval(expr, {"sqrt": math.sqrt, "__builtins__": {}}))


# ---------------------------------------------------------------------------
# Hand-worked example
# ---------------------------------------------------------------------------
def test_hand_example():
    g = json.load(open(os.path.join(HERE, "golden", "hand_n6_k2_m1_p2.json")))
    X = np.array(g["X"], float)
    Y = np.array(g["Y"], float)
    folds = np.array(g["folds"], np.int32)
    P = g["P"]
    for impl in (oracle.naive, oracle.fast):
        for case in g["cases"]:
            xtx, xty, mean, std = impl(X, Y, folds, P, case["flags"], case["ddof"])
            p = case["fold"]
            exp_xtx = np.array([_eval(e) for e in case["XTX"]]).reshape(2, 2)
            exp_xty = np.array([_eval(e) for e in case["XTY"]]).reshape(2, 1)
            np.testing.assert_allclose(xtx[p], exp_xtx, rtol=1e-14, atol=1e-13, err_msg=str(case))
            np.testing.assert_allclose(xty[p], exp_xty, rtol=1e-14, atol=1e-13, err_msg=str(case))
        xtx, xty, mean, std = impl(X, Y, folds, P, 15, 1)
        for p in range(2):
            np.testing.assert_allclose(mean[p], [_eval(e) for e in g["means"][f"fold{p}"]], rtol=1e-15)
            np.testing.assert_allclose(std[p], [_eval(e) for e in g["std_ddof1"][f"fold{p}"]], rtol=1e-15)


# ---------------------------------------------------------------------------
# Exact brute force (Definitions 2-5, Algorithm 6)
# ---------------------------------------------------------------------------
getcontext().prec = 50


def _exact_products(X, Y, folds, P, flags, ddof):
    """Training-partition products in exact arithmetic: Fractions for the
    means and centered values, 50-digit Decimals once a square root enters."""
    N, K = X.shape
    M = Y.shape[1]
    Z = [[Fraction(int(v)) for v in list(X[n]) + list(Y[n])] for n in range(N)]
    out_xtx = np.zeros((P, K, K))
    out_xty = np.zeros((P, K, M))
    for p in range(P):
        T = [n for n in range(N) if folds[n] != p]
        nt = len(T)
        cols = []
        for j in range(K + M):
            c = (flags & CX) if j < K else (flags & CY)
            s = (flags & SX) if j < K else (flags & SY)
            vals = [Z[n][j] for n in T]
            mean = sum(vals, Fraction(0)) / nt
            var = sum(((v - mean) ** 2 for v in vals), Fraction(0)) / (nt - ddof)
            sd = Decimal(var.numerator) / Decimal(var.denominator)
            sd = sd.sqrt() if var != 0 else Decimal(1)
            col = [(v - mean) if c else v for v in vals]
            if s:
                col = [Decimal(v.numerator) / Decimal(v.denominator) / sd for v in col]
            else:
                col = [Decimal(v.numerator) / Decimal(v.denominator) for v in col]
            cols.append(col)
        for i in range(K):
            for j in range(K):
                out_xtx[p, i, j] = float(sum((a * b for a, b in zip(cols[i], cols[j])), Decimal(0)))
            for m in range(M):
                out_xty[p, i, m] = float(sum((a * b for a, b in zip(cols[i], cols[K + m])), Decimal(0)))
    return out_xtx, out_xty


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_exact(seed):
    rng = np.random.default_rng(1000 + seed)
    N = int(rng.integers(6, 13))
    K = int(rng.integers(1, 5))
    M = int(rng.integers(0, 3))
    P = int(rng.integers(2, min(N // 2, 5) + 1))
    folds = workloads.folds_unbalanced_random(N, P, rng)
    X = rng.integers(-9, 10, size=(N, K)).astype(float)
    Y = rng.integers(-9, 10, size=(N, M)).astype(float)
    if seed == 0:
        X[:, 0] = 4.0       # a constant column: sigma = 0 is replaced by 1
    for flags in ALL_FLAGS:
        for ddof in (0, 1):
            ex, ey = _exact_products(X, Y, folds, P, flags, ddof)
            # Algorithm 7 in floating point leaves a rounding residue in
            # Lemma 12's radicand for a constant column, so its exact-zero test
            # (step 24) does not fire; the constant-column case pins only the
            # two-pass definition.
            impls = (oracle.naive,) if seed == 0 else (oracle.naive, oracle.fast)
            for impl in impls:
                xtx, xty, _, _ = impl(X, Y, folds, P, flags, ddof)
                scale = max(1.0, np.abs(ex).max())
                np.testing.assert_allclose(xtx, ex, rtol=1e-13, atol=1e-12 * scale,
                                           err_msg=f"{impl.__name__} flags={flags} ddof={ddof}")
                if M:
                    scale = max(1.0, np.abs(ey).max())
                    np.testing.assert_allclose(xty, ey, rtol=1e-13, atol=1e-12 * scale,
                                               err_msg=f"{impl.__name__} flags={flags} ddof={ddof}")


# ---------------------------------------------------------------------------
# Special cases that reduce to library routines
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ddof", [0, 1])
def test_library_special_cases(ddof):
    pr = workloads.random_case(7, N=300, K=6, M=3, P=4, scheme="unbalanced")
    X, Y, folds, P = pr.X, pr.Y, pr.folds, pr.P
    res = {f: oracle.naive(X, Y, folds, P, f, ddof) for f in (0, CX | CY, CX | SX | CY | SY)}
    for p in range(P):
        T = folds != p
        XT, YT = X[T], Y[T]
        nt = XT.shape[0]
        np.testing.assert_allclose(res[0][0][p], XT.T @ XT, rtol=1e-13)
        np.testing.assert_allclose(res[0][1][p], XT.T @ YT, rtol=1e-13)
        cov = np.cov(np.hstack([XT, YT]), rowvar=False, ddof=ddof) * (nt - ddof)
        np.testing.assert_allclose(res[CX | CY][0][p], cov[:6, :6], rtol=1e-11, atol=1e-9)
        np.testing.assert_allclose(res[CX | CY][1][p], cov[:6, 6:], rtol=1e-11, atol=1e-9)
        corr = np.corrcoef(np.hstack([XT, YT]), rowvar=False) * (nt - ddof)
        np.testing.assert_allclose(res[15][0][p], corr[:6, :6], rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(res[15][1][p], corr[:6, 6:], rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(res[15][2][p], np.hstack([XT, YT]).mean(0), rtol=1e-13)
        np.testing.assert_allclose(res[15][3][p], np.hstack([XT, YT]).std(0, ddof=ddof), rtol=1e-12)


# ---------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------
def test_invariants():
    pr = workloads.random_case(11, N=240, K=7, M=2, P=5, scheme="random")
    X, Y, folds, P = pr.X, pr.Y, pr.folds, pr.P
    N = X.shape[0]
    counts = np.bincount(folds, minlength=P)
    for flags in ALL_FLAGS:
        xtx, xty, _, _ = oracle.naive(X, Y, folds, P, flags, 1)
        assert np.array_equal(xtx, np.transpose(xtx, (0, 2, 1))), "X^T X must be symmetric"
        if flags & CX:
            for p in range(P):
                w = np.linalg.eigvalsh(xtx[p])
                assert w.min() >= -1e-12 * np.abs(w).max()
        if (flags & CX) and (flags & SX):
            for p in range(P):
                np.testing.assert_allclose(np.diag(xtx[p]), N - counts[p] - 1, rtol=1e-13)
    # Lemma 2 summed over folds: sum_p X_Tp^T X_Tp = (P - 1) X^T X.
    xtx, xty, _, _ = oracle.naive(X, Y, folds, P, 0, 1)
    np.testing.assert_allclose(xtx.sum(0), (P - 1) * (X.T @ X), rtol=1e-12)
    np.testing.assert_allclose(xty.sum(0), (P - 1) * (X.T @ Y), rtol=1e-12)
    # Adding a constant to a column leaves every centered result unchanged.
    Xs = X + np.arange(1, 8)[None, :] * 3.0
    Ys = Y - 5.0
    for flags in (CX | CY, 15, CX | SX, CX):
        a = oracle.naive(X, Y, folds, P, flags, 1)
        b = oracle.naive(Xs, Ys, folds, P, flags, 1)
        np.testing.assert_allclose(b[0], a[0], rtol=1e-10, atol=1e-9 * np.abs(a[0]).max())
        np.testing.assert_allclose(b[1], a[1], rtol=1e-10, atol=1e-9 * np.abs(a[1]).max())
    # Multiplying a column by c > 0 leaves every result scaled on that side unchanged.
    c = np.linspace(0.5, 4.0, 7)
    a = oracle.naive(X, Y, folds, P, SX | SY, 1)
    b = oracle.naive(X * c[None, :], Y * 2.5, folds, P, SX | SY, 1)
    np.testing.assert_allclose(b[0], a[0], rtol=1e-12)
    np.testing.assert_allclose(b[1], a[1], rtol=1e-12)
    # Column permutation permutes the outputs; fold relabelling permutes folds;
    # row permutation changes nothing.
    perm = np.random.default_rng(0).permutation(7)
    b = oracle.naive(X[:, perm], Y, folds, P, 15, 1)
    np.testing.assert_allclose(b[0], a_full := oracle.naive(X, Y, folds, P, 15, 1)[0][:, perm][:, :, perm], rtol=1e-12)
    relabel = np.random.default_rng(1).permutation(P)
    b = oracle.naive(X, Y, relabel[folds].astype(np.int32), P, 15, 1)
    np.testing.assert_allclose(b[0][relabel], oracle.naive(X, Y, folds, P, 15, 1)[0], rtol=1e-12)
    rp = np.random.default_rng(2).permutation(N)
    b = oracle.naive(X[rp], Y[rp], folds[rp], P, 15, 1)
    a = oracle.naive(X, Y, folds, P, 15, 1)
    np.testing.assert_allclose(b[0], a[0], rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(b[1], a[1], rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------------------
# Table 1 coincidences and the 12 distinct combinations (Section 6)
# ---------------------------------------------------------------------------
def test_table1_coincidences():
    pr = workloads.random_case(3, N=200, K=5, M=3, P=4, scheme="random")
    X, Y, folds, P = pr.X, pr.Y, pr.folds, pr.P
    res = {f: oracle.naive(X, Y, folds, P, f, 1) for f in ALL_FLAGS}
    for f in ALL_FLAGS:
        if f & CX:
            # with X centered, centering Y as well changes nothing (Lemma 9)
            g = f ^ CY
            np.testing.assert_allclose(res[f][0], res[g][0], rtol=1e-12, atol=1e-10)
            np.testing.assert_allclose(res[f][1], res[g][1], rtol=1e-12, atol=1e-10)
    for s in (0, SX, SY, SX | SY):
        # centering only Y gives the same X^T Y as centering only X
        np.testing.assert_allclose(res[CY | s][1], res[CX | s][1], rtol=1e-12, atol=1e-10)
        # ... but not the same X^T X
        assert not np.allclose(res[CY | s][0], res[CX | s][0], rtol=1e-6)
    # Count distinct (XTX, XTY) pairs among the 16 combinations.
    reps = []
    for f in ALL_FLAGS:
        pair = np.concatenate([res[f][0].ravel(), res[f][1].ravel()])
        if not any(np.allclose(pair, r, rtol=1e-9, atol=1e-9) for r in reps):
            reps.append(pair)
    assert len(reps) == 12
    # X^T Y alone: 8 distinct products.
    reps = []
    for f in ALL_FLAGS:
        if not any(np.allclose(res[f][1], r, rtol=1e-9, atol=1e-9) for r in reps):
            reps.append(res[f][1])
    assert len(reps) == 8


# ---------------------------------------------------------------------------
# Leakage counterexample (Lemma 11 and the argument after it)
# ---------------------------------------------------------------------------
def _lindgren_centered(X, folds, P, p):
    """Lemma 11: (X_T^T X_T) - N xbar xbar^T (2 - 1/P) + |T| xbar xbar_T^T + |T| xbar_T xbar^T."""
    N = X.shape[0]
    T = folds != p
    XT = X[T]
    xbar = X.mean(0)
    xbt = XT.mean(0)
    nt = XT.shape[0]
    return (XT.T @ XT - N * np.outer(xbar, xbar) * (2 - 1 / P)
            + nt * np.outer(xbar, xbt) + nt * np.outer(xbt, xbar))


def test_leakage_counterexample():
    # Training partition of fold 0 is centered, the full data set is not.
    X = np.array([[4.0, 2.0], [6.0, 3.0], [-1.0, 5.0], [1.0, -5.0]])
    Y = np.zeros((4, 0))
    folds = np.array([0, 0, 1, 1], np.int32)
    xtx = oracle.naive(X, Y, folds, 2, CX, 1)[0]
    XT = X[2:]
    np.testing.assert_allclose(xtx[0], XT.T @ XT)   # already centered
    lind = _lindgren_centered(X, folds, 2, 0)
    assert np.abs(lind - xtx[0]).max() > 1.0
    # Standardising with full-data statistics also differs (leakage).
    Xg = (X - X.mean(0)) / X.std(0, ddof=1)
    glob = Xg[2:].T @ Xg[2:]
    xtx_cs = oracle.naive(X, Y, folds, 2, CX | SX, 1)[0]
    assert np.abs(glob - xtx_cs[0]).max() > 0.1
    # On random data with a non-zero mean the same holds for every fold.
    pr = workloads.random_case(5, N=100, K=4, M=0, P=5, offset=20.0)
    xtx = oracle.naive(pr.X, pr.Y, pr.folds, 5, CX, 1)[0]
    for p in range(5):
        lind = _lindgren_centered(pr.X, pr.folds, 5, p)
        assert np.abs(lind - xtx[p]).max() > 1e-3 * np.abs(xtx[p]).max()


# ---------------------------------------------------------------------------
# Two independent CPU algorithms agree (Proposition 17)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,ddof", [("random", 1), ("contiguous", 0), ("venetian", 1), ("unbalanced", 1)])
def test_fast_matches_naive(scheme, ddof):
    pr = workloads.random_case(21, N=400, K=12, M=3, P=7, scheme=scheme)
    for flags in ALL_FLAGS:
        a = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
        b = oracle.fast(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
        for u, v in zip(a, b):
            err = np.linalg.norm((u - v).ravel()) / np.linalg.norm(u.ravel())
            assert err < 1e-12, (flags, err)


def test_small_config_fast_matches_naive():
    pr = workloads.small_case()
    for flags in ALL_FLAGS:
        a = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, 1)
        b = oracle.fast(pr.X, pr.Y, pr.folds, pr.P, flags, 1)
        for u, v in zip(a[:2], b[:2]):
            for p in range(pr.P):
                err = np.linalg.norm(u[p] - v[p]) / np.linalg.norm(u[p])
                assert err < 1e-12, (flags, p, err)


def test_naive_entry_is_bitwise_entry_of_naive():
    pr = workloads.random_case(8, N=150, K=6, M=2, P=3)
    rng = np.random.default_rng(0)
    for flags in (0, 5, 10, 15):
        xtx, xty, _, _ = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, 1)
        samples = [(int(rng.integers(3)), 0, int(rng.integers(6)), int(rng.integers(6))) for _ in range(10)]
        samples += [(int(rng.integers(3)), 1, int(rng.integers(6)), int(rng.integers(2))) for _ in range(10)]
        vals = oracle.naive_entries(pr.X, pr.Y, pr.folds, pr.P, flags, 1, samples)
        for (p, w, i, j), v in zip(samples, vals):
            assert v == (xtx if w == 0 else xty)[p, i, j]


@pytest.mark.parametrize("which", [[3], [0], [4, 1], [2, 0, 3], [1, 2, 3, 4, 0], [3, 3]])
def test_naive_subset_is_naive_on_listed_folds(which):
    """The fold-subset entry point is the full algorithm restricted to the
    listed folds: bitwise the same rows of every output for each listed fold,
    whatever the list's order (unsorted, single, repeated), and every other
    fold left at its initial zeros."""
    pr = workloads.random_case(21, N=130, K=5, M=2, P=5, scheme="unbalanced")
    for flags, ddof in ((15, 1), (0, 0), (5, 1), (10, 0)):
        full = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
        sub = oracle.naive_subset(pr.X, pr.Y, pr.folds, pr.P, flags, ddof, which)
        for a, b in zip(sub, full):
            for p in range(pr.P):
                if p in which:
                    assert np.array_equal(a[p], b[p]), (which, flags, p)
                else:
                    assert not a[p].any(), (which, flags, p)
    with pytest.raises(oracle.OracleError) as e:
        oracle.naive_subset(pr.X, pr.Y, pr.folds, pr.P, 15, 1, [5])
    assert e.value.code == 1


def test_threads_do_not_change_any_bit():
    """Host threads only split the oracle's columns and output rows; every
    value is formed by one thread in the same order."""
    pr = workloads.random_case(22, N=400, K=37, M=3, P=4, scheme="random")
    prev = oracle.get_threads()
    try:
        oracle.set_threads(1)
        one = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, 15, 1)
        for t in (2, 3, 8):
            oracle.set_threads(t)
            many = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, 15, 1)
            assert all(np.array_equal(a, b) for a, b in zip(one, many)), t
        assert oracle.set_threads(0) >= 1
    finally:
        oracle.set_threads(prev)


# ---------------------------------------------------------------------------
# Algorithm 1 and argument checks
# ---------------------------------------------------------------------------
def test_validation_partitions():
    rng = np.random.default_rng(4)
    folds = workloads.folds_unbalanced_random(50, 6, rng)
    off, rows = oracle.validation_partitions(folds, 6)
    for p in range(6):
        assert list(rows[off[p]:off[p + 1]]) == [n for n in range(50) if folds[n] == p]
    with pytest.raises(oracle.OracleError) as e:
        oracle.validation_partitions(np.array([0, 1, 3], np.int32), 3)
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.validation_partitions(np.array([0, 2, 2], np.int32), 3)
    assert e.value.code == 3


def test_not_scalable():
    X = np.arange(6.0).reshape(3, 2)
    Y = np.ones((3, 1))
    folds = np.array([0, 0, 1], np.int32)       # fold 0 trains on one row
    for impl in (oracle.naive, oracle.fast):
        with pytest.raises(oracle.OracleError) as e:
            impl(X, Y, folds, 2, SX, 1)
        assert e.value.code == 4
        impl(X, Y, folds, 2, SX, 0)                 # ddof = 0 only needs |T| >= 1
        impl(X, Y, folds, 2, CX | CY, 1)            # centering alone is fine


def test_partitioning_generators():
    assert list(workloads.folds_contiguous(10, 3)) == [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    assert list(workloads.folds_venetian(7, 3)) == [0, 1, 2, 0, 1, 2, 0]
    f = workloads.folds_balanced_random(100, 3, np.random.default_rng(0))
    assert sorted(np.bincount(f)) == [33, 33, 34]
