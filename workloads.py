"""Seeded synthetic inputs for partition-based cross-validation products.

This module only draws random inputs: data matrices X (N x K) and Y (N x M)
and fold assignments. It holds none of the method's arithmetic, so that both
the CUDA path and the CPU oracle can be fed from it without sharing any
computation.

Fold assignments are 0-based int32 arrays (the paper's Definition 1 uses
1-based partition numbers; ``fold = p - 1``). Every generator returns a
partitioning in which each fold is non-empty.

Partitioning schemes (Section 3 and Section 7 of the paper):
  * venetian blinds: row n goes to fold n mod P;
  * contiguous blocks of (nearly) equal size: fold(n) = floor(n * P / N).
    The paper's printed block formula gives blocks of P rows (hence
    ceil(N / P) folds); for "P contiguous folds" this floor(n P / N) reading
    is used instead;
  * balanced random: fold sizes N // P, the first N mod P folds one row
    larger (Section 7 describes the P = 3 case with one fold one sample
    larger), assigned to rows by a seeded permutation.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 2401131850


def folds_venetian(N: int, P: int) -> np.ndarray:
    return (np.arange(N, dtype=np.int64) % P).astype(np.int32)


def folds_contiguous(N: int, P: int) -> np.ndarray:
    n = np.arange(N, dtype=np.int64)
    return ((n * P) // N).astype(np.int32)


def fold_sizes_balanced(N: int, P: int) -> np.ndarray:
    sizes = np.full(P, N // P, dtype=np.int64)
    sizes[: N % P] += 1
    return sizes


def folds_balanced_random(N: int, P: int, rng: np.random.Generator) -> np.ndarray:
    sizes = fold_sizes_balanced(N, P)
    base = np.repeat(np.arange(P, dtype=np.int32), sizes)
    return base[rng.permutation(N)].astype(np.int32)


def folds_unbalanced_random(N: int, P: int, rng: np.random.Generator) -> np.ndarray:
    """Every fold non-empty, sizes drawn from a Dirichlet-like split."""
    assert 1 <= P <= N
    w = rng.exponential(1.0, size=P)
    extra = N - P
    sizes = np.floor(w / w.sum() * extra).astype(np.int64)
    sizes[: extra - sizes.sum()] += 1
    sizes += 1
    base = np.repeat(np.arange(P, dtype=np.int32), sizes)
    return base[rng.permutation(N)].astype(np.int32)


@dataclasses.dataclass
class Problem:
    name: str
    X: np.ndarray          # N x K, row-major
    Y: np.ndarray          # N x M, row-major
    folds: np.ndarray      # int32[N], values in [0, P)
    P: int
    flags: int = 15
    ddof: int = 1

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def K(self) -> int:
        return self.X.shape[1]

    @property
    def M(self) -> int:
        return self.Y.shape[1]


def gaussian_columns(rng, N, mu, sigma, dtype=np.float64):
    """X[:, k] ~ N(mu[k], sigma[k]^2), drawn in float64, then cast."""
    Z = rng.standard_normal((N, len(mu)))
    Z *= np.asarray(sigma)[None, :]
    Z += np.asarray(mu)[None, :]
    return np.ascontiguousarray(Z.astype(dtype, copy=False))


def linear_response(rng, X, M, noise=0.1, b_scale=1.0, dtype=np.float64):
    """Y = X B + noise * eps with B ~ N(0, b_scale^2) of shape K x M."""
    K = X.shape[1]
    B = rng.standard_normal((K, M)) * b_scale
    Y = X.astype(np.float64) @ B + noise * rng.standard_normal((X.shape[0], M))
    return np.ascontiguousarray(Y.astype(dtype, copy=False))


def small_case(seed: int = SEED_BASE + 0, dtype=np.float64, N=1000, K=50, M=2, P=5) -> Problem:
    """N=1000, K=50, M=2, P=5 random balanced folds; mu_k ~ U(-10, 10),
    sigma_k ~ U(0.1, 5); Y = X B + 0.1 eps, B ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-10, 10, K)
    sig = rng.uniform(0.1, 5, K)
    X = gaussian_columns(rng, N, mu, sig, np.float64)
    Y = linear_response(rng, X, M, 0.1, 1.0, np.float64)
    folds = folds_balanced_random(N, P, rng)
    return Problem(f"n{N}_k{K}_m{M}_p{P}_random", X.astype(dtype), Y.astype(dtype), folds, P)


def wide_range_case(seed: int = SEED_BASE + 1, dtype=np.float32, N=100_000, K=500, M=10, P=10) -> Problem:
    """N=1e5, K=500, M=10, P=10 contiguous folds; mu_k ~ U(-100, 100),
    sigma_k log-uniform on [1e-2, 1e2]; Y linear in X plus Gaussian noise.
    The shape is the paper's benchmark shape (Section 7)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-100, 100, K)
    sig = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), K))
    X = gaussian_columns(rng, N, mu, sig, np.float64)
    Y = linear_response(rng, X, M, 0.1, 1.0, np.float64)
    folds = folds_contiguous(N, P)
    return Problem(f"n{N}_k{K}_m{M}_p{P}_contiguous", X.astype(dtype), Y.astype(dtype), folds, P)


def offset_case(seed: int = SEED_BASE + 2, dtype=np.float32, N=1_000_000, K=1024, M=16, P=20) -> Problem:
    """Large offsets to stress cancellation: mu_k = 1e3, sigma_k ~ U(0.5, 2);
    P random balanced folds; Y = X B / sqrt(K) + 0.1 eps."""
    rng = np.random.default_rng(seed)
    mu = np.full(K, 1e3)
    sig = rng.uniform(0.5, 2.0, K)
    X = gaussian_columns(rng, N, mu, sig, np.float32)
    Y = linear_response(rng, X, M, 0.1, 1.0 / np.sqrt(K), np.float32)
    folds = folds_balanced_random(N, P, rng)
    return Problem(f"n{N}_k{K}_m{M}_p{P}_offset", X.astype(dtype), Y.astype(dtype), folds, P)


def many_folds_case(seed: int = SEED_BASE + 3, dtype=np.float32, N=50_000, K=256, M=4, fold_rows=10) -> Problem:
    """N=5e4, K=256, M=4, P=N/10 random balanced folds of 10 rows;
    X ~ N(0, 1) + 50."""
    rng = np.random.default_rng(seed)
    P = N // fold_rows
    X = gaussian_columns(rng, N, np.full(K, 50.0), np.ones(K), np.float32)
    Y = linear_response(rng, X, M, 0.1, 1.0 / np.sqrt(K), np.float32)
    folds = folds_balanced_random(N, P, rng)
    return Problem(f"n{N}_k{K}_m{M}_p{P}_smallfolds", X.astype(dtype), Y.astype(dtype), folds, P, flags=1)


def batched_cases(seed: int = SEED_BASE + 4, count: int = 256, dtype=np.float32,
                  n_range=(500, 20000), k_range=(16, 512), m_range=(1, 8),
                  p_choices=(5, 10, 20)) -> list:
    """Independent CV problems of uneven shape: N ~ U[500, 20000],
    K ~ U[16, 512], M ~ U[1, 8], P in {5, 10, 20}, flags uniform over the 16
    combinations, ddof = 1, mu ~ U(-100, 100), sigma log-uniform [1e-1, 1e1]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        K = int(rng.integers(k_range[0], k_range[1] + 1))
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        P = int(rng.choice(p_choices))
        mu = rng.uniform(-100, 100, K)
        sig = np.exp(rng.uniform(np.log(1e-1), np.log(1e1), K))
        X = gaussian_columns(rng, N, mu, sig, np.float64)
        Y = linear_response(rng, X, M, 0.1, 1.0 / np.sqrt(K), np.float64)
        folds = folds_balanced_random(N, P, rng)
        flags = int(rng.integers(0, 16))
        out.append(Problem(f"batch{b}", X.astype(dtype), Y.astype(dtype), folds, P, flags=flags, ddof=1))
    return out


def random_case(seed: int, N: int, K: int, M: int, P: int, dtype=np.float64,
                scheme: str = "random", offset: float = 0.0, flags: int = 15,
                ddof: int = 1, mu_range: float = 10.0) -> Problem:
    """General small case for parity sweeps."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-mu_range, mu_range, K) + offset
    sig = rng.uniform(0.1, 5, K)
    X = gaussian_columns(rng, N, mu, sig, np.float64)
    Y = linear_response(rng, X, M, 0.1, 1.0 / max(1.0, np.sqrt(K)), np.float64) if M > 0 \
        else np.zeros((N, 0))
    if scheme == "random":
        folds = folds_balanced_random(N, P, rng)
    elif scheme == "contiguous":
        folds = folds_contiguous(N, P)
    elif scheme == "venetian":
        folds = folds_venetian(N, P)
    elif scheme == "unbalanced":
        folds = folds_unbalanced_random(N, P, rng)
    else:
        raise ValueError(scheme)
    return Problem(f"{scheme}_n{N}_k{K}_m{M}_p{P}", X.astype(dtype), Y.astype(dtype),
                   folds, P, flags=flags, ddof=ddof)


def odd_k_case(seed: int = 7, dtype=np.float32, N=400_000, K=1021, M=16, P=20) -> Problem:
    """N=4e5, K=1021 (rows of X not 16-byte aligned), M=16, P=20 random
    balanced folds; the random_case value recipe with a common offset of 10."""
    return random_case(seed, N, K, M, P, dtype=dtype, scheme="random", offset=10.0)


CONFIGS = {
    "small": small_case,
    "wide_range": wide_range_case,
    "offset": offset_case,
    "many_folds": many_folds_case,
    "odd_k": odd_k_case,
}
