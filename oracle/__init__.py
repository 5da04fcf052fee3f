"""CPU oracle for partition-based cross-validation products (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python
binding never import it.

The arithmetic lives in ``cv_oracle.c`` (plain C, float64, no fused
multiply-add), written from Engstrom & Jensen (arXiv 2401.13185):

  validation_partitions  Algorithm 1
  naive                  Algorithms 2 / 4 / 6 generalised to the 16
                         centering/scaling flag combinations (Table 1)
  naive_subset           ``naive`` for a list of folds
  set_threads            host threads for the two above (results unchanged)
  naive_entry            a single output entry of ``naive``
  fast                   Algorithms 3 / 5 / 7 generalised the same way
  ridge                  per-fold ridge / OLS coefficients from the products
                         (normal equations, Cholesky)
  press                  the per-fold models' squared error on each
                         validation partition

This module only marshals numpy arrays into that library (built with gcc on
first use into ``oracle/_build``).  Inputs of any float dtype are widened to
float64 exactly before the call.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcv_oracle.so")
_lock = threading.Lock()
_lib = None

CENTER_X, SCALE_X, CENTER_Y, SCALE_Y = 1, 2, 4, 8
STATUS = {0: "ok", 1: "invalid argument", 2: "fold id out of range", 3: "empty fold",
          4: "partitioning not scalable", 5: "allocation failed"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}: {STATUS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile cv_oracle.c into a shared library (plain gcc, no fp contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, ci = ctypes.c_int64, ctypes.c_int32, ctypes.c_int
            vp = ctypes.c_void_p
            lib.cvo_validation_partitions.argtypes = [i64, i32, vp, vp, vp]
            lib.cvo_validation_partitions.restype = ci
            for name in ("cvo_naive", "cvo_fast"):
                f = getattr(lib, name)
                f.argtypes = [i64, i32, i32, i32, vp, vp, vp, ci, ci, vp, vp, vp, vp]
                f.restype = ci
            lib.cvo_naive_subset.argtypes = [i64, i32, i32, i32, vp, vp, vp, ci, ci, vp, i32,
                                             vp, vp, vp, vp]
            lib.cvo_naive_subset.restype = ci
            lib.cvo_naive_entry.argtypes = [i64, i32, i32, i32, vp, vp, vp, ci, ci,
                                            i32, ci, i32, i32, vp]
            lib.cvo_naive_entry.restype = ci
            lib.cvo_ridge.argtypes = [i32, i32, i32, vp, vp, ctypes.c_double, vp, vp]
            lib.cvo_ridge.restype = ci
            lib.cvo_press.argtypes = [i64, i32, i32, i32, vp, vp, vp, ci, vp, vp, vp, vp]
            lib.cvo_press.restype = ci
            lib.cvo_set_threads.argtypes = [ci]
            lib.cvo_set_threads.restype = ci
            lib.cvo_get_threads.argtypes = []
            lib.cvo_get_threads.restype = ci
            _lib = lib
    return _lib


def set_threads(n):
    """Host threads for ``naive`` / ``naive_subset`` (n <= 0: every online
    processor).  Returns the count now in use.  The results do not depend on
    it: each value is formed by one thread in the same order."""
    return int(_load().cvo_set_threads(int(n)))


def get_threads():
    return int(_load().cvo_get_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _prep(X, Y, folds):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if Y is None:
        Y = np.zeros((X.shape[0], 0))
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    folds = np.ascontiguousarray(folds, dtype=np.int32)
    assert X.ndim == 2 and Y.ndim == 2 and X.shape[0] == Y.shape[0] == folds.shape[0]
    return X, Y, folds


def validation_partitions(folds, P):
    """Algorithm 1: returns (offsets[P+1], rows[N]); fold p's rows are
    rows[offsets[p]:offsets[p+1]] in increasing order."""
    folds = np.ascontiguousarray(folds, dtype=np.int32)
    N = folds.shape[0]
    off = np.zeros(P + 1, np.int64)
    rows = np.zeros(N, np.int64)
    rc = _load().cvo_validation_partitions(N, P, _ptr(folds), _ptr(off), _ptr(rows))
    if rc:
        raise OracleError(rc)
    return off, rows


def _run(name, X, Y, folds, P, flags, ddof):
    X, Y, folds = _prep(X, Y, folds)
    N, K = X.shape
    M = Y.shape[1]
    xtx = np.empty((P, K, K))
    xty = np.empty((P, K, M))
    mean = np.empty((P, K + M))
    std = np.empty((P, K + M))
    rc = getattr(_load(), name)(N, K, M, P, _ptr(folds), _ptr(X), _ptr(Y), int(flags), int(ddof),
                                _ptr(xtx), _ptr(xty), _ptr(mean), _ptr(std))
    if rc:
        raise OracleError(rc)
    return xtx, xty, mean, std


def naive(X, Y, folds, P, flags, ddof=1):
    """Algorithms 2/4/6 for any flags: returns (XTX[P,K,K], XTY[P,K,M],
    mean[P,K+M], std[P,K+M]) for the training partition of every fold."""
    return _run("cvo_naive", X, Y, folds, P, flags, ddof)


def naive_subset(X, Y, folds, P, flags, ddof, which):
    """``naive`` for the folds listed in ``which`` only; returns the same
    P-sized arrays with the other folds' entries left as zeros."""
    X, Y, folds = _prep(X, Y, folds)
    N, K = X.shape
    M = Y.shape[1]
    sel = np.ascontiguousarray(which, dtype=np.int32)
    xtx = np.zeros((P, K, K))
    xty = np.zeros((P, K, M))
    mean = np.zeros((P, K + M))
    std = np.zeros((P, K + M))
    rc = _load().cvo_naive_subset(N, K, M, P, _ptr(folds), _ptr(X), _ptr(Y), int(flags), int(ddof),
                                  _ptr(sel), len(sel), _ptr(xtx), _ptr(xty), _ptr(mean), _ptr(std))
    if rc:
        raise OracleError(rc)
    return xtx, xty, mean, std


def fast(X, Y, folds, P, flags, ddof=1):
    """Algorithms 3/5/7 for any flags; same outputs as ``naive``."""
    return _run("cvo_fast", X, Y, folds, P, flags, ddof)


def naive_entry(X, Y, folds, P, flags, ddof, p, which, i, j):
    """One entry of ``naive``: which=0 -> XTX[p, i, j], which=1 -> XTY[p, i, j]."""
    X, Y, folds = _prep(X, Y, folds)
    N, K = X.shape
    M = Y.shape[1]
    out = np.zeros(1)
    rc = _load().cvo_naive_entry(N, K, M, P, _ptr(folds), _ptr(X), _ptr(Y), int(flags), int(ddof),
                                 int(p), int(which), int(i), int(j), _ptr(out))
    if rc:
        raise OracleError(rc)
    return float(out[0])


def naive_entries(X, Y, folds, P, flags, ddof, samples):
    """Many entries of ``naive``: samples is an iterable of (p, which, i, j).
    The inputs are widened to float64 once for all entries."""
    X, Y, folds = _prep(X, Y, folds)
    N, K = X.shape
    M = Y.shape[1]
    lib = _load()
    out = np.zeros(1)
    res = []
    for (p, which, i, j) in samples:
        rc = lib.cvo_naive_entry(N, K, M, P, _ptr(folds), _ptr(X), _ptr(Y), int(flags), int(ddof),
                                 int(p), int(which), int(i), int(j), _ptr(out))
        if rc:
            raise OracleError(rc)
        res.append(float(out[0]))
    return np.array(res)


def ridge(XTX, XTY, lam):
    """Per-fold B_p = (XTX_p + lam I)^-1 XTY_p (Cholesky; lam = 0 is OLS).
    Returns (B [P, K, M], info [P]): info[p] = j + 1 when column j's pivot is
    not positive (B_p is then NaN)."""
    XTX = np.ascontiguousarray(XTX, dtype=np.float64)
    XTY = np.ascontiguousarray(XTY, dtype=np.float64)
    P, K, _ = XTX.shape
    M = XTY.shape[2]
    B = np.empty((P, K, M))
    info = np.empty(P, dtype=np.int32)
    rc = _load().cvo_ridge(P, K, M, _ptr(XTX), _ptr(XTY), float(lam), _ptr(B), _ptr(info))
    if rc:
        raise OracleError(rc)
    return B, info


def press(X, Y, folds, P, flags, mean, std, B):
    """Squared prediction error of the per-fold models on each validation
    partition, [P, M] (rows preprocessed with their fold's training
    statistics; predictions mapped back to Y's units)."""
    X, Y, folds = _prep(X, Y, folds)
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    std = np.ascontiguousarray(std, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    N, K = X.shape
    M = Y.shape[1]
    out = np.empty((P, M))
    rc = _load().cvo_press(N, K, M, P, _ptr(folds), _ptr(X), _ptr(Y), int(flags), _ptr(mean), _ptr(std),
                           _ptr(B), _ptr(out))
    if rc:
        raise OracleError(rc)
    return out
