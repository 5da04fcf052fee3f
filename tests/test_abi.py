"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every symbol include/cvx.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2401_13185_gb300 as cvx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "cvx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cv_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    syms = _declared_symbols()
    for s in ("cv_plan", "cv_products", "cv_plan_destroy", "cv_status_string"):
        assert s in syms
    assert sorted(cvx.EXPORTED) == syms


def test_library_loads_and_exports_every_declared_symbol():
    L = cvx.lib()
    for s in _declared_symbols():
        assert hasattr(L, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", cvx.lib_path()], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\bT (cv_\w+)", out.stdout))
        assert set(_declared_symbols()) <= exported


def test_build_targets_sm_103a_only():
    from paper_2401_13185_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings():
    for code, name in enumerate(cvx.STATUS_NAMES):
        assert cvx.cv_status_string(code) == name
    assert cvx.cv_status_string(99) == "CV_ERR_UNKNOWN"


def test_invalid_arguments_rejected_on_host():
    L = cvx.lib()
    h = ctypes.c_void_p()
    folds = (ctypes.c_int32 * 4)(0, 1, 0, 1)
    # null out-pointer
    assert L.cv_plan(None, 4, 2, 1, 2, folds, 0, 0, 1, 0, None) == 1
    # N < 2, P < 2, P > N, K < 1, M < 0, null folds
    for args in [(1, 2, 1, 2), (4, 2, 1, 1), (4, 2, 1, 5), (4, 0, 1, 2), (4, 2, -1, 2)]:
        assert L.cv_plan(ctypes.byref(h), *args, folds, 0, 0, 1, 0, None) == 1
        assert h.value is None
    assert L.cv_plan(ctypes.byref(h), 4, 2, 1, 2, None, 0, 0, 1, 0, None) == 1
    # bad dtypes / precisions
    assert L.cv_plan(ctypes.byref(h), 4, 2, 1, 2, folds, 0, 7, 1, 0, None) == 1
    assert L.cv_plan(ctypes.byref(h), 4, 2, 1, 2, folds, 0, 0, 1, 42, None) == 1
    # plan options: unknown strategy, negative ctas, fold ranges outside
    # [0, P) or empty, the small-fold strategy with a fold range, unknown
    # layout, reserved != 0, negative wait limit
    for o in [(3, 0), (-1, 0), (0, -1), (0, 0, 1, 1), (0, 0, 0, 3), (0, 0, -1, 1), (0, 0, 1, 0),
              (2, 0, 0, 1), (0, 0, 0, 0, 2), (0, 0, 0, 0, 0, 1), (0, 0, 0, 0, 0, 0, -5)]:
        opts = cvx.CvPlanOptions(*o)
        assert L.cv_plan_ex(ctypes.byref(h), 4, 2, 1, 2, folds, 0, 0, 1, 0, ctypes.byref(opts), None) == 1, o
        assert h.value is None
    assert ctypes.sizeof(cvx.CvPlanOptions) == 32
    # tuning entry points: null outputs and pointers are rejected before any device call
    best = cvx.CvPlanOptions()
    assert L.cv_plan_tune(4, 2, 1, 2, folds, 0, 0, 1, 0, None, 2, None, 1, 15, 1, None, None, None, None) == 1
    assert L.cv_plan_tune(4, 2, 1, 2, None, 0, 0, 1, 0, None, 2, None, 1, 15, 1, None, ctypes.byref(best),
                          None, None) == 1
    assert L.cv_tune_key(4, 2, 1, 2, 0, 1, 0, None, 64) == 1
    assert L.cv_tune_cache_get(None, b"k", None, None) == 1
    # sharding entry points with a null plan
    n = ctypes.c_int64()
    assert L.cv_plan_exchange_size(None, ctypes.byref(n), ctypes.byref(n)) == 1
    assert L.cv_products_partial(None, None, 2, None, 1, None, None, None) == 1
    assert L.cv_finalize_total(None, None, None, 15, 1, None, None, None, None, None) == 1
    assert L.cv_batch_plan_options(None, 0, None) == 1
    # ridge entry points: bad sizes, null pointers, a non-finite lambda
    assert L.cv_ridge(0, 3, 1, None, None, 0.0, None, None, None, None) == 1
    assert L.cv_ridge(1, 3, 1, None, None, float("inf"), None, None, None, None) == 1
    assert L.cv_ridge_press(None, None, 3, None, 1, 0, None, None, None, None, None) == 1
    assert L.cv_batch_launches(None, None, None) == 1
    # products / queries with a null plan
    assert L.cv_products(None, None, 2, None, 1, 0, 1, None, None, None, None, None) == 1
    assert L.cv_finalize(None, None, 2, None, 1, 0, 1, None, None, None, None, None) == 1
    assert L.cv_plan_status(None, None) == 1
    assert L.cv_plan_fold_offsets(None, None) == 1
    assert L.cv_plan_permutation(None, None) == 1
    assert L.cv_plan_workspace_bytes(None, None) == 1
    assert L.cv_plan_destroy(None) == 0
