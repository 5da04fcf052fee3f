"""Python binding of libcvx.so, the GB300 library for fast partition-based
cross-validation products with training-partition centering and scaling
(Engstrom & Jensen, arXiv 2401.13185).

The functions below carry the names of the C ABI in ``include/cvx.h`` and do
argument marshalling only: every step of the computation runs in the CUDA
kernels of libcvx.so.  PyTorch supplies device memory and streams.  If the
library is missing and cannot be built, importing works but every call raises
``CVXLibraryError``; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "CV_CENTER_X", "CV_SCALE_X", "CV_CENTER_Y", "CV_SCALE_Y",
    "CV_F32", "CV_F64", "CV_PREC_FP64", "CV_PREC_TF32", "CV_PREC_TF32X3", "CV_PREC_BF16X3", "CV_PREC_FP16X3",
    "CV_PREC_AUTO",
    "CVError", "CVXLibraryError", "Plan", "lib", "lib_path",
    "cv_plan", "cv_products", "cv_finalize", "cv_plan_status", "cv_plan_fold_offsets",
    "cv_plan_permutation", "cv_plan_workspace_bytes", "cv_plan_profile", "cv_plan_phase_ms",
    "cv_plan_launches", "cv_products_f64_static", "cv_plan_destroy", "cv_status_string",
    "CvProblem", "CvPlanOptions", "CV_STRATEGY_AUTO", "CV_STRATEGY_FOLD_GROUPED", "Batch", "cv_batch_plan", "cv_batch_products", "cv_batch_status",
    "cv_batch_launches", "cv_batch_plan_options", "cv_batch_destroy", "cv_plan_ex", "cv_ridge",
    "cv_ridge_press", "cv_products_batched", "products", "CV_XTX_FULL", "CV_XTX_PACKED_UPPER",
    "cv_plan_exchange_size", "cv_products_partial", "cv_finalize_total", "xtx_shape",
    "CV_STRATEGY_SMALL_FOLDS", "cv_tune_key", "cv_tune_cache_get", "cv_tune_cache_put", "cv_plan_tune",
]

CV_CENTER_X, CV_SCALE_X, CV_CENTER_Y, CV_SCALE_Y = 1, 2, 4, 8
CV_F32, CV_F64 = 0, 1
CV_PREC_FP64, CV_PREC_TF32, CV_PREC_TF32X3, CV_PREC_BF16X3, CV_PREC_FP16X3, CV_PREC_AUTO = range(6)
PRECISIONS = {"fp64": CV_PREC_FP64, "fp16x3": CV_PREC_FP16X3, "auto": CV_PREC_AUTO,
              "tf32": CV_PREC_TF32, "tf32x3": CV_PREC_TF32X3, "bf16x3": CV_PREC_BF16X3}

STATUS_NAMES = ["CV_OK", "CV_ERR_INVALID_ARG", "CV_ERR_FOLD_RANGE", "CV_ERR_EMPTY_FOLD",
                "CV_ERR_NOT_SCALABLE", "CV_ERR_ALLOC", "CV_ERR_CUDA", "CV_ERR_UNSUPPORTED",
                "CV_ERR_TIMEOUT", "CV_ERR_RANGE"]

# Every symbol include/cvx.h declares.
EXPORTED = ["cv_plan", "cv_products", "cv_finalize", "cv_plan_status", "cv_plan_fold_offsets",
            "cv_plan_permutation", "cv_plan_workspace_bytes", "cv_plan_profile", "cv_plan_phase_ms",
            "cv_plan_launches", "cv_batch_plan", "cv_batch_products", "cv_batch_status",
            "cv_batch_launches", "cv_batch_plan_options", "cv_batch_destroy", "cv_plan_ex",
            "cv_ridge", "cv_ridge_press", "cv_products_batched", "cv_products_f64_static", "cv_plan_destroy",
            "cv_status_string", "cv_plan_exchange_size", "cv_products_partial", "cv_finalize_total",
            "cv_tune_key", "cv_tune_cache_get", "cv_tune_cache_put", "cv_plan_tune"]


class CVXLibraryError(RuntimeError):
    pass


CV_STRATEGY_AUTO, CV_STRATEGY_FOLD_GROUPED, CV_STRATEGY_SMALL_FOLDS = 0, 1, 2


CV_XTX_FULL, CV_XTX_PACKED_UPPER = 0, 1


class CvPlanOptions(ctypes.Structure):
    """struct cv_plan_options of include/cvx.h (zero = defaults)."""
    _fields_ = [("strategy", ctypes.c_int32), ("ctas", ctypes.c_int32), ("fold_begin", ctypes.c_int32),
                ("fold_end", ctypes.c_int32), ("xtx_layout", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("wait_limit_ns", ctypes.c_int64)]


class CvProblem(ctypes.Structure):
    """struct cv_problem of include/cvx.h."""
    _fields_ = [("N", ctypes.c_int64), ("K", ctypes.c_int32), ("M", ctypes.c_int32),
                ("P", ctypes.c_int32), ("fold_ids", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("ldx", ctypes.c_int64), ("Y", ctypes.c_void_p), ("ldy", ctypes.c_int64),
                ("flags", ctypes.c_int), ("ddof", ctypes.c_int), ("XTX", ctypes.c_void_p),
                ("XTY", ctypes.c_void_p), ("mean_out", ctypes.c_void_p), ("std_out", ctypes.c_void_p)]


class CVError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else f"status {code}"
        super().__init__(f"{where}: {name}" if where else name)
        self.code = code
        self.name = name


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libcvx.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            try:
                path = _build.build()
            except Exception as e:  # no nvcc / compile error
                if os.path.exists(_build.LIB):
                    path = _build.LIB
                else:
                    raise CVXLibraryError(f"libcvx.so is not built and cannot be built: {e}") from e
            L = ctypes.CDLL(path)
            vp, i64, i32, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
            L.cv_plan.argtypes = [ctypes.POINTER(vp), i64, i32, i32, i32, vp, ci, ci, ci, ci, vp]
            L.cv_plan.restype = ci
            L.cv_plan_ex.argtypes = [ctypes.POINTER(vp), i64, i32, i32, i32, vp, ci, ci, ci, ci,
                                     ctypes.POINTER(CvPlanOptions), vp]
            L.cv_plan_ex.restype = ci
            L.cv_tune_key.argtypes = [i64, i32, i32, i32, ci, ci, ci, ctypes.c_char_p, i32]
            L.cv_tune_key.restype = ci
            L.cv_tune_cache_get.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(CvPlanOptions),
                                            ctypes.POINTER(ctypes.c_double)]
            L.cv_tune_cache_get.restype = ci
            L.cv_tune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(CvPlanOptions),
                                            ctypes.c_double]
            L.cv_tune_cache_put.restype = ci
            L.cv_plan_tune.argtypes = [i64, i32, i32, i32, vp, ci, ci, ci, ci, vp, i64, vp, i64, ci, ci,
                                       ctypes.c_char_p, ctypes.POINTER(CvPlanOptions),
                                       ctypes.POINTER(ctypes.c_double), vp]
            L.cv_plan_tune.restype = ci
            L.cv_products.argtypes = [vp, vp, i64, vp, i64, ci, ci, vp, vp, vp, vp, vp]
            L.cv_products.restype = ci
            L.cv_finalize.argtypes = [vp, vp, i64, vp, i64, ci, ci, vp, vp, vp, vp, vp]
            L.cv_finalize.restype = ci
            L.cv_plan_status.argtypes = [vp, vp]
            L.cv_plan_status.restype = ci
            L.cv_plan_fold_offsets.argtypes = [vp, vp]
            L.cv_plan_fold_offsets.restype = ci
            L.cv_plan_permutation.argtypes = [vp, vp]
            L.cv_plan_permutation.restype = ci
            L.cv_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(i64)]
            L.cv_plan_workspace_bytes.restype = ci
            L.cv_plan_profile.argtypes = [vp, ci]
            L.cv_plan_profile.restype = ci
            L.cv_plan_phase_ms.argtypes = [vp, vp, ctypes.POINTER(i32)]
            L.cv_plan_phase_ms.restype = ci
            L.cv_plan_launches.argtypes = [vp, ctypes.POINTER(i64)]
            L.cv_plan_launches.restype = ci
            PP = ctypes.POINTER(CvProblem)
            L.cv_batch_plan.argtypes = [ctypes.POINTER(vp), PP, i32, ci, ci, ci, ci, vp]
            L.cv_batch_plan.restype = ci
            L.cv_batch_products.argtypes = [vp, PP, vp]
            L.cv_batch_products.restype = ci
            L.cv_batch_status.argtypes = [vp, vp]
            L.cv_batch_status.restype = ci
            L.cv_ridge.argtypes = [i32, i32, i32, vp, vp, ctypes.c_double, vp, vp, vp, vp]
            L.cv_ridge.restype = ci
            L.cv_ridge_press.argtypes = [vp, vp, i64, vp, i64, ci, vp, vp, vp, vp, vp]
            L.cv_ridge_press.restype = ci
            L.cv_batch_plan_options.argtypes = [vp, i32, ctypes.POINTER(CvPlanOptions)]
            L.cv_batch_plan_options.restype = ci
            L.cv_batch_launches.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
            L.cv_batch_launches.restype = ci
            L.cv_batch_destroy.argtypes = [vp]
            L.cv_batch_destroy.restype = ci
            L.cv_products_batched.argtypes = [PP, i32, ci, ci, ci, vp]
            L.cv_products_batched.restype = ci
            L.cv_products_f64_static.argtypes = [i64, i32, i32, i32, vp, vp, i64, vp, i64, ci, ci, ci, ci,
                                                 vp, vp, vp, vp, vp]
            L.cv_products_f64_static.restype = ci
            L.cv_plan_exchange_size.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
            L.cv_plan_exchange_size.restype = ci
            L.cv_products_partial.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp]
            L.cv_products_partial.restype = ci
            L.cv_finalize_total.argtypes = [vp, vp, vp, ci, ci, vp, vp, vp, vp, vp]
            L.cv_finalize_total.restype = ci
            L.cv_plan_destroy.argtypes = [vp]
            L.cv_plan_destroy.restype = ci
            L.cv_status_string.argtypes = [ci]
            L.cv_status_string.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise CVError(code, where)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t) -> int:
    import torch
    if t in (torch.float32, np.float32, "f32", "float32"):
        return CV_F32
    if t in (torch.float64, np.float64, "f64", "float64"):
        return CV_F64
    raise ValueError(f"unsupported dtype {t}")


class Plan:
    """Owner of a cv_plan_t handle (destroyed with the object)."""

    def __init__(self, handle: int, N: int, K: int, M: int, P: int, in_dtype: int, out_dtype: int,
                 prec: int, options: Optional["CvPlanOptions"] = None):
        self.handle = handle
        self.N, self.K, self.M, self.P = N, K, M, P
        self.in_dtype, self.out_dtype, self.prec = in_dtype, out_dtype, prec
        o = options if options is not None else CvPlanOptions()
        self.sharded = not (o.fold_begin == 0 and o.fold_end == 0)
        self.fold_begin = o.fold_begin if self.sharded else 0
        self.fold_end = o.fold_end if self.sharded else P
        self.packed = o.xtx_layout == CV_XTX_PACKED_UPPER

    @property
    def folds_out(self) -> int:
        """Folds the plan's outputs hold (its fold range)."""
        return self.fold_end - self.fold_begin

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.handle:
            lib().cv_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    @property
    def _h(self):
        if not self.handle:
            raise CVError(1, "plan destroyed")
        return ctypes.c_void_p(self.handle)


def cv_plan(N: int, K: int, M: int, P: int, fold_ids, in_dtype=CV_F32, out_dtype=CV_F64,
            prec=CV_PREC_AUTO, stream=None) -> Plan:
    """cv_plan: fold_ids is a CUDA int32 tensor or a host int32 array/tensor."""
    return cv_plan_ex(N, K, M, P, fold_ids, in_dtype, out_dtype, prec, None, stream)


def _options(options) -> Optional[CvPlanOptions]:
    """None, a CvPlanOptions, a (strategy, ctas) pair or a dict of field values."""
    if options is None or isinstance(options, CvPlanOptions):
        return options
    if isinstance(options, dict):
        return CvPlanOptions(**options)
    return CvPlanOptions(*options)


def cv_plan_ex(N: int, K: int, M: int, P: int, fold_ids, in_dtype=CV_F32, out_dtype=CV_F64,
               prec=CV_PREC_AUTO, options=None, stream=None) -> Plan:
    """cv_plan_ex: options is None (cv_plan), a CvPlanOptions, a (strategy,
    ctas) pair or a dict of CvPlanOptions fields."""
    import torch
    if isinstance(prec, str):
        prec = PRECISIONS[prec]
    in_code = in_dtype if isinstance(in_dtype, int) else _dtype_code(in_dtype)
    out_code = out_dtype if isinstance(out_dtype, int) else _dtype_code(out_dtype)
    keep = None
    if isinstance(fold_ids, torch.Tensor):
        if fold_ids.dtype != torch.int32 or not fold_ids.is_contiguous():
            raise ValueError("fold_ids must be a contiguous int32 tensor")
        on_dev = 1 if fold_ids.is_cuda else 0
        ptr = fold_ids.data_ptr()
        keep = fold_ids
    else:
        keep = np.ascontiguousarray(fold_ids, dtype=np.int32)
        on_dev = 0
        ptr = keep.ctypes.data
    if len(keep) != N:
        raise ValueError("fold_ids must have N entries")
    h = ctypes.c_void_p()
    opts = _options(options)
    code = lib().cv_plan_ex(ctypes.byref(h), N, K, M, P, ctypes.c_void_p(ptr), on_dev, in_code, out_code,
                            int(prec), ctypes.byref(opts) if opts is not None else None,
                            ctypes.c_void_p(_stream_ptr(stream)))
    _check(code, "cv_plan_ex")
    return Plan(h.value, N, K, M, P, in_code, out_code, int(prec), opts)


def _path_bytes(path):
    return None if path is None else os.fsencode(path)


def cv_tune_key(N: int, K: int, M: int, P: int, in_dtype=CV_F32, out_dtype=CV_F64, prec=CV_PREC_AUTO) -> str:
    """cv_tune_key: the tuning cache's key of a problem shape on the current device."""
    if isinstance(prec, str):
        prec = PRECISIONS[prec]
    in_code = in_dtype if isinstance(in_dtype, int) else _dtype_code(in_dtype)
    out_code = out_dtype if isinstance(out_dtype, int) else _dtype_code(out_dtype)
    buf = ctypes.create_string_buffer(160)
    _check(lib().cv_tune_key(N, K, M, P, in_code, out_code, int(prec), buf, len(buf)), "cv_tune_key")
    return buf.value.decode()


def cv_tune_cache_get(path, key: str):
    """cv_tune_cache_get: (CvPlanOptions, ms) cached for `key` in the JSON file at
    `path` (None: $CVX_TUNE_CACHE), or None when there is no entry."""
    o, ms = CvPlanOptions(), ctypes.c_double(0.0)
    code = lib().cv_tune_cache_get(_path_bytes(path), key.encode(), ctypes.byref(o), ctypes.byref(ms))
    if code == 7:   # CV_ERR_UNSUPPORTED: no entry
        return None
    _check(code, "cv_tune_cache_get")
    return o, ms.value


def cv_tune_cache_put(path, key: str, options, ms: float) -> None:
    """cv_tune_cache_put: record options and time for `key` (None path: $CVX_TUNE_CACHE)."""
    o = _options(options) or CvPlanOptions()
    _check(lib().cv_tune_cache_put(_path_bytes(path), key.encode(), ctypes.byref(o), float(ms)),
           "cv_tune_cache_put")


def cv_plan_tune(N: int, K: int, M: int, P: int, fold_ids, X, Y, flags: int, ddof: int, in_dtype=CV_F32,
                 out_dtype=CV_F64, prec=CV_PREC_AUTO, cache_path=None, stream=None):
    """cv_plan_tune on CUDA tensors X [N, K] and Y [N, M] (fold_ids as for
    cv_plan_ex): the fastest measured (or cached) plan options and their time
    in ms per cv_products call."""
    import torch
    if isinstance(prec, str):
        prec = PRECISIONS[prec]
    in_code = in_dtype if isinstance(in_dtype, int) else _dtype_code(in_dtype)
    out_code = out_dtype if isinstance(out_dtype, int) else _dtype_code(out_dtype)
    if isinstance(fold_ids, torch.Tensor):
        if fold_ids.dtype != torch.int32 or not fold_ids.is_contiguous():
            raise ValueError("fold_ids must be a contiguous int32 tensor")
        keep, on_dev, ptr = fold_ids, (1 if fold_ids.is_cuda else 0), fold_ids.data_ptr()
    else:
        keep = np.ascontiguousarray(fold_ids, dtype=np.int32)
        on_dev, ptr = 0, keep.ctypes.data
    if len(keep) != N:
        raise ValueError("fold_ids must have N entries")
    if X.dim() != 2 or X.stride(1) != 1 or (Y is not None and Y.numel() > 0 and (Y.dim() != 2 or Y.stride(1) != 1)):
        raise ValueError("X and Y must be 2-D with unit column stride")
    for t, name in ((X, "X"), (Y, "Y")):
        if t is not None and t.numel() > 0 and _dtype_code(t.dtype) != in_code:
            raise ValueError(f"{name} must have the plan's input dtype")
    yp, ldy = (_dptr(Y), Y.stride(0)) if Y is not None and Y.numel() > 0 else (ctypes.c_void_p(0), max(M, 1))
    best, ms = CvPlanOptions(), ctypes.c_double(0.0)
    code = lib().cv_plan_tune(N, K, M, P, ctypes.c_void_p(ptr), on_dev, in_code, out_code, int(prec), _dptr(X),
                              X.stride(0) if X.shape[0] > 1 else K, yp, ldy, int(flags), int(ddof),
                              _path_bytes(cache_path), ctypes.byref(best), ctypes.byref(ms),
                              ctypes.c_void_p(_stream_ptr(stream)))
    _check(code, "cv_plan_tune")
    return best, ms.value


def xtx_shape(plan: Plan):
    """Shape of the XTX output of a plan: (folds, K, K), or (folds, K (K + 1) / 2)
    for the packed upper-triangular layout."""
    if plan.packed:
        return (plan.folds_out, plan.K * (plan.K + 1) // 2)
    return (plan.folds_out, plan.K, plan.K)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _require_dtype(t, code: int, what: str):
    """Raise ValueError when tensor t (if given) is not of the cv_dtype code."""
    if t is not None and t.numel() > 0 and _dtype_code(t.dtype) != code:
        raise ValueError(f"{what} must be {'float32' if code == CV_F32 else 'float64'}, got {t.dtype}")


def _require_stats(*ts):
    import torch
    for t in ts:
        if t is not None and t.dtype != torch.float64:
            raise ValueError("mean_out / std_out must be float64")


def _check_call_dtypes(plan: Plan, X, Y, XTX, XTY, mean_out, std_out):
    _require_dtype(X, plan.in_dtype, "X")
    _require_dtype(Y, plan.in_dtype, "Y")
    _require_dtype(XTX, plan.out_dtype, "XTX")
    _require_dtype(XTY, plan.out_dtype, "XTY")
    _require_stats(mean_out, std_out)


def cv_products(plan: Plan, X, Y, flags: int, ddof: int, XTX=None, XTY=None, mean_out=None,
                std_out=None, stream=None):
    """cv_products on CUDA tensors (row-major X: N x K, Y: N x M; outputs as in cvx.h)."""
    _check_call_dtypes(plan, X, Y, XTX, XTY, mean_out, std_out)
    ldx = X.stride(0) if X.dim() == 2 and X.shape[0] > 1 else plan.K
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be 2-D with unit column stride")
    if Y is not None and Y.numel() > 0:
        if Y.dim() != 2 or Y.stride(1) != 1:
            raise ValueError("Y must be 2-D with unit column stride")
        ldy = Y.stride(0)
        yp = _dptr(Y)
    else:
        ldy, yp = max(plan.M, 1), ctypes.c_void_p(0)
    code = lib().cv_products(plan._h, _dptr(X), ldx, yp, ldy, int(flags), int(ddof), _dptr(XTX),
                             _dptr(XTY), _dptr(mean_out), _dptr(std_out),
                             ctypes.c_void_p(_stream_ptr(stream)))
    _check(code, "cv_products")


def _inputs(plan: Plan, X, Y):
    """(X pointer, ldx, Y pointer, ldy) of CUDA tensors; X may be None."""
    if X is None:
        xp, ldx = ctypes.c_void_p(0), plan.K
    else:
        if X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("X must be 2-D with unit column stride")
        xp, ldx = _dptr(X), (X.stride(0) if X.shape[0] > 1 else plan.K)
    if Y is not None and Y.numel() > 0:
        if Y.dim() != 2 or Y.stride(1) != 1:
            raise ValueError("Y must be 2-D with unit column stride")
        yp, ldy = _dptr(Y), Y.stride(0)
    else:
        yp, ldy = ctypes.c_void_p(0), max(plan.M, 1)
    return xp, ldx, yp, ldy


def cv_finalize(plan: Plan, flags: int, ddof: int, XTX=None, XTY=None, mean_out=None, std_out=None,
                X=None, Y=None, stream=None):
    """cv_finalize: other flags / ddof from the plan's last cv_products (X and
    Y are needed only by small-fold plans)."""
    _check_call_dtypes(plan, X, Y, XTX, XTY, mean_out, std_out)
    xp, ldx, yp, ldy = _inputs(plan, X, Y)
    code = lib().cv_finalize(plan._h, xp, ldx, yp, ldy, int(flags), int(ddof), _dptr(XTX), _dptr(XTY),
                             _dptr(mean_out), _dptr(std_out), ctypes.c_void_p(_stream_ptr(stream)))
    _check(code, "cv_finalize")


def cv_plan_exchange_size(plan: Plan):
    """(n_int, n_real): lengths of a plan's int64 and float64 exchange buffers."""
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().cv_plan_exchange_size(plan._h, ctypes.byref(a), ctypes.byref(b)), "cv_plan_exchange_size")
    return a.value, b.value


def cv_products_partial(plan: Plan, X, Y, ex_int, ex_real, stream=None):
    """cv_products_partial on CUDA tensors: this shard's partial total into the
    exchange buffers (int64 [n_int] or None when n_int is 0, float64 [n_real])."""
    import torch
    _require_dtype(X, plan.in_dtype, "X")
    _require_dtype(Y, plan.in_dtype, "Y")
    if ex_real.dtype != torch.float64 or (ex_int is not None and ex_int.dtype != torch.int64):
        raise ValueError("exchange buffers are int64 and float64")
    xp, ldx, yp, ldy = _inputs(plan, X, Y)
    _check(lib().cv_products_partial(plan._h, xp, ldx, yp, ldy, _dptr(ex_int), _dptr(ex_real),
                                     ctypes.c_void_p(_stream_ptr(stream))), "cv_products_partial")


def cv_finalize_total(plan: Plan, ex_int, ex_real, flags: int, ddof: int, XTX=None, XTY=None, mean_out=None,
                      std_out=None, stream=None):
    """cv_finalize_total: the shard's folds from the exchange buffers summed over
    every shard."""
    _check_call_dtypes(plan, None, None, XTX, XTY, mean_out, std_out)
    _check(lib().cv_finalize_total(plan._h, _dptr(ex_int), _dptr(ex_real), int(flags), int(ddof), _dptr(XTX),
                                   _dptr(XTY), _dptr(mean_out), _dptr(std_out),
                                   ctypes.c_void_p(_stream_ptr(stream))), "cv_finalize_total")


def cv_plan_status(plan: Plan, stream=None) -> int:
    return lib().cv_plan_status(plan._h, ctypes.c_void_p(_stream_ptr(stream)))


def cv_plan_fold_offsets(plan: Plan) -> np.ndarray:
    out = np.zeros(plan.P + 1, np.int64)
    _check(lib().cv_plan_fold_offsets(plan._h, ctypes.c_void_p(out.ctypes.data)), "cv_plan_fold_offsets")
    return out


def cv_plan_permutation(plan: Plan) -> np.ndarray:
    out = np.zeros(plan.N, np.int32)
    _check(lib().cv_plan_permutation(plan._h, ctypes.c_void_p(out.ctypes.data)), "cv_plan_permutation")
    return out


def cv_plan_workspace_bytes(plan: Plan) -> int:
    b = ctypes.c_int64(0)
    _check(lib().cv_plan_workspace_bytes(plan._h, ctypes.byref(b)), "cv_plan_workspace_bytes")
    return b.value


def cv_plan_profile(plan: Plan, enable: bool = True):
    _check(lib().cv_plan_profile(plan._h, 1 if enable else 0), "cv_plan_profile")


PHASES = ("shift_estimate", "convert", "gram", "fold_sums", "fold_stats", "epilogue")


def cv_plan_phase_ms(plan: Plan):
    """Summed device ms per phase over the recorded calls, and the call count."""
    ms = np.zeros(len(PHASES), np.float64)
    n = ctypes.c_int32(0)
    _check(lib().cv_plan_phase_ms(plan._h, ctypes.c_void_p(ms.ctypes.data), ctypes.byref(n)),
           "cv_plan_phase_ms")
    return dict(zip(PHASES, ms.tolist())), n.value


def cv_plan_launches(plan: Plan) -> int:
    """Kernels enqueued by cv_products calls on this plan since it was made."""
    n = ctypes.c_int64(0)
    _check(lib().cv_plan_launches(plan._h, ctypes.byref(n)), "cv_plan_launches")
    return n.value


def _problem_array(problems):
    """A ctypes array of CvProblem from dicts with CUDA tensors X, Y, folds and
    optional XTX, XTY, mean, std, plus ints P, flags, ddof."""
    arr = (CvProblem * len(problems))()
    for a, d in zip(arr, problems):
        X, Y, f = d["X"], d.get("Y"), d["folds"]
        if X.dim() != 2 or X.stride(1) != 1 or (Y is not None and Y.numel() and Y.stride(1) != 1):
            raise ValueError("X and Y must be 2-D with unit column stride")
        if f.dtype.itemsize != 4 or not f.is_cuda or not f.is_contiguous():
            raise ValueError("folds must be a contiguous CUDA int32 tensor")
        N, K = X.shape
        M = 0 if Y is None else Y.shape[1]
        a.N, a.K, a.M, a.P = N, K, M, int(d["P"])
        a.fold_ids, a.X, a.ldx = f.data_ptr(), X.data_ptr(), X.stride(0) if N > 1 else K
        a.Y = Y.data_ptr() if M > 0 else None
        a.ldy = Y.stride(0) if M > 0 and N > 1 else max(M, 1)
        a.flags, a.ddof = int(d.get("flags", 15)), int(d.get("ddof", 1))
        for name, key in (("XTX", "XTX"), ("XTY", "XTY"), ("mean_out", "mean"), ("std_out", "std")):
            t = d.get(key)
            setattr(a, name, t.data_ptr() if t is not None else None)
    return arr


class Batch:
    """Owner of a cv_batch_t handle (one plan per problem; batched launches or a CUDA graph)."""

    def __init__(self, handle: int, count: int):
        self.handle, self.count = handle, count

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.handle:
            lib().cv_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    @property
    def _h(self):
        if not self.handle:
            raise CVError(1, "batch destroyed")
        return ctypes.c_void_p(self.handle)


def cv_batch_plan(problems, in_dtype=CV_F32, out_dtype=CV_F64, prec=CV_PREC_AUTO, stream=None) -> Batch:
    """cv_batch_plan over a list of problem dicts (see _problem_array)."""
    if isinstance(prec, str):
        prec = PRECISIONS[prec]
    in_code = in_dtype if isinstance(in_dtype, int) else _dtype_code(in_dtype)
    out_code = out_dtype if isinstance(out_dtype, int) else _dtype_code(out_dtype)
    arr = _problem_array(problems)
    h = ctypes.c_void_p()
    _check(lib().cv_batch_plan(ctypes.byref(h), arr, len(problems), 1, in_code, out_code, int(prec),
                               ctypes.c_void_p(_stream_ptr(stream))), "cv_batch_plan")
    return Batch(h.value, len(problems))


def cv_batch_products(batch: Batch, problems, stream=None):
    if len(problems) != batch.count:
        raise ValueError("problem count differs from the batch's")
    arr = _problem_array(problems)
    _check(lib().cv_batch_products(batch._h, arr, ctypes.c_void_p(_stream_ptr(stream))), "cv_batch_products")


def cv_batch_status(batch: Batch, stream=None) -> int:
    return lib().cv_batch_status(batch._h, ctypes.c_void_p(_stream_ptr(stream)))


def cv_batch_launches(batch: Batch):
    """(kernels enqueued by cv_batch_products so far, True if the batch runs as
    batched launches rather than a graph)."""
    n, b = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().cv_batch_launches(batch._h, ctypes.byref(n), ctypes.byref(b)), "cv_batch_launches")
    return n.value, bool(b.value)


def cv_ridge(XTX, XTY, lam: float, L=None, B=None, info=None, stream=None):
    """cv_ridge on CUDA FP64 tensors XTX [P, K, K] and XTY [P, K, M]: per-fold
    B_p = (XTX_p + lam I)^-1 XTY_p.  Returns (B, info) (allocating them and the
    factor scratch L when not given)."""
    import torch
    if XTX.dtype != torch.float64 or XTY.dtype != torch.float64 or not (XTX.is_cuda and XTY.is_cuda):
        raise ValueError("cv_ridge takes CUDA float64 tensors")
    XTX, XTY = XTX.contiguous(), XTY.contiguous()
    P, K, _ = XTX.shape
    M = XTY.shape[2]
    dev = XTX.device
    L = torch.empty((P, K, K), dtype=torch.float64, device=dev) if L is None else L
    B = torch.empty((P, K, M), dtype=torch.float64, device=dev) if B is None else B
    info = torch.empty(P, dtype=torch.int32, device=dev) if info is None else info
    _check(lib().cv_ridge(P, K, M, _dptr(XTX), _dptr(XTY), float(lam), _dptr(L), _dptr(B), _dptr(info),
                          ctypes.c_void_p(_stream_ptr(stream))), "cv_ridge")
    return B, info


def cv_ridge_press(plan: Plan, X, Y, flags: int, mean, std, B, press=None, stream=None):
    """cv_ridge_press: [P, M] squared validation error of the per-fold models."""
    import torch
    x, ldx, y, ldy = _inputs(plan, X, Y)
    press = torch.empty((plan.P, plan.M), dtype=torch.float64, device=X.device) if press is None else press
    _check(lib().cv_ridge_press(plan._h, x, ldx, y, ldy, int(flags), _dptr(mean.contiguous()),
                                _dptr(std.contiguous()), _dptr(B.contiguous()), _dptr(press),
                                ctypes.c_void_p(_stream_ptr(stream))), "cv_ridge_press")
    return press


def cv_batch_plan_options(batch: Batch, index: int):
    """(strategy, ctas) problem `index` of the batch was planned with."""
    o = CvPlanOptions()
    _check(lib().cv_batch_plan_options(batch._h, int(index), ctypes.byref(o)), "cv_batch_plan_options")
    return o.strategy, o.ctas


def cv_batch_destroy(batch: Batch):
    batch.destroy()


def cv_products_batched(problems, in_dtype=CV_F32, out_dtype=CV_F64, prec=CV_PREC_AUTO, stream=None):
    """One-shot batch (plans, graph, products, status, release); synchronises the stream."""
    if isinstance(prec, str):
        prec = PRECISIONS[prec]
    in_code = in_dtype if isinstance(in_dtype, int) else _dtype_code(in_dtype)
    out_code = out_dtype if isinstance(out_dtype, int) else _dtype_code(out_dtype)
    arr = _problem_array(problems)
    _check(lib().cv_products_batched(arr, len(problems), in_code, out_code, int(prec),
                                     ctypes.c_void_p(_stream_ptr(stream))), "cv_products_batched")


def cv_products_f64_static(X, Y, fold_ids, P: int, flags: int, ddof: int, XTX=None, XTY=None,
                           mean_out=None, std_out=None, stream=None):
    """cv_products_f64_static on CUDA tensors: the FP64 products of a small
    problem (N <= 32768, K + M + 1 <= 128, P <= 16) without any device
    allocation inside the library; the caller provides every output."""
    N, K = X.shape
    M = 0 if Y is None else Y.shape[1]
    if X.stride(1) != 1 or (Y is not None and M > 0 and Y.stride(1) != 1):
        raise ValueError("X and Y need unit column stride")
    if not fold_ids.is_cuda or fold_ids.dtype.itemsize != 4:
        raise ValueError("fold_ids must be a CUDA int32 tensor")
    in_code = _dtype_code(X.dtype)
    if Y is not None and M > 0:
        _require_dtype(Y, in_code, "Y (the dtype of X)")
    out_t = XTX if XTX is not None else XTY
    out_code = _dtype_code(out_t.dtype) if out_t is not None else CV_F64
    _require_dtype(XTY, out_code, "XTY (the dtype of XTX)")
    _require_stats(mean_out, std_out)
    ldy = Y.stride(0) if (Y is not None and M > 0) else max(M, 1)
    code = lib().cv_products_f64_static(N, K, M, P, _dptr(fold_ids), _dptr(X), X.stride(0),
                                        _dptr(Y) if M > 0 else ctypes.c_void_p(0), ldy, in_code, out_code,
                                        int(flags), int(ddof), _dptr(XTX), _dptr(XTY), _dptr(mean_out),
                                        _dptr(std_out), ctypes.c_void_p(_stream_ptr(stream)))
    _check(code, "cv_products_f64_static")


def cv_plan_destroy(plan: Plan):
    plan.destroy()


def cv_status_string(code: int) -> str:
    return lib().cv_status_string(int(code)).decode()


def products(X, Y, folds, P: int, flags: int = 15, ddof: int = 1, precision="auto",
             out_dtype=None, stream=None, plan: Optional[Plan] = None, with_stats: bool = False):
    """Plan (unless given) and run cv_products on CUDA tensors; returns
    (XTX[P,K,K], XTY[P,K,M]) or, with with_stats, also (mean, std)."""
    import torch
    N, K = X.shape
    M = 0 if Y is None else Y.shape[1]
    out_dtype = out_dtype or torch.float64
    if plan is None:
        plan = cv_plan(N, K, M, P, folds, X.dtype, out_dtype, precision, stream)
    XTX = torch.empty(xtx_shape(plan), dtype=out_dtype, device=X.device)
    XTY = torch.empty((P, K, M), dtype=out_dtype, device=X.device) if M > 0 else None
    mean = torch.empty((P, K + M), dtype=torch.float64, device=X.device) if with_stats else None
    std = torch.empty((P, K + M), dtype=torch.float64, device=X.device) if with_stats else None
    cv_products(plan, X, Y, flags, ddof, XTX, XTY, mean, std, stream)
    if with_stats:
        return XTX, XTY, mean, std
    return XTX, XTY
