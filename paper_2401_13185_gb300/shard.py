"""Fold sharding over several GPUs, one process per GPU.

The library's sharded plans (cv_plan_options fold_begin / fold_end) contract
only the rows of the folds a GPU owns.  By Lemma 2 of the paper the Gram over
all rows is the sum of the folds' Grams, so one element-wise sum of the
shards' partial totals (cv_products_partial's exchange buffers) over the
process group gives every shard the total it needs to finish its folds
(cv_finalize_total).  This module only decides which folds a rank owns and
moves the exchange buffers through ``torch.distributed``; every arithmetic
step of the products runs in the CUDA library.
"""
from __future__ import annotations

from typing import Optional, Tuple

from . import (CV_STRATEGY_FOLD_GROUPED, CvPlanOptions, Plan, cv_finalize_total, cv_plan_exchange_size,
               cv_plan_ex, cv_products_partial, xtx_shape)


def owned_folds(P: int, world: int, rank: int) -> Tuple[int, int]:
    """The contiguous fold range [begin, end) rank `rank` of `world` owns: the
    P folds split as evenly as possible, the first P mod world ranks taking
    one fold more."""
    if not (1 <= world <= P) or not (0 <= rank < world):
        raise ValueError("need 1 <= world <= P and 0 <= rank < world")
    base, extra = divmod(P, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def shard_options(P: int, world: int, rank: int, ctas: int = 0, xtx_layout: int = 0,
                  wait_limit_ns: int = 0) -> CvPlanOptions:
    """Plan options of rank `rank`'s shard (every shard must use the same ctas)."""
    b, e = owned_folds(P, world, rank)
    return CvPlanOptions(strategy=CV_STRATEGY_FOLD_GROUPED, ctas=ctas, fold_begin=b, fold_end=e,
                         xtx_layout=xtx_layout, reserved=0, wait_limit_ns=wait_limit_ns)


def shard_plan(N: int, K: int, M: int, P: int, fold_ids, world: int, rank: int, in_dtype, out_dtype, prec,
               ctas: int = 0, xtx_layout: int = 0, stream=None) -> Plan:
    return cv_plan_ex(N, K, M, P, fold_ids, in_dtype, out_dtype, prec,
                      shard_options(P, world, rank, ctas, xtx_layout), stream)


def allreduce_exchange(ex_int, ex_real, group=None, stream=None):
    """Sum the exchange buffers over the process group in place, ordered after
    the work already on `stream` (default: the current stream) and before the
    work enqueued on it afterwards.  A backend that reduces device tensors
    (NCCL) reduces them where they are, on the stream; otherwise (gloo) they
    go through host copies."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    bufs = [t for t in (ex_int, ex_real) if t is not None and t.numel() > 0]
    if not ex_real.is_cuda:
        for t in bufs:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return
    s = stream if stream is not None else torch.cuda.current_stream(ex_real.device)
    with torch.cuda.stream(s):
        if backend == "nccl":
            for t in bufs:
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return
        s.synchronize()
        for t in bufs:
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
            t.copy_(h)
        s.synchronize()


def exchange_buffers(plan: Plan, device):
    """Device exchange buffers of a plan: (int64 tensor or None, float64 tensor)."""
    import torch
    n_int, n_real = cv_plan_exchange_size(plan)
    ex_int = torch.zeros(n_int, dtype=torch.int64, device=device) if n_int else None
    ex_real = torch.zeros(n_real, dtype=torch.float64, device=device)
    return ex_int, ex_real


def sharded_products(plan: Plan, X, Y, flags: int, ddof: int, XTX=None, XTY=None, mean_out=None, std_out=None,
                     group=None, stream=None, buffers: Optional[tuple] = None):
    """One sharded cv_products: partial total, the sum over the group, then the
    shard's folds.  Outputs hold the plan's folds (plan.folds_out)."""
    ex_int, ex_real = buffers if buffers is not None else exchange_buffers(plan, X.device)
    cv_products_partial(plan, X, Y, ex_int, ex_real, stream)
    allreduce_exchange(ex_int, ex_real, group, stream)
    cv_finalize_total(plan, ex_int, ex_real, flags, ddof, XTX, XTY, mean_out, std_out, stream)


def output_tensors(plan: Plan, device, dtype, with_stats: bool = False):
    """Output tensors of the plan's folds: (XTX, XTY[, mean, std])."""
    import torch
    F, K, M = plan.folds_out, plan.K, plan.M
    out = [torch.empty(xtx_shape(plan), dtype=dtype, device=device),
           torch.empty((F, K, M), dtype=dtype, device=device) if M > 0 else None]
    if with_stats:
        out += [torch.empty((F, K + M), dtype=torch.float64, device=device) for _ in range(2)]
    return tuple(out)
