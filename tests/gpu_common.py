"""Shared helpers of the GPU parity tests (no test functions here)."""
import numpy as np
import torch

import paper_2401_13185_gb300 as cvx


def run_library(pr, flags, ddof, prec, out_dtype=torch.float64, folds_on_device=True, plan=None):
    """Run the CUDA path on a workloads.Problem; returns numpy (xtx, xty, mean, std)."""
    dev = torch.device("cuda:0")
    X = torch.from_numpy(np.ascontiguousarray(pr.X)).to(dev)
    Y = torch.from_numpy(np.ascontiguousarray(pr.Y)).to(dev) if pr.M > 0 else None
    folds = torch.from_numpy(pr.folds).to(dev) if folds_on_device else pr.folds
    if plan is None:
        plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, folds, X.dtype, out_dtype, prec)
    xtx, xty, mean, std = cvx.products(X, Y, folds, pr.P, flags, ddof, prec, out_dtype,
                                       plan=plan, with_stats=True)
    status = cvx.cv_plan_status(plan)
    assert status == 0, cvx.cv_status_string(status)
    torch.cuda.synchronize()
    xty_np = xty.double().cpu().numpy() if xty is not None else np.zeros((pr.P, pr.K, 0))
    return xtx.double().cpu().numpy(), xty_np, mean.cpu().numpy(), std.cpu().numpy()


def rel_fro_per_fold(R, O):
    """max over folds of ||R_p - O_p||_F / ||O_p||_F (0 when both vanish)."""
    errs = []
    for p in range(O.shape[0]):
        d = np.linalg.norm((R[p] - O[p]).ravel())
        n = np.linalg.norm(O[p].ravel())
        errs.append(0.0 if d == 0 else d / max(n, 1e-300))
    return max(errs) if errs else 0.0


def corr_scale_error(R, O):
    """max_ij |R - O| / sqrt(|O_ii| |O_jj|) for X^T X (per fold): an error on the
    correlation scale, which the Frobenius norm would hide for small columns."""
    worst = 0.0
    for p in range(O.shape[0]):
        d = np.sqrt(np.abs(np.diag(O[p])))
        den = np.outer(d, d)
        mask = den > 0
        if mask.any():
            worst = max(worst, float((np.abs(R[p] - O[p])[mask] / den[mask]).max()))
    return worst
