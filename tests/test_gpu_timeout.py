"""Failure detection inside the tensor-core kernels, without a GPU fault.
Every wait of the conversion and contraction kernels (an operand copy, an
MMA commit, a drained accumulator) is bounded by the plan's wait limit.  A
plan whose limit is 1 ns makes waits run out (a bulk copy or an MMA takes far
longer), so the kernels stop early: each CTA's producer waits for the copies
it already issued, the MMA thread for its last commit, the CTA frees its
tensor memory and records the timeout, and cv_plan_status returns
CV_ERR_TIMEOUT.  The context stays usable: the same plan times out again, and
a plan with the default limit then gives the oracle's results."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import rel_fro_per_fold

pytestmark = pytest.mark.gpu
TIMEOUT = 8   # CV_ERR_TIMEOUT


@pytest.mark.parametrize("prec", ["fp16x3", "tf32"])
def test_tiny_wait_limit_times_out_and_the_context_recovers(prec):
    pr = workloads.random_case(61, 20000, 100, 4, 5, dtype=np.float32, scheme="random")
    dev = torch.device("cuda:0")
    X, Y, f = (torch.from_numpy(a).to(dev) for a in (pr.X, pr.Y, pr.folds))
    tiny = cvx.cv_plan_ex(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, prec, {"wait_limit_ns": 1})
    for _ in range(2):
        cvx.products(X, Y, f, pr.P, 15, 1, plan=tiny)
        assert cvx.cv_plan_status(tiny) == TIMEOUT
    assert cvx.cv_plan_status(tiny) == 0          # reading the status clears it
    xtx, xty = cvx.products(X, Y, f, pr.P, 15, 1, prec)
    torch.cuda.synchronize()
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, 15, 1)
    tol = 2e-6 if prec == "fp16x3" else 2e-3
    assert rel_fro_per_fold(xtx.cpu().numpy(), o[0]) <= tol
    assert rel_fro_per_fold(xty.cpu().numpy(), o[1]) <= tol
