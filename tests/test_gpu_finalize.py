"""cv_finalize: re-running only the statistics and the epilogue for other
flags and ddof from the fold sums of one cv_products call (Section 6 /
Table 1: the 16 combinations differ only in the corrections of Propositions
15 and 16).  The results must be bitwise those of a full cv_products call
with the same flags, for every precision and for the small-fold strategy,
and must match the CPU oracle (Algorithms 2/4/6) element by element within
each precision's parity tolerance (derived in test_gpu_split.py and
test_gpu_precisions.py)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import corr_scale_error, rel_fro_per_fold
from test_gpu_fp64 import xty_reference_flags

pytestmark = pytest.mark.gpu
TOLS = {"fp64": 1e-12, "fp16x3": 2e-6, "bf16x3": 5e-5, "tf32x3": 5e-5, "tf32": 2e-3}


def _outputs(pr, dev):
    return (torch.full((pr.P, pr.K, pr.K), np.nan, dtype=torch.float64, device=dev),
            torch.full((pr.P, pr.K, pr.M), np.nan, dtype=torch.float64, device=dev),
            torch.zeros((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev),
            torch.zeros((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev))


@pytest.mark.parametrize("prec,N,P", [("fp64", 3000, 7), ("fp16x3", 3000, 7), ("bf16x3", 3000, 7),
                                      ("tf32", 3000, 7), ("tf32x3", 3000, 7), ("fp16x3", 1200, 300),
                                      ("fp64", 1200, 300)])
def test_finalize_matches_products_bitwise(prec, N, P):
    pr = workloads.random_case(31, N, 45, 3, P, dtype=np.float32, scheme="random")
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, prec)
    ref_plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, prec)
    a = _outputs(pr, dev)
    cvx.cv_products(plan, X, Y, 0, 1, *a)
    for ddof in (0, 1):
        for flags in range(16):
            got = _outputs(pr, dev)
            # the inputs again: small-fold plans read them, the others ignore them
            cvx.cv_finalize(plan, flags, ddof, *got, X=X, Y=Y)
            ref = _outputs(pr, dev)
            cvx.cv_products(ref_plan, X, Y, flags, ddof, *ref)
            torch.cuda.synchronize()
            for g, r in zip(got, ref):
                assert torch.equal(g, r), (prec, flags, ddof)
            # and against the oracle
            tol = TOLS[prec]
            o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, ddof)
            oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), ddof)[1]
            xtx, xty = got[0].cpu().numpy(), got[1].cpu().numpy()
            e = (rel_fro_per_fold(xtx, o[0]), rel_fro_per_fold(xty, oy), corr_scale_error(xtx, o[0]))
            assert max(e) <= tol, (prec, N, P, flags, ddof, e)
            np.testing.assert_allclose(got[3].cpu().numpy(), o[3], rtol=max(tol, 1e-12))
    assert cvx.cv_plan_status(plan) == 0 and cvx.cv_plan_status(ref_plan) == 0


def test_finalize_needs_products_first():
    pr = workloads.random_case(32, 500, 5, 1, 4, dtype=np.float32)
    dev = torch.device("cuda:0")
    f = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, "fp16x3")
    out = _outputs(pr, dev)
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_finalize(plan, 15, 1, *out)
    assert e.value.name == "CV_ERR_INVALID_ARG"


def test_finalize_small_folds_needs_inputs():
    pr = workloads.random_case(33, 600, 5, 1, 60, dtype=np.float32)   # folds of 10 rows
    dev = torch.device("cuda:0")
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    f = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, f, torch.float32, torch.float64, "fp16x3")
    out = _outputs(pr, dev)
    cvx.cv_products(plan, X, Y, 15, 1, *out)
    with pytest.raises(cvx.CVError) as e:
        cvx.cv_finalize(plan, 5, 1, *out)
    assert e.value.name == "CV_ERR_INVALID_ARG"
