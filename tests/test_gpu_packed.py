"""The packed upper-triangular X^T X layout (plan option CV_XTX_PACKED_UPPER):
each fold's entries (i, j), i <= j, row by row, K (K + 1) / 2 values.  For
every epilogue the library has (the split path's fused fold-sum epilogue,
the general epilogue of the split and FP64 paths, and the small-fold
recomputation) the packed values must be bitwise the upper triangle of the
full layout from an otherwise identical plan, X^T Y and the statistics
unchanged, and both must match the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import rel_fro_per_fold

pytestmark = pytest.mark.gpu
TOLS = {"fp64": 1e-12, "fp16x3": 2e-6}


def _unpack(packed, K):
    iu = np.triu_indices(K)
    full = np.zeros((packed.shape[0], K, K))
    full[:, iu[0], iu[1]] = packed
    full[:, iu[1], iu[0]] = packed
    return full


@pytest.mark.parametrize("prec,N,K,M,P,out_dtype", [
    ("fp16x3", 4000, 140, 3, 6, torch.float64),     # fused fold-sum epilogue (P <= 32)
    ("fp16x3", 5000, 70, 2, 40, torch.float64),     # general split epilogue (P > 32)
    ("fp64", 3000, 90, 4, 5, torch.float64),        # FP64 epilogue
    ("fp16x3", 1200, 45, 2, 300, torch.float32),    # small-fold recomputation, FP32 outputs
    ("fp64", 900, 37, 1, 150, torch.float64),       # small-fold recomputation, FP64 path
])
def test_packed_is_the_upper_triangle_of_full(prec, N, K, M, P, out_dtype):
    pr = workloads.random_case(81 + P, N, K, M, P, dtype=np.float32, scheme="random", offset=5.0)
    dev = torch.device("cuda:0")
    X, Y, f = (torch.from_numpy(a).to(dev) for a in (pr.X, pr.Y, pr.folds))
    full_plan = cvx.cv_plan(N, K, M, P, f, torch.float32, out_dtype, prec)
    packed_plan = cvx.cv_plan_ex(N, K, M, P, f, torch.float32, out_dtype, prec,
                                 {"xtx_layout": cvx.CV_XTX_PACKED_UPPER})
    assert cvx.xtx_shape(packed_plan) == (P, K * (K + 1) // 2)
    iu = np.triu_indices(K)
    for flags in (15, 5, 0):
        full = cvx.products(X, Y, f, P, flags, 1, prec, out_dtype, plan=full_plan, with_stats=True)
        packed = cvx.products(X, Y, f, P, flags, 1, prec, out_dtype, plan=packed_plan, with_stats=True)
        assert cvx.cv_plan_status(full_plan) == 0 and cvx.cv_plan_status(packed_plan) == 0
        a = full[0].cpu().numpy()
        b = packed[0].cpu().numpy()
        assert np.array_equal(a[:, iu[0], iu[1]], b), (prec, flags)
        for u, v in zip(full[1:], packed[1:]):
            assert torch.equal(u, v)
        o = oracle.naive(pr.X, pr.Y, pr.folds, P, flags, 1)
        tol = TOLS[prec] + (1e-6 if out_dtype == torch.float32 else 0.0)   # FP32 outputs: one more rounding
        assert rel_fro_per_fold(_unpack(b.astype(np.float64), K), o[0]) <= tol
