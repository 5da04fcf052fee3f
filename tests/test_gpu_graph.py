"""cv_products inside a CUDA graph: the call enqueues kernels only (no host
synchronisation, no allocation), so it can be captured on a stream and the
graph replayed with new values in the captured input buffers.  Each replay
must give bitwise the outputs and statistics of a direct call on the same
plan, for the fused small-P epilogue, the general epilogue, the small-fold
strategy and the FP64 path."""
import numpy as np
import pytest
import torch

import paper_2401_13185_gb300 as cvx
import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,P", [("fp16x3", 10), ("fp16x3", 40), ("fp16x3", 300), ("fp64", 10),
                                    ("fp64", 300)])
def test_capture_and_replay_match_direct_calls(prec, P):
    N, K, M = 6000, 130, 3
    dev = torch.device("cuda:0")
    prs = [workloads.random_case(900 + s, N, K, M, P, dtype=np.float32, scheme="random", offset=10.0)
           for s in range(3)]
    f = torch.from_numpy(prs[0].folds).to(dev)
    plan = cvx.cv_plan(N, K, M, P, f, torch.float32, torch.float64, prec)
    X = torch.from_numpy(prs[0].X).to(dev)
    Y = torch.from_numpy(prs[0].Y).to(dev)
    outs = [torch.empty((P, K, K), dtype=torch.float64, device=dev),
            torch.empty((P, K, M), dtype=torch.float64, device=dev),
            torch.empty((P, K + M), dtype=torch.float64, device=dev),
            torch.empty((P, K + M), dtype=torch.float64, device=dev)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        cvx.cv_products(plan, X, Y, 15, 1, *outs, stream=s)   # warm-up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cvx.cv_products(plan, X, Y, 15, 1, *outs, stream=s)
    for pr in prs[1:] + prs[:1]:
        X.copy_(torch.from_numpy(pr.X))
        Y.copy_(torch.from_numpy(pr.Y))
        g.replay()
        torch.cuda.synchronize()
        got = [t.clone() for t in outs]
        cvx.cv_products(plan, X, Y, 15, 1, *outs)
        torch.cuda.synchronize()
        assert cvx.cv_plan_status(plan) == 0
        for a, b in zip(got, outs):
            assert torch.equal(a, b), (prec, P)
