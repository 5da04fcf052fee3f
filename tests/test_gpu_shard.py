"""Fold sharding (the paper's Lemma 2: the folds' Grams sum to the Gram over
all rows) on the GPU: two or three processes, each a rank of a gloo process
group, each with a plan that owns a contiguous range of the folds.  Every
rank contracts only its folds' rows, the ranks sum their partial totals once
(over gloo, through host copies of the exchange buffers), and each rank
finishes its folds.  The ranks share the one GPU of the test machine; none
of their kernels waits on another rank's.  Each rank's outputs are compared
element by element with the oracle (Algorithms 2/4/6) for its folds, for
the FP64 path (1e-12) and the split FP16 path (its 2e-6 parity bound), for
the products call and for a cv_finalize with other flags from the same
total.  Not measured on several GPUs: every machine here has one."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu
TOLS = {"fp64": 1e-12, "fp16x3": 2e-6}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rel_fro(R, O):
    worst = 0.0
    for p in range(O.shape[0]):
        n = np.linalg.norm(O[p].ravel())
        d = np.linalg.norm((R[p] - O[p]).ravel())
        worst = max(worst, 0.0 if d == 0 else d / max(n, 1e-300))
    return worst


def _rank(rank, world, port, case, prec, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    import oracle
    import paper_2401_13185_gb300 as cvx
    import workloads
    from paper_2401_13185_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        dev = torch.device("cuda:0")
        seed, N, K, M, P, scheme = case
        pr = workloads.random_case(seed, N, K, M, P, dtype=np.float32, scheme=scheme, offset=20.0)
        X = torch.from_numpy(pr.X).to(dev)
        Y = torch.from_numpy(pr.Y).to(dev) if M > 0 else None
        f = torch.from_numpy(pr.folds).to(dev)
        plan = shard.shard_plan(N, K, M, P, f, world, rank, torch.float32, torch.float64, prec)
        b, e = plan.fold_begin, plan.fold_end
        outs = shard.output_tensors(plan, dev, torch.float64, with_stats=True)
        shard.sharded_products(plan, X, Y, 15, 1, *outs)
        outs0 = shard.output_tensors(plan, dev, torch.float64, with_stats=True)
        cvx.cv_finalize(plan, 0, 0, *outs0)        # other flags and ddof from the same total
        status = cvx.cv_plan_status(plan)
        errs = {}
        for name, o_flags, ddof, got in (("flags15", 15, 1, outs), ("flags0", 0, 0, outs0)):
            o = oracle.naive_subset(pr.X, pr.Y if M > 0 else None, pr.folds, P, o_flags, ddof, list(range(b, e)))
            xtx = got[0].cpu().numpy()
            errs[name + "_xtx"] = _rel_fro(xtx, o[0][b:e])
            if M > 0:
                errs[name + "_xty"] = _rel_fro(got[1].cpu().numpy(), o[1][b:e])
            errs[name + "_std"] = float(np.max(np.abs(got[3].cpu().numpy() / o[3][b:e] - 1.0)))
        out[rank] = (b, e, status, errs)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
@pytest.mark.parametrize("world,case", [
    (2, (71, 6000, 70, 3, 7, "random")),
    (3, (72, 9000, 200, 5, 8, "unbalanced")),   # uneven shards, a narrow last column block
    (2, (73, 3000, 33, 0, 4, "contiguous")),    # M = 0
])
def test_sharded_ranks_match_the_oracle(world, case, prec):
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, prec, out), nprocs=world, join=True)
        res = dict(out)
    P = case[4]
    covered = []
    for r in range(world):
        b, e, status, errs = res[r]
        assert status == 0, (r, status)
        covered += list(range(b, e))
        for k, v in errs.items():
            assert v <= TOLS[prec], (prec, r, k, v)
    assert covered == list(range(P))
