"""Batches of independent problems (cv_batch_* / cv_products_batched).

Graph batches (FP64, or anything not eligible for batched launches) run each
problem's own cv_products.  Batched launches (split precisions, FP32 inputs,
P <= 32) plan every problem with the fold-grouped strategy and its share of
the SMs, and run the same per-element arithmetic.  Either way every problem is
bitwise equal to a single plan made with the options cv_batch_plan_options
reports, and everything is checked against the oracle within the precision's
tolerance."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_13185_gb300 as cvx
import workloads
from gpu_common import rel_fro_per_fold
from test_gpu_fp64 import xty_reference_flags

pytestmark = pytest.mark.gpu
TOLS = {"fp64": 1e-12, "fp16x3": 2e-6, "bf16x3": 5e-5, "tf32": 2e-3}


def _problems(seed, count, dtype=np.float32):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        N = int(rng.integers(200, 3000))
        K = int(rng.integers(4, 200))
        M = int(rng.integers(0, 6))
        P = int(rng.choice([2, 5, 10, 20]))
        scheme = ["random", "contiguous", "venetian", "unbalanced"][b % 4]
        pr = workloads.random_case(int(seed * 1000 + b), N, K, M, P, dtype=dtype, scheme=scheme,
                                   flags=int(rng.integers(0, 16)))
        out.append(pr)
    return out


def _device_problem(pr, dev, out_dtype=torch.float64):
    d = {"X": torch.from_numpy(pr.X).to(dev),
         "Y": torch.from_numpy(pr.Y).to(dev) if pr.M else None,
         "folds": torch.from_numpy(pr.folds).to(dev), "P": pr.P, "flags": pr.flags, "ddof": pr.ddof,
         "XTX": torch.full((pr.P, pr.K, pr.K), np.nan, dtype=out_dtype, device=dev),
         "XTY": torch.full((pr.P, pr.K, pr.M), np.nan, dtype=out_dtype, device=dev) if pr.M else None,
         "mean": torch.zeros((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev),
         "std": torch.zeros((pr.P, pr.K + pr.M), dtype=torch.float64, device=dev)}
    return d


def _single(pr, d, prec, options=None):
    plan = cvx.cv_plan_ex(pr.N, pr.K, pr.M, pr.P, d["folds"], d["X"].dtype, d["XTX"].dtype, prec, options)
    xtx = torch.empty_like(d["XTX"])
    xty = torch.empty_like(d["XTY"]) if pr.M else None
    cvx.cv_products(plan, d["X"], d["Y"], d["flags"], d["ddof"], xtx, xty)
    assert cvx.cv_plan_status(plan) == 0
    return xtx, xty


def _oracle_check(pr, d, prec, flags):
    o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, flags, pr.ddof)
    tol = TOLS[prec]
    assert rel_fro_per_fold(d["XTX"].cpu().numpy(), o[0]) <= tol, (pr.name, prec, flags)
    if pr.M:
        oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(flags), pr.ddof)[1]
        assert rel_fro_per_fold(d["XTY"].cpu().numpy(), oy) <= tol, (pr.name, prec, flags)
    if prec in ("fp64", "fp16x3"):
        np.testing.assert_allclose(d["mean"].cpu().numpy(), o[2], rtol=1e-7, atol=1e-7 * np.abs(o[2]).max())
    else:   # FP32-accumulated column sums: the error in units of the column's spread
        assert np.max(np.abs(d["mean"].cpu().numpy() - o[2]) / o[3]) <= tol, (pr.name, prec, "mean")


@pytest.mark.parametrize("prec", ["fp16x3", "fp64", "bf16x3", "tf32"])
def test_batch_matches_single_plans_and_oracle(prec):
    dev = torch.device("cuda:0")
    # twelve random problems and two whose folds average at most 64 rows
    prs = _problems(3, 12) + [workloads.random_case(31, 600, 50, 2, 20, dtype=np.float32, flags=15),
                              workloads.random_case(32, 300, 130, 0, 10, dtype=np.float32, scheme="venetian",
                                                    flags=5)]
    ds = [_device_problem(pr, dev) for pr in prs]
    batch = cvx.cv_batch_plan(ds, torch.float32, torch.float64, prec)
    batched = prec != "fp64"
    assert cvx.cv_batch_launches(batch) == (0, batched)
    per_call = None
    for rep in range(2):   # first call (capture or argument upload), then a repeat
        for d in ds:
            d["XTX"].fill_(np.nan)
        cvx.cv_batch_products(batch, ds)
        assert cvx.cv_batch_status(batch) == 0
        n, _ = cvx.cv_batch_launches(batch)
        per_call = n if per_call is None else per_call
        assert n == per_call * (rep + 1)
        for i, (pr, d) in enumerate(zip(prs, ds)):
            opts = cvx.cv_batch_plan_options(batch, i)
            assert opts[0] == (cvx.CV_STRATEGY_FOLD_GROUPED if batched else cvx.CV_STRATEGY_AUTO)
            assert (opts[1] >= 1) if batched else (opts[1] == 0)
            xtx, xty = _single(pr, d, prec, opts)
            assert torch.equal(xtx, d["XTX"]), (pr.name, rep)
            if pr.M:
                assert torch.equal(xty, d["XTY"]), (pr.name, rep)
    if batched:   # four stages plus one epilogue launch per class of fold counts
        assert per_call == 4 + len({0 if pr.P <= 8 else (1 if pr.P <= 16 else 2) for pr in prs})
    for pr, d in zip(prs, ds):
        _oracle_check(pr, d, prec, pr.flags)
    # new flags for every problem: the graph is captured again (in-place update)
    for d in ds:
        d["flags"] = (d["flags"] + 5) % 16
    cvx.cv_batch_products(batch, ds)
    assert cvx.cv_batch_status(batch) == 0
    for pr, d in zip(prs[:4], ds[:4]):
        _oracle_check(pr, d, prec, d["flags"])
    cvx.cv_batch_destroy(batch)


def test_batch_many_small_folds_and_float32_output():
    """Batched launches with folds of a few rows (planned fold-grouped, so one
    segment per fold) and FP32 outputs."""
    dev = torch.device("cuda:0")
    prs = [workloads.random_case(700 + b, N, K, M, P, dtype=np.float32, scheme=sch, flags=fl)
           for b, (N, K, M, P, sch, fl) in enumerate([(96, 40, 2, 32, "venetian", 15), (257, 130, 3, 31, "random", 5),
                                                     (64, 3, 1, 32, "contiguous", 0), (2000, 300, 0, 7, "unbalanced", 1)])]
    ds = [_device_problem(pr, dev, torch.float32) for pr in prs]
    batch = cvx.cv_batch_plan(ds, torch.float32, torch.float32, "fp16x3")
    assert cvx.cv_batch_launches(batch)[1]
    cvx.cv_batch_products(batch, ds)
    assert cvx.cv_batch_status(batch) == 0
    for pr, d in zip(prs, ds):
        o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, pr.flags, pr.ddof)
        assert rel_fro_per_fold(d["XTX"].double().cpu().numpy(), o[0]) <= 2e-6, pr.name
        if pr.M:
            oy = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, xty_reference_flags(pr.flags), pr.ddof)[1]
            assert rel_fro_per_fold(d["XTY"].double().cpu().numpy(), oy) <= 2e-6, pr.name
        assert torch.equal(d["XTX"], d["XTX"].transpose(1, 2))


def test_batch_with_many_folds_uses_graph():
    """A problem with more than 32 folds keeps the whole batch on the graph path."""
    dev = torch.device("cuda:0")
    prs = [workloads.random_case(40, 3000, 20, 2, 40, dtype=np.float32),
           workloads.random_case(41, 1000, 10, 1, 5, dtype=np.float32)]
    ds = [_device_problem(pr, dev) for pr in prs]
    batch = cvx.cv_batch_plan(ds, torch.float32, torch.float64, "fp16x3")
    assert cvx.cv_batch_launches(batch)[1] is False
    cvx.cv_batch_products(batch, ds)
    assert cvx.cv_batch_status(batch) == 0
    for pr, d in zip(prs, ds):
        _oracle_check(pr, d, "fp16x3", pr.flags)


def test_products_batched_one_shot():
    dev = torch.device("cuda:0")
    prs = _problems(4, 6, dtype=np.float64)
    ds = [_device_problem(pr, dev, torch.float32) for pr in prs]
    cvx.cv_products_batched(ds, torch.float64, torch.float32, "fp64")
    for pr, d in zip(prs, ds):
        o = oracle.naive(pr.X, pr.Y, pr.folds, pr.P, pr.flags, pr.ddof)
        assert rel_fro_per_fold(d["XTX"].double().cpu().numpy(), o[0]) <= 2e-7, pr.name


def test_batch_argument_errors():
    dev = torch.device("cuda:0")
    prs = _problems(5, 3)
    ds = [_device_problem(pr, dev) for pr in prs]
    batch = cvx.cv_batch_plan(ds, torch.float32, torch.float64, "fp16x3")
    bad = [dict(d) for d in ds]
    bad[1]["X"] = bad[1]["X"][:, :-1] if prs[1].K > 1 else bad[1]["X"]
    if prs[1].K > 1:
        with pytest.raises(cvx.CVError) as ei:
            cvx.cv_batch_products(batch, bad)
        assert ei.value.name == "CV_ERR_INVALID_ARG"
    bad = [dict(d) for d in ds]
    bad[2]["flags"] = 99
    with pytest.raises(cvx.CVError) as ei:
        cvx.cv_batch_products(batch, bad)
    assert ei.value.name == "CV_ERR_INVALID_ARG"
    # a valid call still works afterwards
    cvx.cv_batch_products(batch, ds)
    assert cvx.cv_batch_status(batch) == 0


def test_batched_launches_can_be_captured_in_a_cuda_graph():
    """A batch of at most 256 problems on the batched launches passes the
    call's arguments as kernel parameters: the call copies nothing and waits
    for nothing on the host, so it can be captured into a CUDA graph.  The
    graph's replays give bitwise the outputs of a direct call with the same
    arguments, also after the outputs were overwritten in between."""
    dev = torch.device("cuda:0")
    prs = _problems(71, 12)
    ds = [_device_problem(pr, dev) for pr in prs]
    batch = cvx.cv_batch_plan(ds, torch.float32, torch.float64, "fp16x3")
    assert cvx.cv_batch_launches(batch)[1]
    cvx.cv_batch_products(batch, ds)
    torch.cuda.synchronize()
    want = [(d["XTX"].clone(), d["XTY"].clone() if d["XTY"] is not None else None) for d in ds]
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cvx.cv_batch_products(batch, ds, stream=s)
    for _ in range(2):
        for d in ds:
            d["XTX"].fill_(float("nan"))
            if d["XTY"] is not None:
                d["XTY"].fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for d, (wx, wy) in zip(ds, want):
            assert torch.equal(d["XTX"], wx)
            if wy is not None:
                assert torch.equal(d["XTY"], wy)
    assert cvx.cv_batch_status(batch) == 0
    cvx.cv_batch_destroy(batch)
