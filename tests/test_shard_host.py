"""Host side of fold sharding, without a GPU: which folds each rank owns, and
the all-reduce of the exchange buffers over a gloo process group of two CPU
ranks.  Each rank contributes the Gram of W = [X | Y | 1] over the rows of
its own folds; after the all-reduce both ranks hold the Gram over all rows
(Lemma 2: the folds' validation Grams sum to X^T X), exactly for integer data
in the int64 buffer and to rounding in the float64 buffer."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2401_13185_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("P", [2, 3, 5, 10, 17, 20, 64])
def test_owned_folds_partition_the_folds(P):
    for world in range(1, min(P, 9) + 1):
        ranges = [shard.owned_folds(P, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == P
        for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
            assert e0 == b1
        sizes = [e - b for b, e in ranges]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.owned_folds(3, 4, 0)
    with pytest.raises(ValueError):
        shard.owned_folds(3, 2, 2)


def test_shard_options_carry_the_range():
    o = shard.shard_options(20, 3, 1, ctas=100, xtx_layout=1)
    assert (o.fold_begin, o.fold_end, o.strategy, o.ctas, o.xtx_layout, o.reserved) == (7, 14, 1, 100, 1, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    rng = np.random.default_rng(2401)
    N, K, M, P = 203, 6, 2, 5
    Xi = rng.integers(-50, 50, size=(N, K + M))          # integer data: exact int64 Grams
    Xf = rng.standard_normal((N, K + M)) * 3.0 + 7.0
    folds = np.repeat(np.arange(P), -(-N // P))[:N]
    rng.shuffle(folds)
    return Xi, Xf, folds.astype(np.int32), P


def _gram(A):
    W = np.concatenate([A, np.ones((A.shape[0], 1), A.dtype)], axis=1)
    return W.T @ W


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2401_13185_gb300 import shard as sh
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        Xi, Xf, folds, P = _problem()
        b, e = sh.owned_folds(P, world, rank)
        mine = (folds >= b) & (folds < e)
        ex_int = torch.from_numpy(_gram(Xi[mine]).astype(np.int64).ravel().copy())
        ex_real = torch.from_numpy(_gram(Xf[mine]).ravel().copy())
        sh.allreduce_exchange(ex_int, ex_real)
        out[rank] = (ex_int.numpy().copy(), ex_real.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_gram_over_all_rows():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    Xi, Xf, folds, P = _problem()
    want_i = _gram(Xi).astype(np.int64).ravel()
    want_f = _gram(Xf).ravel()
    for r in range(world):
        assert np.array_equal(res[r][0], want_i)
        np.testing.assert_allclose(res[r][1], want_f, rtol=1e-12)
