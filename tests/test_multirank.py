"""The multi-process timing of bench.py on CPU: two gloo ranks on 127.0.0.1.
Under torchrun the ranks shard one problem's folds (tests/test_shard_host.py
and tests/test_gpu_shard.py cover the sharding); the job's time is the
slowest rank's and its rate is the problem's work over that time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [1.25, 2.5][rank]
        slowest = bench.max_over_ranks(ms, world, "cpu")
        out[rank] = (slowest, bench.job_tflops(5.1e10, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == pytest.approx(5.1e10 / 2.5e-3 / 1e12)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_tflops(1e12, 1.0) == pytest.approx(1000.0)
