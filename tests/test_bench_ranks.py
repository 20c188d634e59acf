"""The multi-rank bookkeeping of bench.py on two gloo ranks (CPU): every rank
reports the slowest rank's times, and the whole-job rate counts the units of
all ranks over that time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_ms, e2e_ms = bench.max_over_ranks(torch, dist, [100.0 + 50.0 * rank, 300.0 - 20.0 * rank], "cpu")
        out[rank] = (t_ms, e2e_ms, bench.whole_job_rate(5, world, t_ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t_ms, e2e_ms, rate = out[rank]
        assert t_ms == 150.0 and e2e_ms == 300.0
        assert rate == pytest.approx(5 * 2 / 0.150)


def test_one_rank_is_unchanged():
    assert bench.max_over_ranks(torch, None, [12.5, 3.0], "cpu") == [12.5, 3.0]
    assert bench.whole_job_rate(5, 1, 500.0) == pytest.approx(10.0)
