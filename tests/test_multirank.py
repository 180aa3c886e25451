"""Multi-process host logic of bench.py, on CPU with the gloo backend and
world size 2 (one process per GPU on a real node): the job's step time is the
slowest rank's, the reported throughput counts every replica (weak scaling,
no collective on the data path), and the reference arm works on rank 0 only.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)    # rank 1 is the slow one
        out[rank] = (ms, bench.job_throughput(world, 1000, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_throughput():
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(2 * 2 * 1000 / 15e-3)


def test_single_rank_is_plain():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_throughput(1, 4_000_000, 10.0) == pytest.approx(8e8)


def test_reference_arm_only_on_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench
    class A:
        n, steps, warmup, gpus = 1000, 1, 1, 2
    assert bench.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""
