"""The multi-rank arithmetic of bench.py, on CPU: two gloo ranks (the same
calls a torchrun launch makes over NCCL).  Each rank advances its own replica,
so a job's time is its slowest rank's and its rate counts every rank's cells."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [0.5, 2.0][rank]               # rank 1 is the slow one
        worst = bench.max_over_ranks(secs)
        rate = bench.job_rate(1000.0, secs, world)
        out.put((rank, worst, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_every_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, rate in got:
        assert worst == 2.0                   # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.job_rate(300.0, 1.5, 1) == pytest.approx(200.0)
