"""Multi-GPU is replicas only: every rank sorts its own data and the job's throughput is all
ranks' records over the slowest rank's time.  The aggregation runs here on two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]  # rank 1 is the slower one
        m = bench.max_over_ranks(local_ms, dist, "cpu")
        v = bench.replica_throughput(1000, world, 5, m)
        dist.barrier()
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[1] for g in got] == [150.0, 150.0]
    assert all(g[2] == pytest.approx(1000 * 2 * 5 / 0.150) for g in got)


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.replica_throughput(10, 1, 2, 1000.0) == pytest.approx(20.0)
