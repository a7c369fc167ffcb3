"""Multi-rank path of the benchmark (independent replicas, one per rank, no
data-path collective): the slowest rank's time sets the whole-job throughput.
Run as two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]             # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, "cpu")
    value = bench.whole_job_throughput(1000, 100, 5, world, ms)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 180.0
        assert abs(value - 1000 * 100 * 5 * 2 / 0.18) < 1e-6 * value


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_throughput(10, 10, 1, 1, 1000.0) == 100.0
