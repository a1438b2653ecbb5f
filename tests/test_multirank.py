"""The bench's multi-GPU path is replicas only: every rank solves its own
copy of the workload and the only collective is the max-over-ranks of the
timed region.  That aggregation runs here on two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    T = bench.job_seconds(1.0 + rank, world, "cpu")          # rank 1 is the slow one
    out[rank] = (T, bench.job_throughput(12, 3, world, T))
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_throughput_counts_all_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, PORT, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        T, v = out[r]
        assert T == 2.0
        assert v == pytest.approx(12 * 3 * 2 / 2.0)


PORT = _free_port()
