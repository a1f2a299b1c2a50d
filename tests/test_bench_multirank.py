"""bench.py's multi-rank host logic with world_size 2 on CPU (gloo): the timing
is the max over ranks and the job value counts every rank's replica."""

from __future__ import annotations

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [1.5, 4.25][rank]                     # the slower rank decides
    t = bench.reduce_max(local, dist, "cpu")
    out.put((rank, t, bench.job_throughput(1000, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [4.25, 4.25]
    assert res[0][2] == pytest.approx(2000 / 4.25)


def test_single_process_defaults():
    import bench
    assert bench.reduce_max(3.0) == 3.0
    assert bench.job_throughput(400000, 1, 5.0) == 80000.0
