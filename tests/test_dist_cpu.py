"""The multi-rank bench path (independent replicas, one per GPU) reduces only timings: each
rank's total, the slowest rank's time and the whole-job throughput. Checked with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 100.0 + 25.0 * rank  # per-rank timed total, ms
    out[rank] = bench.max_over_ranks(mine, torch.device("cpu"))
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 125.0
    import bench
    assert bench.job_throughput(world, 10, 125.0) == pytest.approx(160.0)
    assert bench.max_over_ranks(7.0, torch.device("cpu")) == 7.0  # not initialized
