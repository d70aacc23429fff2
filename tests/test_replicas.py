"""bench.py's N > 1 path (independent replicas, no data-path collective): the
whole-job time is the slowest rank's and the units are summed, checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
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
    ms, units = bench.job_totals(100.0 + 50.0 * rank, 1000.0 * (rank + 1), world)
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_max_time_and_sum_units():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (150.0, 3000.0)


def test_single_rank_passthrough():
    import bench
    assert bench.job_totals(12.5, 7.0, 1) == (12.5, 7.0)
