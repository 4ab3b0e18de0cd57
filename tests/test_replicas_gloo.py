"""bench.py's multi-GPU mode runs independent replicas (the sweep is not sharded across GPUs);
the job time is the slowest rank's and the job throughput counts every rank's work.  Checked
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 17.0][rank]
    m = bench.max_over_ranks(ms)
    out[rank] = (m, bench.job_throughput(world, 1000, 10, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_slowest_time_and_total_work():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        m, v = out[r]
        assert m == 17.0
        assert abs(v - 2 * 1000 * 10 / 0.017) < 1e-6 * v


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
