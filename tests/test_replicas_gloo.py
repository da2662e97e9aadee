"""The N > 1 path is replicas only: every rank runs the whole workload and the
job's time is the slowest rank's.  Checked with two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_s = 0.010 * (rank + 1)  # rank 1 is the slow one
    t = bench.max_over_ranks(step_s, dist, "cpu")
    out[rank] = (t, bench.job_throughput(1000.0, t, world))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_replica_sets_the_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, rate = out[r]
        assert t == pytest.approx(0.020)
        assert rate == pytest.approx(2 * 1000.0 / 0.020)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(0.5) == 0.5
    assert bench.job_throughput(10.0, 2.0, 1) == 5.0
