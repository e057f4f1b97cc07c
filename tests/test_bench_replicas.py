"""The multi-GPU path of the bench is replicas only: each rank advances its
own copy and the job's time is the MAX over ranks.  The host logic runs here
as world-size-2 gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.reduce_job_time(times[rank], world, "cpu")
        out[rank] = (t, bench.job_value(1000, 20, world, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        times = [12.5, 40.0]
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(120)
            assert pr.exitcode == 0
        for r in range(2):
            t, v = out[r]
            assert t == 40.0
            assert v == pytest.approx(2 * 1000 * 20 / 0.040)


def test_single_rank_value():
    import bench
    assert bench.reduce_job_time(7.0, 1, "cpu") == 7.0
    assert bench.job_value(4198401, 1000, 1, 213.0) == pytest.approx(4198401 * 1000 / 0.213)
