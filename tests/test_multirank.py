"""Host logic of the N > 1 bench path on CPU (gloo, world size 2): the job's
time is the maximum over ranks, the whole-job value counts every replica,
and only rank 0 prints."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")
    dist.barrier()
    out[rank] = ms
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    import bench
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = dict(out)
    assert got == {0: 150.0, 1: 150.0}
    # two replicas, each one step per 15 ms -> 133.3 steps/s for the job
    assert bench.job_value(world, 15.0) == pytest.approx(2 * 1000.0 / 15.0)
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
