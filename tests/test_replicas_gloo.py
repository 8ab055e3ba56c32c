"""Multi-process (world size 2, gloo, CPU) check of the replica aggregation used
by bench.py --gpus N: the job time is the maximum over ranks and the job
throughput counts every rank's independent solves. The method's unit of work
(one solve) has no exchange step, so this max-reduction is the only collective."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [12.5, 40.0][rank]
    ms = bench.max_over_ranks(ms_local, world, "cpu")
    out[rank] = (ms, bench.job_throughput(1000, 4, world, ms))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, thr = out[r]
        assert ms == 40.0
        assert abs(thr - 1000 * 4 * 2 / 0.040) < 1e-6
