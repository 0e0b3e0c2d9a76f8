"""Multi-process host logic of `bench.py --gpus N` on CPU (gloo, world size 2):
the job step time is the maximum over ranks and the job throughput is the sum
of the units all ranks processed over that time (replicas, weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [1.5, 2.5][rank]
        units = [1000, 3000][rank]
        val, ms_job = bench.job_throughput(dist, ms, units, "cpu")
        dist.barrier()
        out[rank] = (val, ms_job)
    finally:
        dist.destroy_process_group()


def test_job_throughput_two_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        val, ms_job = out[r]
        assert ms_job == 2.5
        assert val == pytest.approx(4000 / 2.5e-3)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    val, ms = bench.job_throughput(None, 2.0, 500, "cpu")
    assert ms == 2.0 and val == pytest.approx(500 / 2e-3)
