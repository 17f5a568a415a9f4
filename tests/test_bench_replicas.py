"""Whole-job aggregation of bench.py's replica runs (one process per GPU, weak scaling): the job
time is the slowest rank's and the throughput counts every rank's units.  Run as two gloo ranks on
CPU; the same functions run over NCCL in a multi-GPU bench."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]
        value, job_ms = bench.job_throughput(1000, ms)
        q.put((rank, value, job_ms, bench.max_over_ranks(float(rank + 7))))
    finally:
        dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, job_ms, mx in out:
        assert job_ms == 150.0                          # the slower replica sets the job time
        assert value == pytest.approx(2 * 1000 / 0.150)  # both replicas' units
        assert mx == 8.0


def test_single_process_aggregation_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    value, ms = bench.job_throughput(500, 250.0)
    assert ms == 250.0 and value == pytest.approx(2000.0)
