"""The multi-rank path of bench.py (replicas: every rank solves its own problem, no data
exchange): job time = maximum over ranks, job throughput = ranks x DoF / job time.  Run as
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.job_time_ms(10.0 + 5.0 * rank, torch.device("cpu"))
    out[rank] = (ms, bench.job_value(1_000_000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
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
        ms, value = out[r]
        assert ms == 15.0
        assert abs(value - 2 * 1_000_000 / 15e-3 / 1e9) < 1e-12


def test_single_rank_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, torch.device("cpu")) == 7.5
    assert abs(bench.job_value(8_291_838, 1, 161.0) - 8_291_838 / 0.161 / 1e9) < 1e-12
