"""Host logic of the multi-GPU runs, on the CPU: the path has no exchange step,
so N GPUs run N independent replicas; the benchmark's only collectives are a
barrier and the max over the ranks of the timed region.  Here two gloo ranks
exercise that reduction, and the reference arm's rule that only rank 0 works.
"""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")  # rank 1 is the slower replica
    q.put((rank, t, bench.job_value(world, 60, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, v in res:
        assert t == 15.0  # both ranks see the max
        assert abs(v - 2 * 60 / 0.015) < 1e-6  # frames of both replicas over the slowest time
    del torch


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_value(1, 30, 1000.0) == 30.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(gpus=2, steps=3, warmup=3)
    out = io.StringIO()
    with redirect_stdout(out):
        bench.reference_arm(args)  # returns at once: no workload built, nothing printed
    assert out.getvalue() == ""
