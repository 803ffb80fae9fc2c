"""The multi-GPU form is replicas only: every rank simulates its own copy of
the workload and the bench reports all ranks' transitions over the slowest
rank's time.  The host-side reduction runs here as two gloo ranks on the
CPU; the reference arm runs on rank 0 alone."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.replica_reduce(10.0 + 5 * rank, "max", "cpu")      # slowest rank's time
        out = bench.replica_reduce(1000 + rank, "sum", "cpu")         # all ranks' transitions
        results[rank] = (ms, out)
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(results) == {0: (15.0, 2001.0), 1: (15.0, 2001.0)}


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.replica_reduce(3.5, "max", "cpu") == 3.5
    assert bench.replica_reduce(7, "sum", "cpu") == 7.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.main() == 0
    assert buf.getvalue() == ""
