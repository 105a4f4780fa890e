"""The benchmark's multi-rank path on the CPU (gloo, world size 2).

Rendering shards by frames with no collective on the data path: every rank
renders its own frame and the job reports the units of all ranks over the
slowest rank's time.  These tests run that host logic with two gloo ranks,
and check that under torchrun the reference arm runs on rank 0 alone.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as td

    import bench
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, device="cpu")      # rank 1 is the slow one
        out.put((rank, t, bench.job_rate(1000, world, t)))
    finally:
        td.destroy_process_group()


def test_two_rank_job_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the rate counts both ranks' units
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(abs(r[2] - 2 * 1000 / 2.5) < 1e-9 for r in res)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda a: called.append(a))
    bench.main()
    assert called == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.main()
    assert len(called) == 1
