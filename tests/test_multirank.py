"""The multi-GPU path of bench.py without GPUs: ranks are replicas; the only
exchange is the max-over-ranks duration and the sum of processed units,
checked with two gloo ranks on the CPU.  The reference arm runs on rank 0
only.  A rank that dies between steps makes the survivor's next exchange
raise instead of hang (failure detection on the host)."""
import datetime
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, units, value = bench.job_throughput(10.0 * (rank + 1), 64, world)
    out.put((rank, ms, units, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_units():
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
    for rank, ms, units, value in res:
        assert ms == 20.0 and units == 128.0
        assert value == pytest.approx(128 / 0.020)


def _rank_dies(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)        # leaves between steps: nothing of it in flight
    try:
        bench.job_throughput(10.0, 64, world)
        out.put((rank, "returned"))
    except Exception as exc:   # the gloo error type differs between torch versions
        out.put((rank, type(exc).__name__))


def test_a_rank_that_dies_ends_the_next_exchange_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what != "returned"
    assert procs[1].exitcode == 3


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(8.0, 64, 1) == (8.0, 64.0, 8000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
