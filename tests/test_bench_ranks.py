"""The multi-GPU path of bench.py is replicas: each rank runs the step on its
own GPU and the ranks only combine their timings.  Checked here with two gloo
ranks on the CPU: every rank sees the slowest rank's duration and the sum of
the ranks' work, and the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, units = bench.combine_over_ranks(10.0 + rank, 100 * (rank + 1), world, device="cpu")
        q.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_total_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(7.5, 42, 1) == (7.5, 42)


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference(bench.argparse.Namespace(n=1 << 10, degree=4, steps=1, warmup=0))
    assert buf.getvalue() == ""
