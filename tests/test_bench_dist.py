"""The benchmark's multi-rank logic on CPU: two gloo ranks on 127.0.0.1.
The job time is the slowest rank's (max over ranks), the value the units of
all ranks over it; the reference arm prints from rank 0 only."""
import io
import os
import sys
import contextlib

import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402


def _rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [3.0, 5.0][rank]
    t = bench.max_over_ranks(ms, dist)
    out.put((rank, t, bench.aggregate_rate(1000, 10, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 5.0                                  # the slowest rank's time on every rank
        assert abs(v - 1000 * 10 * 2 / 5e-3) < 1e-6      # all ranks' units over it


def test_single_process_no_group():
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.aggregate_rate(64, 5, 1, 2.0) == 64 * 5 / 2e-3


def test_reference_arm_prints_from_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 1, "warmup": 1, "cpu_seconds": 1.0})())
    assert buf.getvalue() == ""
