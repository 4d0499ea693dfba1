"""The benchmark's host logic on CPU: two gloo ranks on 127.0.0.1 (max over
ranks), the roofline's algorithmic bytes and the traffic digest.
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


def test_sweep_bytes_by_hand():
    """The roofline's bytes: the scope table's 8 B (FP32) / 16 B (FP64) per
    band-direction cell update.  Beside it, this design's own minimum for the
    32^3 cube's sweep, item by item: records (cell, slot, export, G and three
    inflow (reference, coefficient) pairs = 40 B) per (direction, cell), the
    per-cell FP64 collision-moment sum once, the (T', Qdot) pairs, and the
    wall rows of all bands."""
    N, D, Bp = 32768, 128, 40
    assert bench.sweep_algorithmic_bytes(N * D * Bp, 4) == 8 * N * D * Bp
    assert bench.sweep_algorithmic_bytes(N * D * Bp, 8) == 16 * N * D * Bp
    st = {"K": 3, "items": 1280, "exports": 381056, "imports": 393216}
    expect = D * N * 40 + N * 8 + N * 8 + (381056 + 393216) * Bp * 4
    assert bench.sweep_design_bytes(st, N, D, 4, Bp) == expect == 292179968
    # second order adds the source read and the distribution kept, per band
    assert bench.sweep_design_bytes(st, N, D, 4, Bp, order=2) == expect + 2 * D * N * Bp * 4
    # FP operations per update: one FMA per inflow face (half the faces) + 7
    assert bench.sweep_flops_per_update(4) == 11 and bench.sweep_flops_per_update(6) == 13


def test_sweep_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    """The committed DRAM traffic is reported only while the digest of the
    sweep's sources and the launch layout match the capture's; a capture on
    a smaller case is scaled by the updates a launch processes."""
    import hashlib
    import shutil
    csrc = tmp_path / "paper_2607_03226_b300" / "csrc"
    csrc.mkdir(parents=True)
    names = ("sweep.cu", "vecio.cuh", "layout.h", "sweep_args.h")
    for f in names:
        shutil.copy(os.path.join(os.path.dirname(HERE), "paper_2607_03226_b300", "csrc", f), csrc / f)
    h = hashlib.sha256()
    for f in names:
        h.update((csrc / f).read_bytes())
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "sweep_kernel_finfet3d_fp32.md"
    prof.write_text("# capture\n\ntraffic_bytes_per_launch: 123456\nupdates_per_launch: 1000\n"
                    f"sweep_source_digest: {h.hexdigest()[:16]}\nlayout: band_group=8 cta_threads=544\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._sweep_traffic("finfet3d", "fp32", 8, 544, 1000) == 123456
    assert bench._sweep_traffic("finfet3d", "fp32", 8, 544, 8000) == 8 * 123456   # scaled to a full launch
    assert bench._sweep_traffic("finfet3d", "fp32", 4, 256, 1000) is None          # another layout
    assert bench._sweep_traffic("finfet2d", "fp32", 8, 544, 1000) is None          # no capture of that workload
    with open(csrc / "sweep.cu", "a") as fh:             # the kernel changed since the capture
        fh.write("\n// edited\n")
    assert bench._sweep_traffic("finfet3d", "fp32", 8, 544, 1000) is None
