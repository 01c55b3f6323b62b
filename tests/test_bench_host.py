"""Host-side logic of bench.py: the N-replica aggregation over a world_size-2 `gloo` group on
CPU, the reference arm's rank handling, and the stored-traffic lookup."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (10 + r) ms for (r + 1) * 1e9 cells*iters
        ms, work = bench.reduce_ranks(dist, torch.device("cpu"), 10.0 + rank, (rank + 1) * 1e9)
        out.put((rank, ms, work))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    # every rank sees the slowest time and the work of all ranks: value = 3e9 / 11 ms
    for _, ms, work in got:
        assert ms == 11.0
        assert work == 3e9


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, ref_rows = 1, 0, 100

    def boom():
        raise AssertionError("rank 1 must not build inputs")

    monkeypatch.setattr(bench, "make_inputs", boom)
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_stored_traffic_follows_the_solver_sources(tmp_path, monkeypatch):
    f = tmp_path / "p.md"
    f.write_text(f"x\ntraffic_bytes_per_launch: 1.5e9\nsolver_source_sha256: {bench.solver_source_hash()}\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(f))
    assert bench.stored_traffic() == 1.5e9
    f.write_text("traffic_bytes_per_launch: 1.5e9\nsolver_source_sha256: 0123456789abcdef\n")
    assert bench.stored_traffic() is None  # captured on other sources: no figure
    f.write_text("no figures here\n")
    assert bench.stored_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.stored_traffic() is None


def test_stored_euclid_instruction_count_follows_the_solver_sources(tmp_path, monkeypatch):
    f = tmp_path / "e.md"
    f.write_text(f"x\nwarp_inst_per_cell_sweep: 1.25\nsolver_source_sha256: {bench.solver_source_hash()}\n")
    monkeypatch.setattr(bench, "EUCLID_PROFILE", str(f))
    assert bench.stored_euclid_inst() == 1.25
    f.write_text("warp_inst_per_cell_sweep: 1.25\nsolver_source_sha256: 0123456789abcdef\n")
    assert bench.stored_euclid_inst() is None
    monkeypatch.setattr(bench, "EUCLID_PROFILE", str(tmp_path / "missing.md"))
    assert bench.stored_euclid_inst() is None
