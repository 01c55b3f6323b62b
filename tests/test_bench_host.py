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


def test_solve_roofline_counts_iterations_of_every_launch():
    # two steps of three solves: (kernel ms, iterations, completed sweeps)
    per = [[(0.6, 17, 17), (0.8, 17, 17)], [(1.0, 27, 27), (1.0, 27, 27)], [(1.5, 41, 41), (1.5, 41, 41)]]
    I, J, peak = 50_000, 800, 6000.0
    r = bench.solve_roofline(per, I, J, peak)
    cell = 4.0 * I * J
    alg = cell * 2 * (17 + 27 + 41)
    ms = 0.6 + 0.8 + 2 * 1.0 + 2 * 1.5
    assert r["launches_timed"] == 6
    assert r["achieved"] == pytest.approx(alg / 1e9 / (ms / 1e3))
    assert r["alg_bytes_per_launch"] == pytest.approx(alg / 6)
    assert r["frac_incl_setup_finalize"] == pytest.approx(cell * 2 * (19 + 29 + 43) / 1e9 / (ms / 1e3) / peak)
    first = r["per_launch"][0]
    assert first["iters"] == 17 and first["ms"] == pytest.approx(0.7)
    assert first["frac"] == pytest.approx(cell * 17 / 1e9 / 0.7e-3 / peak)
    assert bench.solve_roofline([[], [], []], I, J, peak)["achieved"] is None


def test_clock_sampler_decodes_nvml_reason_bits():
    cs = bench.ClockSampler(0)
    cs._nvml = object()  # stands in for an opened NVML handle; nothing is polled

    class _T:
        def join(self, timeout=None):
            pass

    cs.t = _T()
    cs.samples = [(2070.0, 2070.0, 0x0), (1900.0, 2070.0, 0x4), (2000.0, 2070.0, 0x4 | 0x40)]
    out = cs.stop()
    assert out["sm_mhz"] == 2000.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
