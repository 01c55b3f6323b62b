#!/usr/bin/env python3
"""Benchmark of the entropic-OT association hot path on one GB300 (or N replicas).

Workload (one "step"): the 50,000 devices x 800 RRHs instance (4 km^2, 5 hot spots,
lognormal(0, 1.5) traffic, capacity-proportional RRH marginal) with gains resident in HBM:
rates (Sec. II-A) -> cost C = 1/(mu R) and the median of C -> three Sinkhorn solves
(Algorithm 1, FP32 log domain, tol 1e-6, <= 2000 iterations) at eps = {0.1, 0.03, 0.01} x
median(C), each with its FP64 finalize.  Metric: Sinkhorn cells x iterations per second
over the whole step.  C (160 MB) is larger than the 126 MB L2, so no flush is needed
between steps.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs an independent replica (the single instance does not
shard without a per-iteration exchange); value = cells*iters of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sinkhorn cells*iters/s"
UNIT = "cells*iters/s"
EPS_REL = (0.1, 0.03, 0.01)
TOL = 1e-6
MAX_ITER = 2000


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_inputs():
    from paper_1805_01559_gb300 import instances
    return instances.config2(seed=0)


# ------------------------------------------------------------------------------ CPU baseline
def cpu_baseline(inst, rows: int = 0, iters: int = 0):
    """The FP64 oracle timed on the host cores on the Sinkhorn work of one step.

    Default (rows = iters = 0): the full instance, all three eps, tol 1e-6 -- the same
    solves one GPU step makes.  rows/iters > 0 bound the sample to the first `rows`
    devices and a fixed iteration count at the first eps.
    """
    import oracle
    n = rows or inst.I
    G = inst.G[:n].astype(np.float64)
    R = oracle.rates(G, inst.P, inst.N0, inst.W_hz)
    C = oracle.cost(R, inst.mu)
    lam = inst.lam[:n] / inst.lam[:n].sum()
    q = inst.q / inst.q.sum()
    med = oracle.median(C)
    work, t_all = 0, 0.0
    for er in (EPS_REL[:1] if iters else EPS_REL):
        t0 = time.perf_counter()
        _, _, it, _ = oracle.sinkhorn(C, lam, q, er * med, 0.0 if iters else TOL, iters or MAX_ITER)
        t_all += time.perf_counter() - t0
        work += n * inst.J * it
    if iters:
        what = f"first {n} of {inst.I} devices x {inst.J} RRHs, {iters} iterations at eps = {EPS_REL[0]} x median(C)"
    else:
        what = f"the full {inst.I} x {inst.J} instance solved to tol {TOL} at eps = {list(EPS_REL)} x median(C)"
    return {"value": work / t_all, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{what}; FP64 Sinkhorn only (rates and cost untimed), wall {t_all:.2f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    inst = make_inputs()
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(inst, rows=args.ref_rows, iters=1)
    t_all = 0.0
    work = 0.0
    for _ in range(args.steps):
        cb = cpu_baseline(inst, rows=args.ref_rows, iters=1)
        vals.append(cb["value"])
        work += args.ref_rows * inst.J
        t_all += args.ref_rows * inst.J / cb["value"]
    value = work / t_all
    cb["value"] = value
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"c2_50000x800 sample: {args.ref_rows} devices x 800 RRHs, 1 iteration/step",
                       "I": args.ref_rows, "J": inst.J},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch

    from paper_1805_01559_gb300 import binding

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    inst = make_inputs()
    I, J = inst.I, inst.J
    dev = torch.device("cuda", local)
    G_h = torch.from_numpy(np.ascontiguousarray(inst.G, dtype=np.float32)).pin_memory()
    P_h = torch.from_numpy(inst.P.astype(np.float32)).pin_memory()
    lam_h = torch.from_numpy(inst.lam.astype(np.float32)).pin_memory()
    q_h = torch.from_numpy(inst.q.astype(np.float32)).pin_memory()
    G = G_h.to(dev)
    P = P_h.to(dev)
    lam = lam_h.to(dev)
    q = q_h.to(dev)
    R = torch.empty((I, J), dtype=torch.float32, device=dev)
    C = torch.empty((I, J), dtype=torch.float32, device=dev)
    fs = [torch.empty(I, dtype=torch.float64, device=dev) for _ in EPS_REL]
    gs = [torch.empty(J, dtype=torch.float64, device=dev) for _ in EPS_REL]
    ctx = binding.Context(local)
    ctx.enable_timing(True)
    loop_ms, loop_bytes, loop_launches = [], [], 0
    iters_seen = []

    def step(record=False):
        ctx.build_rates(G, P, inst.N0, inst.W_hz, R_out=R)
        _, med = ctx.build_cost(R, inst.mu, eps_rel=1.0, C_out=C)
        cells = 0
        its = []
        for k, er in enumerate(EPS_REL):
            res = ctx.solve_cost(C, lam, q, er * med, tol=TOL, max_iter=MAX_ITER, f=fs[k], g=gs[k])
            cells += I * J * res.iters
            its.append(res.iters)
            if record:
                t = ctx.last_timings()
                if t["valid"]:
                    loop_ms.append(t["loop_ms"])
                    loop_bytes.append(4.0 * I * J * t["sweeps"])
        return cells, its

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = ctx.launch_count()
    s = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(s)
    cells = 0
    for _ in range(args.steps):
        c, its = step(record=True)
        cells += c
        iters_seen.append(its)
    ev1.record(s)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if dist:
        dist.barrier()
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        c = torch.tensor([float(cells)], device=dev, dtype=torch.float64)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        cells = float(c.item())
    value = cells / (ms / 1e3)

    # e2e: the same step through the public API with host buffers, copies inside the timed region.
    f_h = [torch.empty(I, dtype=torch.float64).pin_memory() for _ in EPS_REL]
    g_h = [torch.empty(J, dtype=torch.float64).pin_memory() for _ in EPS_REL]
    e2e_cells = 0
    torch.cuda.synchronize()
    ev0.record(s)
    for _ in range(args.steps):
        G.copy_(G_h, non_blocking=True)
        P.copy_(P_h, non_blocking=True)
        lam.copy_(lam_h, non_blocking=True)
        q.copy_(q_h, non_blocking=True)
        c, _ = step()
        e2e_cells += c
        for k in range(len(EPS_REL)):
            f_h[k].copy_(fs[k], non_blocking=True)
            g_h[k].copy_(gs[k], non_blocking=True)
    ev1.record(s)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
        c = torch.tensor([float(e2e_cells)], device=dev, dtype=torch.float64)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        e2e_cells = float(c.item())
    h2d = G_h.numel() * 4 + P_h.numel() * 4 + lam_h.numel() * 4 + q_h.numel() * 4
    d2h = sum(x.numel() * 8 for x in f_h) + sum(x.numel() * 8 for x in g_h)

    peak, peak_kind = _peaks()
    achieved = (sum(loop_bytes) / 1e9) / (sum(loop_ms) / 1e3) if loop_ms else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "sk_loop_traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get("traffic_bytes_per_launch")
        except Exception:
            traffic = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c2_50000x800: rates -> cost+median -> Sinkhorn at eps={0.1,0.03,0.01}*median",
                       "I": I, "J": J, "eps_rel": list(EPS_REL), "tol": TOL, "max_iter": MAX_ITER,
                       "iters": iters_seen[0] if iters_seen else None,
                       "l2": "inputs larger than L2 (C and G 160 MB each > 126 MB)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": "sk_loop (persistent Sinkhorn sweep)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "bytes_per_cell_iter": 4, "launches_timed": len(loop_ms)},
            "e2e": {"value": e2e_cells / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_solve(args):
    """Driver for ncu captures of the solver: build the 50,000 x 800 instance, then
    `--profile-solves` solves at eps = 0.1 median(C) (capture the last with -s/-c)."""
    import torch

    from paper_1805_01559_gb300 import binding
    inst = make_inputs()
    dev = torch.device("cuda", 0)
    G = torch.from_numpy(np.ascontiguousarray(inst.G, dtype=np.float32)).to(dev)
    P = torch.from_numpy(inst.P.astype(np.float32)).to(dev)
    lam = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    ctx = binding.Context(0)
    R = ctx.build_rates(G, P, inst.N0, inst.W_hz)
    C, med = ctx.build_cost(R, inst.mu, eps_rel=1.0)
    for _ in range(args.profile_solves):
        res = ctx.solve_cost(C, lam, q, 0.1 * med, tol=TOL, max_iter=MAX_ITER)
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": "c2_50000x800 eps=0.1*median", "iters": res.iters,
                      "cost": res.transport_cost}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=12_500)
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="only run this many solves of the benchmark instance (for profiler captures)")
    args = ap.parse_args()
    if args.profile_solves > 0:
        return run_profile_solve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
