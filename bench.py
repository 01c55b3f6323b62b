#!/usr/bin/env python3
"""Benchmark of the entropic-OT association hot path on one GB300 (or N replicas).

Workload (one "step"): the 50,000 devices x 800 RRHs instance (4 km^2, 5 hot spots,
lognormal(0, 1.5) traffic, capacity-proportional RRH marginal) with gains resident in HBM:
rates (Sec. II-A) and cost C = 1/(mu R) in one pass, the median of C -> three Sinkhorn solves
(Algorithm 1, FP32 log domain, tol 1e-6, <= 2000 iterations) at eps = {0.1, 0.03, 0.01} x
median(C), each with its FP64 finalize, enqueued back to back through the asynchronous API
(--multi: the two smaller eps in one launch that shares each read of C, sk_solve_multi).
Metric: Sinkhorn cells x iterations per second over the whole step.  C (160 MB) is larger
than the 126 MB L2, so no flush is needed between steps.

On one GPU the line also carries three records (--sub-records 0 leaves them out):
  batched    64 ragged instances, the batched persistent launch against a loop of solves;
  serving    one Poisson trace through the server and through plain per-instance calls;
  precision  the 400,000 x 4,096 instance, FP32 log domain against BF16 and FP16 K~.
--workload selects the full-size form of one of them (or another workload) instead.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs an independent replica (the single instance does not
shard without a per-iteration exchange); value = cells*iters of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import re
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
    """SM clocks and throttle reasons sampled while the timed region runs.

    Reads NVML through ctypes every 10 ms (the timed region can be shorter than
    nvidia-smi's shortest interval); falls back to `nvidia-smi -lms 200` when NVML cannot be
    loaded.  Only reads: no clock, power or other setting is changed."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clocks-event reason bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40}

    def __init__(self, device_index: int, period_s: float = 0.01):
        self.dev = device_index
        self.period = period_s
        self.proc = None
        self.lines = []
        self.samples = []  # (sm_mhz, max_mhz, reason bits) from NVML
        self.t = None
        self._halt = threading.Event()
        self._nvml = None

    def _nvml_open(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return None
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.dev), ctypes.byref(h)) != 0:
            return None
        return lib, h

    def start(self):
        self._nvml = self._nvml_open()
        if self._nvml is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _poll(self):
        import ctypes
        lib, h = self._nvml
        mhz, mx = ctypes.c_uint(), ctypes.c_uint()
        bits = ctypes.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._halt.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    get_reasons(h, ctypes.byref(bits)) == 0):
                self.samples.append((float(mhz.value), float(mx.value), int(bits.value)))
            self._halt.wait(self.period)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self._nvml is not None:
            self._halt.set()
            self.t.join(timeout=2)
            if not self.samples:
                return None
            reasons = sorted(nm for nm, bit in self.REASONS.items() if any(b & bit for _, _, b in self.samples))
            return {"sm_mhz": statistics.median(x[0] for x in self.samples),
                    "sm_max_mhz": max(x[1] for x in self.samples), "reasons": reasons,
                    "samples": len(self.samples), "source": "nvml, 10 ms"}
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
                "samples": len(sm), "source": "nvidia-smi, 200 ms"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_ranks(dist, dev, ms: float, work: float):
    """Whole-job figures of N replicas: the slowest rank's time and the work of all ranks."""
    import torch
    t = torch.tensor([float(ms)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(work)], device=dev, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


# Solver sources whose change invalidates a stored DRAM-traffic figure of sk_solve.
SOLVER_SOURCES = ("sk_core.cuh", "k_sinkhorn.cu", "ot_common.cuh")
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "sk_solve_c2_50000x800.md")


def solver_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in SOLVER_SOURCES:
        with open(os.path.join(ROOT, "paper_1805_01559_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic():
    """DRAM bytes per sk_solve launch from the committed ncu summary, or None when the summary
    is missing or was taken on other solver sources than the ones built now."""
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    m_t = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", text, re.M)
    m_h = re.search(r"^solver_source_sha256:\s*([0-9a-f]+)", text, re.M)
    if not m_t or not m_h or m_h.group(1) != solver_source_hash():
        return None
    return float(m_t.group(1))


EUCLID_PROFILE = os.path.join(ROOT, "profiles", "sk_solve_euclid_50000x800.md")


def stored_euclid_inst():
    """Warp instructions per cell and sweep of sk_solve_euclid from the committed ncu summary,
    or None when it is missing or was taken on other solver sources than the ones built now."""
    try:
        text = open(EUCLID_PROFILE).read()
    except OSError:
        return None
    m_i = re.search(r"^warp_inst_per_cell_sweep:\s*([0-9.eE+]+)", text, re.M)
    m_h = re.search(r"^solver_source_sha256:\s*([0-9a-f]+)", text, re.M)
    if not m_i or not m_h or m_h.group(1) != solver_source_hash():
        return None
    return float(m_i.group(1))


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


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal: stated beside the measured copy bandwidth


def solve_roofline(per_launch, I: int, J: int, peak: float):
    """Roofline of the solver over a step's launches.

    per_launch[k] lists (kernel ms, iterations, completed sweeps) of every timed launch of the
    k-th eps.  The algorithmic bytes of a launch are 4 B x I x J x iterations (one read of C per
    iteration of Algorithm 1); achieved = their sum over all launches / the summed kernel
    time.  The same with the two extra reads the kernel makes (testing the last plan, the
    finalize sweep) is reported apart as frac_incl_setup_finalize."""
    launches = [x for lst in per_launch for x in lst]
    if not launches:
        return {"achieved": None, "alg_bytes_per_launch": None, "frac_incl_setup_finalize": None,
                "per_launch": [], "launches_timed": 0}
    cell = 4.0 * I * J
    ms = sum(x[0] for x in launches)
    alg = sum(cell * x[1] for x in launches)
    reads = sum(cell * (x[2] + 2) for x in launches)
    rows = []
    for lst in per_launch:
        if not lst:
            continue
        lms = sum(x[0] for x in lst) / len(lst)
        it = sum(x[1] for x in lst) / len(lst)
        gbs = cell * it / 1e9 / (lms / 1e3)
        rows.append({"iters": it, "ms": lms, "achieved": gbs, "frac": gbs / peak,
                     "frac_incl_setup_finalize": cell * (it + 2) / 1e9 / (lms / 1e3) / peak})
    return {"achieved": alg / 1e9 / (ms / 1e3), "alg_bytes_per_launch": alg / len(launches),
            "frac_incl_setup_finalize": reads / 1e9 / (ms / 1e3) / peak, "per_launch": rows,
            "launches_timed": len(launches)}


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
    G0 = G_h.to(dev)
    P0 = P_h.to(dev)
    lam0 = lam_h.to(dev)
    q0 = q_h.to(dev)
    C = torch.empty((I, J), dtype=torch.float32, device=dev)
    fs = [torch.empty(I, dtype=torch.float64, device=dev) for _ in EPS_REL]
    gs = [torch.empty(J, dtype=torch.float64, device=dev) for _ in EPS_REL]
    ctx = binding.Context(local)
    ctx.enable_timing(True)
    # per eps: (kernel ms, iterations, completed sweeps) of every timed launch
    per_launch = [[] for _ in EPS_REL]
    iters_seen = []

    def step(record=False, buf=None):
        G, P, lam, q = buf if buf is not None else (G0, P0, lam0, q0)
        # rates (Sec. II-A) and the cost in one pass over the gains, then the median of C
        _, med = ctx.build_cost_from_gains(G, P, inst.N0, inst.W_hz, inst.mu, eps_rel=1.0, C_out=C)
        if not args.multi:
            # the three solves enqueued back to back, each reading C on its own; each solve's
            # kernel timing is read right after its own wait (the next wait replaces it)
            tickets = [ctx.solve_cost_async(C, lam, q, er * med, tol=TOL, max_iter=MAX_ITER, f=fs[k], g=gs[k])
                       for k, er in enumerate(EPS_REL)]
            results = []
            for k, x in enumerate(tickets):
                res = x.wait()
                results.append(res)
                if record:
                    t = ctx.last_timings()
                    if t["valid"]:
                        per_launch[k].append((t["loop_ms"], res.iters, t["sweeps"]))
        else:
            # the first eps on its own launch, the two smaller ones in one launch sharing each
            # read of C while both iterate
            first = ctx.solve_cost_async(C, lam, q, EPS_REL[0] * med, tol=TOL, max_iter=MAX_ITER, f=fs[0], g=gs[0])
            r0 = first.wait()
            if record:
                t = ctx.last_timings()
                if t["valid"]:
                    per_launch[0].append((t["loop_ms"], r0.iters, t["sweeps"]))
            results = [r0] + ctx.solve_cost_multi(C, lam, q, [er * med for er in EPS_REL[1:]], tol=TOL,
                                                  max_iter=MAX_ITER, fs=fs[1:], gs=gs[1:])
        cells = 0
        its = []
        for res in results:
            cells += I * J * res.iters
            its.append(res.iters)
        if record and args.multi:
            t = ctx.last_timings()
            if t["valid"]:
                per_launch[1].append((t["loop_ms"], sum(r.iters for r in results[1:]), t["sweeps"]))
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
        ms, cells = reduce_ranks(dist, dev, ms, cells)
    value = cells / (ms / 1e3)

    # e2e: the same step through the public API with host buffers, every step's inputs copied
    # from pinned host memory and its potentials read back inside the timed region.  Inputs
    # are double-buffered: step k+1's copy runs on a copy stream while step k computes.
    f_h = [torch.empty(I, dtype=torch.float64).pin_memory() for _ in EPS_REL]
    g_h = [torch.empty(J, dtype=torch.float64).pin_memory() for _ in EPS_REL]
    e2e_cells = 0
    bufs = [(G0, P0, lam0, q0), tuple(torch.empty_like(x) for x in (G0, P0, lam0, q0))]
    cs = torch.cuda.Stream(device=dev)
    ev_copy = [torch.cuda.Event(), torch.cuda.Event()]
    ev_free = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(k):
        cs.wait_event(ev_free[k % 2])  # the step that used this buffer last has finished
        with torch.cuda.stream(cs):
            for dst, src in zip(bufs[k % 2], (G_h, P_h, lam_h, q_h)):
                dst.copy_(src, non_blocking=True)
        ev_copy[k % 2].record(cs)

    torch.cuda.synchronize()
    ev0.record(s)
    cs.wait_event(ev0)
    upload(0)
    for k in range(args.steps):
        if k + 1 < args.steps:
            upload(k + 1)
        s.wait_event(ev_copy[k % 2])
        c, _ = step(buf=bufs[k % 2])
        ev_free[k % 2].record(s)
        e2e_cells += c
        for j in range(len(EPS_REL)):
            f_h[j].copy_(fs[j], non_blocking=True)
            g_h[j].copy_(gs[j], non_blocking=True)
    ev1.record(s)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1)
    if dist:
        e2e_ms, e2e_cells = reduce_ranks(dist, dev, e2e_ms, e2e_cells)
    h2d = G_h.numel() * 4 + P_h.numel() * 4 + lam_h.numel() * 4 + q_h.numel() * 4
    d2h = sum(x.numel() * 8 for x in f_h) + sum(x.numel() * 8 for x in g_h)

    peak, peak_kind = _peaks()
    roof = solve_roofline(per_launch, I, J, peak)
    traffic = stored_traffic()
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
            "roofline": {"bound": "hbm",
                         "kernel": ("sk_solve (persistent Sinkhorn: setup, sweeps, finalize sweep), one launch per eps"
                                    if not args.multi else
                                    "sk_solve for the first eps, sk_solve_multi for the other two (first and "
                                    "finalize sweeps one solve after the other, plan-scale sweeps shared)"),
                         "achieved": roof["achieved"], "peak": peak, "unit": "GB/s",
                         "frac": (roof["achieved"] / peak) if roof["achieved"] else None, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "bytes_per_cell_iter": 4,
                         "definition": "4 B x I x J x iterations, summed over the step's solver launches, / "
                                       "their summed kernel time (CUDA events on the solve stream)",
                         "alg_bytes_per_launch": roof["alg_bytes_per_launch"],
                         "frac_incl_setup_finalize": roof["frac_incl_setup_finalize"],
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "frac_of_nominal": (roof["achieved"] / NOMINAL_HBM_GBS) if roof["achieved"] else None,
                         "reads_of_C_per_launch": "iters + 2" if not args.multi else
                         "iters + 2, then max(iters) + 2 x 2",
                         "per_launch": roof["per_launch"],
                         "launches_timed": roof["launches_timed"]},
            "e2e": {"value": e2e_cells / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if ws == 1:
            # the per-cell exponential against the SFU's measured ceiling: one ex2 a cell and
            # sweep, iters + 2 sweeps a launch
            rate = ctx.measure_ex2_rate()
            ls = [x for lst in per_launch for x in lst]
            if ls and rate > 0:
                need = sum(float(I) * J * (x[1] + 2) for x in ls) / (sum(x[0] for x in ls) / 1e3)
                line["sfu"] = {"ex2_per_s_measured": rate, "solver_ex2_per_s": need, "frac": need / rate,
                               "definition": "ex2 results/s of ot_assoc_measure_ex2_rate (8 independent chains a "
                                             "thread) against I x J x (iters + 2) / sk_solve time"}
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst)
        if ws == 1 and args.sub_records:
            # the batched and serving configurations, smaller than their own workloads so that the
            # default run stays within minutes (--workload c3 / c5 run them at full size)
            pool = _pool(min(16, os.cpu_count() or 1))
            try:
                line["batched"] = batched_record(ctx, pool, args.sub_c3_instances, 2, 3)
                line["serving"] = serving_record(ctx, pool, args.c5_rate, args.sub_c5_seconds, args.c5_group)
                line["precision"] = precision_record(ctx, pool, args.c4_rows, 1)
            finally:
                pool.close()
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_solve(args):
    """Driver for ncu captures of the solver: build the 50,000 x 800 instance, then
    `--profile-solves` rounds of the step's three solves (eps = 0.1, 0.03, 0.01 median(C));
    capture the last round's three sk_solve launches with -s/-c."""
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
    its = []
    for _ in range(args.profile_solves):
        its = [ctx.solve_cost(C, lam, q, er * med, tol=TOL, max_iter=MAX_ITER).iters for er in EPS_REL]
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": "c2_50000x800 eps=(0.1,0.03,0.01)*median", "iters": its,
                      "alg_bytes_per_launch": 4.0 * inst.I * inst.J * (sum(its) / len(its) + 2),
                      "solver_source_sha256": solver_source_hash()}))
    ctx.close()
    return 0


# ------------------------------------------------------------------------------ other workloads
# The default line above is the headline benchmark.  These modes measure the other
# configurations (one JSON line each, "workload" names them); inputs are generated on the host
# in a process pool started before any CUDA call.
def _pool(n: int):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)


def _gen_c3(args):
    from paper_1805_01559_gb300 import instances as ins
    I, J, seed = args
    x = ins.config3_cell(I, J, seed, dtype=np.float32)
    return (np.ascontiguousarray(x.G, np.float32), x.P.astype(np.float32), x.lam.astype(np.float32),
            x.q.astype(np.float32), x.N0, x.W_hz, x.mu)


_C4 = {}


def _gen_c4_block(args):
    from paper_1805_01559_gb300 import instances as ins
    seed, I, J, block, b = args
    key = (seed, I, J, block)
    if key not in _C4:
        _C4.clear()
        _C4[key] = ins.config4_blocked(seed, I, J, block)
    return b, _C4[key].gains_block(b)


def _gen_c5(args):
    from multiprocessing import shared_memory
    from paper_1805_01559_gb300 import instances as ins
    I, J, seed = args
    c = ins.serving_cell(I, J, seed)
    sh = np.ascontiguousarray(c.shadow_db, np.float32)
    shm = shared_memory.SharedMemory(create=True, size=sh.nbytes)
    np.ndarray(sh.shape, np.float32, buffer=shm.buf)[:] = sh
    name = shm.name
    shm.close()
    return dict(I=I, J=J, dev_xy=c.dev_xy, vel=c.vel, rrh_xy=c.rrh_xy.astype(np.float32), lam=c.lam, q=c.q,
                side=c.side, shm=name)


def _timed(fn, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0)


def batched_record(ctx, pool, n_instances: int, warmup: int, steps: int, autotune: bool = False):
    """The first n ragged instances of the batched configuration (I ~ U{2000..60000},
    J ~ U{64..1024}, channel as the 1000 x 50 configuration), eps = 0.05 median(C) each: the
    batched persistent launch (captured graph) against the per-instance solver loop, same
    tolerance."""
    import torch
    from paper_1805_01559_gb300 import binding
    from paper_1805_01559_gb300 import instances as ins
    shapes = ins.config3_shapes()[:n_instances]
    dev = torch.device("cuda", 0)
    items = []
    t0 = time.perf_counter()
    for (G, P, lam, q, N0, W, mu), (I, J, _) in zip(pool.imap(_gen_c3, shapes, chunksize=1), shapes):
        Gd = torch.from_numpy(G).to(dev)
        R = ctx.build_rates(Gd, torch.from_numpy(P).to(dev), N0, W)
        ld = (J + 3) // 4 * 4
        C = torch.empty((I, ld), dtype=torch.float32, device=dev)[:, :J]
        _, med = ctx.build_cost(R, mu, eps_rel=1.0, C_out=C)
        del Gd, R
        items.append(dict(C=C, p=torch.from_numpy(lam).to(dev), q=torch.from_numpy(q).to(dev), eps=0.05 * med))
    gen_s = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    mk = lambda: [binding.Instance(C=x["C"], p=x["p"], q=x["q"], eps=x["eps"], tol=TOL, max_iter=MAX_ITER)
                  for x in items]
    cells = [x["C"].shape[0] * x["C"].shape[1] for x in items]

    def plain():
        return [ctx.solve_cost(x["C"], x["p"], x["q"], x["eps"], tol=TOL, max_iter=MAX_ITER).iters for x in items]

    res = {}
    for name in ("plain", "batched", "batched_tuned"):
        if name == "batched_tuned":
            if not autotune:
                continue
            t_tune = time.perf_counter()
            ctx.autotune(mk(), iters=6)
            res["tune_s"] = time.perf_counter() - t_tune
        b = ctx.batch(mk(), graph=True) if name != "plain" else None
        run = plain if b is None else (lambda: [r.iters for r in b.run()])
        for _ in range(warmup):
            run()
        ms_all, its = [], None
        for _ in range(steps):
            its, ms, _ = _timed(run, s)
            ms_all.append(ms)
        ms = statistics.median(ms_all)
        ci = sum(c * it for c, it in zip(cells, its))
        res[name] = {"ms": ms, "solves_per_s": len(items) / (ms / 1e3), "cells_iters_per_s": ci / (ms / 1e3),
                     "gbs_equiv": 4.0 * sum(c * (it + 2) for c, it in zip(cells, its)) / (ms / 1e3) / 1e9,
                     "gbs_alg": 4.0 * ci / (ms / 1e3) / 1e9, "iters_total": int(sum(its))}
        if b is not None:
            b.close()
    best = res.get("batched_tuned", res["batched"])
    peak, peak_kind = _peaks()
    return {"workload": f"c3_{len(items)}_ragged: batched persistent launch (graph) vs per-instance loop",
            "instances": len(items), "cells": int(sum(cells)), "tol": TOL, "eps_rel": 0.05, "inputs_s": gen_s,
            "solves_per_s_ratio": best["solves_per_s"] / res["plain"]["solves_per_s"], **res,
            "roofline": {"bound": "hbm", "kernel": "sk_batch", "achieved": best["gbs_alg"], "peak": peak,
                         "unit": "GB/s", "frac": best["gbs_alg"] / peak,
                         "frac_incl_setup_finalize": best["gbs_equiv"] / peak, "traffic": None,
                         "peak_kind": peak_kind}}


def run_c3(args):
    """256 ragged instances (I ~ U{2000..60000}, J ~ U{64..1024}, channel as the 1000 x 50
    configuration), eps = 0.05 median(C) each: the batched persistent launch (captured graph)
    against the per-instance solver loop, same tolerance."""
    pool = _pool(min(16, os.cpu_count() or 1))
    from paper_1805_01559_gb300 import binding
    ctx = binding.Context(0)
    rec = batched_record(ctx, pool, args.c3_instances, args.warmup, args.steps, args.autotune)
    pool.close()
    best = rec.get("batched_tuned", rec["batched"])
    line = {"metric": METRIC, "value": best["cells_iters_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rec["workload"], "instances": rec["instances"], "cells": rec["cells"],
                       "tol": TOL, "eps_rel": 0.05, "inputs_s": rec["inputs_s"]},
            "batched_vs_plain": rec, "roofline": rec["roofline"]}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def precision_record(ctx, pool, rows: int, warmup: int):
    """The 400,000 x 4,096 instance (16 km^2, hot spots, capacity q), eps = 0.05 median(C):
    the log-domain FP32 solver against the stored-kernel solver with K~ in BF16 and FP16."""
    import torch
    from paper_1805_01559_gb300 import binding
    from paper_1805_01559_gb300 import instances as ins
    I, J, block = rows, 4096, 8192
    inst = ins.config4_blocked(0, I, J, block)
    dev = torch.device("cuda", 0)
    P = torch.from_numpy(inst.P.astype(np.float32)).to(dev)
    C = torch.empty((I, J), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    jobs = [(0, I, J, block, b) for b in range(inst.nblocks)]
    for b, G in pool.imap_unordered(_gen_c4_block, jobs):
        r0 = b * block
        Gd = torch.from_numpy(G).to(dev)
        ctx.build_cost_from_gains(Gd, P, inst.N0, inst.W_hz, inst.mu, C_out=C[r0:r0 + G.shape[0]])
        del Gd
    gen_s = time.perf_counter() - t0
    med = ctx.median_f32(C.view(-1))
    eps = 0.05 * med
    p = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    s = torch.cuda.current_stream()
    out = {}
    ref = None
    ctx.enable_timing(True)
    for name, fn in (("f32_log", lambda: ctx.solve_cost(C, p, q, eps, tol=TOL, max_iter=MAX_ITER)),
                     ("bf16_K", lambda: ctx.solve_lowp(C, p, q, eps, tol=TOL, max_iter=MAX_ITER,
                                                       fmt=binding.OT_KERNEL_BF16)),
                     ("f16_K", lambda: ctx.solve_lowp(C, p, q, eps, tol=TOL, max_iter=MAX_ITER,
                                                      fmt=binding.OT_KERNEL_F16))):
        for _ in range(max(1, warmup)):
            fn()
        r, ms, _ = _timed(fn, s)
        t = ctx.last_timings()
        if ref is None:
            ref = r
        # the solver's persistent loop: C (4 bytes a cell) once per iteration for the log domain,
        # K~ (2 bytes a cell) once per loop iteration for the stored kernel
        if name == "f32_log":
            loop_bytes = 4.0 * I * J * r.iters
        else:
            loop_bytes = 2.0 * I * J * t["sweeps"]
        loop_gbs = loop_bytes / (t["loop_ms"] / 1e3) / 1e9 if t["valid"] and t["loop_ms"] > 0 else None
        out[name] = {"ms": ms, "loop_ms": t["loop_ms"] if t["valid"] else None, "loop_gbs": loop_gbs,
                     "first_iteration_and_build_ms": t["init_ms"] if (t["valid"] and name != "f32_log") else None,
                     "finalize_ms": t["finalize_ms"] if t["valid"] else None,
                     "iters": r.iters, "absorptions": r.absorptions,
                     "cells_iters_per_s": I * J * r.iters / (ms / 1e3), "transport_cost": r.transport_cost,
                     "cost_rel_vs_f32": abs(r.transport_cost - ref.transport_cost) / ref.transport_cost,
                     "marg_err_row": r.marg_err_row, "marg_err_col": r.marg_err_col, "status": r.status}
    del C
    torch.cuda.empty_cache()
    peak, peak_kind = _peaks()
    best = out["bf16_K"]
    roof = None
    if best["loop_gbs"]:
        roof = {"bound": "hbm", "kernel": "lp_loop (stored BF16 kernel, 2 bytes a cell and iteration)",
                "achieved": best["loop_gbs"], "peak": peak, "unit": "GB/s", "frac": best["loop_gbs"] / peak,
                "traffic": None, "peak_kind": peak_kind}
    return {"workload": f"c4_{I}x{J}: stored-kernel BF16/FP16 vs log-domain FP32", "I": I, "J": J, "eps": eps,
            "tol": TOL, "inputs_s": gen_s, "formats": out,
            "bf16_speedup_vs_f32": out["f32_log"]["ms"] / out["bf16_K"]["ms"], "roofline": roof,
            "note": "marginal errors are the device's FP64 evaluation of the returned potentials on the true C "
                    "(the whole-instance comparison with the FP64 oracle is a test)"}


def run_c4(args):
    """The 400,000 x 4,096 instance: FP32 log domain against BF16 and FP16 stored kernels."""
    pool = _pool(min(16, os.cpu_count() or 1))
    from paper_1805_01559_gb300 import binding
    ctx = binding.Context(0)
    rec = precision_record(ctx, pool, args.c4_rows, args.warmup)
    pool.close()
    best = rec["formats"]["bf16_K"]
    line = {"metric": METRIC, "value": best["cells_iters_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 K~ (FP32 accumulation)", "data": "synthetic",
            "config": {"workload": rec["workload"], "I": rec["I"], "J": rec["J"], "eps": rec["eps"], "tol": TOL,
                       "inputs_s": rec["inputs_s"]},
            "formats": rec["formats"], "roofline": rec["roofline"]}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _c5_cells(shapes, pool):
    """Host data of the serving cells (drawn in a spawn pool): positions, velocities, RRHs,
    traffic, marginal and the fixed shadowing of every link."""
    from multiprocessing import shared_memory
    cells = []
    gen = list(pool.imap(_gen_c5, shapes, chunksize=1))
    try:
        for d in gen:
            shm = shared_memory.SharedMemory(name=d["shm"])
            try:
                d["shadow"] = np.ndarray((d["I"], d["J"]), np.float32, buffer=shm.buf).copy()
            finally:
                shm.close()
                shm.unlink()
                d["shm"] = None
            cells.append(d)
    finally:
        for d in gen:
            if d["shm"]:
                try:
                    shared_memory.SharedMemory(name=d["shm"]).unlink()
                except FileNotFoundError:
                    pass
    return cells


def _lat_stats(lat_ms):
    lat = np.asarray(lat_ms, dtype=np.float64)
    if lat.size == 0:
        return None
    return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
            "mean": float(lat.mean())}


def _arm_record(name, t0, t_end, lat, queue, device, errs, iters, failed, extra=None, classes=None):
    """classes: per request the size class (I x J) it belongs to, for latency per class."""
    n = len(lat)
    rec = {"arm": name, "requests": n + failed, "failed": failed,
           "solves_per_s": n / max(t_end - t0, 1e-9), "latency_ms": _lat_stats(lat),
           "queue_wait_ms": _lat_stats(queue), "device_ms": _lat_stats(device),
           "marg_err_max": float(max(errs)) if errs else None,
           "iters_mean": float(np.mean(iters)) if iters else None}
    if classes is not None:
        by = {}
        for c, l in zip(classes, lat):
            by.setdefault(c, []).append(l)
        rec["latency_ms_by_class"] = {f"{c[0]}x{c[1]}": {**_lat_stats(v), "n": len(v)} for c, v in sorted(by.items())}
    if extra:
        rec.update(extra)
    return rec


def _serve_run(ctx, cells, t_arr, cidx, realtime: bool, group: int, trace=None):
    """The trace through the server (continuous batching, resident cells, warm starts).
    realtime: submit each request at its arrival time; else submit the whole trace at once."""
    import torch
    from paper_1805_01559_gb300 import instances as ins
    srv = ctx.server(group_ctas=group)
    try:
        ids = [srv.add_cell(d["I"], d["J"], 0.0, np.ones(d["J"]), d["lam"], d["q"], ins.MU_PER_BIT,
                            ins.noise_power_w(), ins.W_HZ, tol=TOL, max_iter=MAX_ITER, dev_xy=d["dev_xy"],
                            dev_v=d["vel"], rrh_xy=d["rrh_xy"], shadow_db=d["shadow"], side_m=d["side"],
                            eps_rel=0.05) for d in cells]
        last = np.zeros(len(ids))
        results = []
        torch.cuda.synchronize()
        start = time.perf_counter()
        t0_us = None
        for t, c in zip(t_arr, cidx):
            if realtime:
                while time.perf_counter() - start < t:
                    results += srv.poll()
            dt = float(t - last[c]) if last[c] > 0 else 0.0
            last[c] = t
            srv.submit(ids[c], None, dt)
        results += srv.drain(timeout_s=600)
        st = srv.stats()
    finally:
        srv.close()
    ok = [r for r in results if r.status in (0, 1)]
    t0 = min(r.t_submit_us for r in results)
    t_end = max(r.t_done_us for r in results)
    cell_of = {cid: k for k, cid in enumerate(ids)}
    if trace is not None:  # per request: cell, submitted, published, seen done (us), status
        trace.extend((cell_of[r.cell], r.t_submit_us, r.t_start_us, r.t_done_us, r.status) for r in results)
    return _arm_record("served" if realtime else "served_backlog", t0 / 1e6, t_end / 1e6,
                       [(r.t_done_us - r.t_submit_us) / 1e3 for r in ok],
                       [(r.t_start_us - r.t_submit_us) / 1e3 for r in ok],
                       [(r.t_done_us - r.t_start_us) / 1e3 for r in ok],
                       [max(r.marg_err_row, r.marg_err_col) for r in ok], [r.iters for r in ok],
                       len(results) - len(ok),
                       {"group_ctas": group, "resident_bytes": st["resident_bytes"], "launches": st["launches"]},
                       classes=[(cells[cell_of[r.cell]]["I"], cells[cell_of[r.cell]]["J"]) for r in ok])


def _plain_run(ctx, cells, t_arr, cidx, realtime: bool, fmt=None):
    """The same trace through the plain per-instance entry points, one request at a time in
    arrival order: ot_assoc_build_cost_mobile (devices moved by dt, C rebuilt) then a solve
    warm-started from the cell's previous g -- ot_assoc_solve_cost (FP32 log domain) or, with
    fmt, ot_assoc_solve_lowp (stored kernel K~ in that format)."""
    import torch
    from paper_1805_01559_gb300 import instances as ins
    dev = torch.device("cuda", 0)
    state = []
    for d in cells:
        I, J = d["I"], d["J"]
        ld = (J + 3) // 4 * 4
        st = {"xy": torch.from_numpy(np.ascontiguousarray(d["dev_xy"], np.float64)).to(dev),
              "v": torch.from_numpy(np.ascontiguousarray(d["vel"], np.float64)).to(dev),
              "rrh": torch.from_numpy(np.ascontiguousarray(d["rrh_xy"], np.float32)).to(dev),
              "sh": torch.from_numpy(d["shadow"]).to(dev),
              "P": torch.ones(J, dtype=torch.float32, device=dev),
              "p": torch.from_numpy(np.ascontiguousarray(d["lam"], np.float32)).to(dev),
              "q": torch.from_numpy(np.ascontiguousarray(d["q"], np.float32)).to(dev),
              "C": torch.empty((I, ld), dtype=torch.float32, device=dev)[:, :J],
              "f": torch.empty(I, dtype=torch.float64, device=dev),
              "g": torch.zeros(J, dtype=torch.float64, device=dev), "warm": False}
        _, st["eps"] = ctx.build_cost_mobile(st["xy"], st["v"], st["rrh"], st["sh"], st["P"], 0.0, d["side"],
                                             ins.noise_power_w(), ins.W_HZ, ins.MU_PER_BIT, C_out=st["C"],
                                             eps_rel=0.05)
        state.append(st)
    last = np.zeros(len(cells))
    lat, queue, device, errs, iters, classes = [], [], [], [], [], []
    failed = 0
    torch.cuda.synchronize()
    start = time.perf_counter()
    for t, c in zip(t_arr, cidx):
        if realtime:
            while time.perf_counter() - start < t:
                pass
        t_begin = time.perf_counter() - start
        d, st = cells[c], state[c]
        dt = float(t - last[c]) if last[c] > 0 else 0.0
        last[c] = t
        ctx.build_cost_mobile(st["xy"], st["v"], st["rrh"], st["sh"], st["P"], dt, d["side"], ins.noise_power_w(),
                              ins.W_HZ, ins.MU_PER_BIT, C_out=st["C"])
        warm = st["g"] if st["warm"] else None
        if fmt is None:
            r = ctx.solve_cost(st["C"], st["p"], st["q"], st["eps"], tol=TOL, max_iter=MAX_ITER, warm_g=warm,
                               f=st["f"], g=st["g"], want_load=False)
        else:
            r = ctx.solve_lowp(st["C"], st["p"], st["q"], st["eps"], tol=TOL, max_iter=MAX_ITER, fmt=fmt,
                               warm_g=warm, want_load=False)
            st["g"].copy_(r.g)
        st["warm"] = True
        t_done = time.perf_counter() - start
        arrival = t if realtime else 0.0
        if r.status in (0, 1):
            lat.append(1e3 * (t_done - arrival))
            queue.append(1e3 * (t_begin - arrival))
            device.append(1e3 * (t_done - t_begin))
            errs.append(max(r.marg_err_row, r.marg_err_col))
            iters.append(r.iters)
            classes.append((d["I"], d["J"]))
        else:
            failed += 1
    t_end = time.perf_counter() - start
    name = ("plain" if fmt is None else "plain_bf16") + ("" if realtime else "_backlog")
    return _arm_record(name, 0.0 if not realtime else float(t_arr[0]) if len(t_arr) else 0.0, t_end, lat, queue,
                       device, errs, iters, failed, classes=classes)


def serving_record(ctx, pool, rate: float, seconds: float, group: int, bf16: bool = True):
    """Served (continuous batching) against plain per-instance solves on one Poisson trace over
    the 64 serving cells, at the offered rate (latency) and as a backlog (capacity)."""
    from paper_1805_01559_gb300 import binding
    from paper_1805_01559_gb300 import instances as ins
    shapes = ins.serving_cell_shapes(64)
    t0 = time.perf_counter()
    cells = _c5_cells(shapes, pool)
    gen_s = time.perf_counter() - t0
    t_arr, cidx = ins.poisson_arrivals(rate, seconds, len(cells), seed=0)
    arms = [_serve_run(ctx, cells, t_arr, cidx, True, group), _serve_run(ctx, cells, t_arr, cidx, False, group),
            _plain_run(ctx, cells, t_arr, cidx, True), _plain_run(ctx, cells, t_arr, cidx, False)]
    if bf16:
        arms.append(_plain_run(ctx, cells, t_arr, cidx, False, fmt=binding.OT_KERNEL_BF16))
    by = {a["arm"]: a for a in arms}
    cap_ratio = by["served_backlog"]["solves_per_s"] / by["plain_backlog"]["solves_per_s"]
    return {"workload": f"c5_serving: 64 cells (I in {{5k, 20k, 80k}}, J in {{128, 512, 1024}}), Poisson "
                        f"{rate:g} req/s for {seconds:g} s, devices moving 1-30 m/s, tol {TOL}",
            "offered_per_s": len(t_arr) / seconds, "requests": int(len(t_arr)),
            "served_vs_plain_capacity": cap_ratio, "arms": by, "inputs_s": gen_s,
            "note": "served: ot_assoc_server_* (resident cells, warm starts, continuous batching in one "
                    "persistent launch); plain: ot_assoc_build_cost_mobile + ot_assoc_solve_cost (or "
                    "ot_assoc_solve_lowp BF16) per request in arrival order on one stream; backlog = the "
                    "whole trace submitted at once (capacity); latency = done - arrival"}


def run_c5(args):
    """Serving: 64 cells (I in {5k, 20k, 80k}, J in {128, 512, 1024}), devices moving 1-30 m/s,
    Poisson arrivals at args.c5_rate req/s for args.c5_seconds s, replayed in real time through
    the server and through plain per-instance solves (and as a backlog through both, for
    capacity); --c5-sweep adds the server at several offered rates (fractions of its capacity)."""
    pool = _pool(min(16, os.cpu_count() or 1))
    import torch  # noqa: F401
    from paper_1805_01559_gb300 import binding
    from paper_1805_01559_gb300 import instances as ins
    ctx = binding.Context(0)
    clocks = ClockSampler(0)
    clocks.start()
    rec = serving_record(ctx, pool, args.c5_rate, args.c5_seconds, args.c5_group)
    sweep = []
    if args.c5_sweep:
        cells = _c5_cells(ins.serving_cell_shapes(64), pool)
        cap = rec["arms"]["served_backlog"]["solves_per_s"]
        for frac in (0.5, 0.8, 0.95):
            t_arr, cidx = ins.poisson_arrivals(frac * cap, args.c5_seconds, len(cells), seed=1)
            r = _serve_run(ctx, cells, t_arr, cidx, True, args.c5_group)
            r["offered_fraction_of_capacity"] = frac
            r["offered_per_s"] = len(t_arr) / args.c5_seconds
            sweep.append(r)
    pool.close()
    clk = clocks.stop()
    served = rec["arms"]["served"]
    line = {"metric": "served solves/s", "value": served["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": served["requests"], "warmup": 0, "ms_per_step": served["latency_ms"]["mean"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rec["workload"], "group_ctas": args.c5_group},
            "serving": rec, "load_sweep": sweep, "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_alg2(args):
    """Algorithm 2 (adaptive Sinkhorn association) on the 50,000 x 800 hot-spot instance:
    `--alg2-outer` outer steps at eps = 0.1 median(C), delta = 5% of one RRH's equal share,
    in one persistent launch; against the same steps driven from the host (one solve per
    step, argmax and the q update on the host)."""
    import torch

    from paper_1805_01559_gb300 import binding
    inst = make_inputs()
    I, J = inst.I, inst.J
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    G = torch.from_numpy(np.ascontiguousarray(inst.G, dtype=np.float32)).to(dev)
    R = ctx.build_rates(G, torch.from_numpy(inst.P.astype(np.float32)).to(dev), inst.N0, inst.W_hz)
    C, med = ctx.build_cost(R, inst.mu, eps_rel=1.0)
    del G, R
    lam = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    eps = 0.1 * med
    outer = args.alg2_outer
    delta = 0.05 * float(inst.lam.sum()) / J
    s = torch.cuda.current_stream()

    def fused():
        return ctx.adaptive(C, lam, eps, delta, outer, tol=TOL, max_iter=MAX_ITER)

    def host_loop():
        q = np.full(J, float(inst.lam.astype(np.float32).astype(np.float64).sum()) / J)
        g = None
        its, ml = [], []
        for k in range(outer):
            r = ctx.solve_cost(C, lam, torch.from_numpy(q.astype(np.float32)).to(dev), eps, tol=TOL,
                               max_iter=MAX_ITER, warm_g=g)
            g = r.g
            rho = r.rrh_load.cpu().numpy()
            js = int(np.argmax(rho))
            its.append(r.iters)
            ml.append(float(rho[js]))
            if k + 1 < outer:
                d = delta if delta < q[js] else 0.5 * q[js]
                q = np.where(np.arange(J) == js, q - d, q + d / (J - 1))
        return its, ml

    for _ in range(args.warmup):
        fused()
        host_loop()
    ms_f, ms_h, iters = [], [], None
    ctx.enable_timing(False)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = ctx.launch_count()
    for _ in range(args.steps):
        res, ms, _ = _timed(fused, s)
        ms_f.append(ms)
    launches = (ctx.launch_count() - l0) / args.steps
    clk = clocks.stop()
    for _ in range(max(1, args.steps // 2)):
        (its_h, ml_h), ms, _ = _timed(host_loop, s)
        ms_h.append(ms)
    iters = [st["iters"] for st in res.steps]
    ml = [st["max_load"] for st in res.steps]
    ms = statistics.median(ms_f)
    cells_iters = float(I) * J * sum(iters)
    alg_bytes = 4.0 * I * J * sum(it + 2 for it in iters)
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": cells_iters / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"alg2_adaptive_50000x800: {outer} outer steps, eps = 0.1 median(C), "
                                   f"delta = 5% of an equal share", "I": I, "J": J, "outer": outer, "tol": TOL,
                       "l2": "C (160 MB) larger than L2"},
            "outer_steps_per_s": outer / (ms / 1e3),
            "host_loop": {"ms": statistics.median(ms_h), "iters": its_h, "max_load_last": ml_h[-1],
                          "fused_speedup": statistics.median(ms_h) / ms},
            "iters": iters, "max_load": {"first": ml[0], "last": ml[-1], "min": min(ml)},
            "jstar": [st["jstar"] for st in res.steps],
            "roofline": {"bound": "hbm", "kernel": "sk_adaptive (whole launch)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "alg_bytes_per_launch": alg_bytes},
            "gpu_launches": launches, "clocks": clk}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_policies(args):
    """Sec. IV's uniform-traffic comparison: 25 RRHs in 1 km^2, N devices, policies (a)
    maxSINR, (b) OT Euclidean cost + equal RRH traffic, (c) OT load cost + equal traffic,
    (d) OT load cost + q = Lambda (Lemma 1); completion-time ratios to (a).  All cells' OT
    solves run as one batched launch."""
    import torch

    from paper_1805_01559_gb300 import binding, instances as ins, policies
    ctx = binding.Context(0)
    sizes = (100, 200, 500, 1000, 2000, 5000)
    seeds = range(args.policy_seeds)
    cells = [(N, sd, ins.policy_cell(N, sd)) for N in sizes for sd in seeds]
    s = torch.cuda.current_stream()
    t0 = time.perf_counter()
    preps = [policies.prepare(ctx, c, load_target=0.3, eps_best=0.01, tol=TOL, max_iter=MAX_ITER)
             for _, _, c in cells]
    prep_s = time.perf_counter() - t0
    insts = [x for p in preps for x in p.instances]
    for _ in range(args.warmup):
        ctx.solve_batched(insts)
    ms_all = []
    for _ in range(args.steps):
        res, ms, _ = _timed(lambda: ctx.solve_batched(insts), s)
        ms_all.append(ms)
    ms = statistics.median(ms_all)
    t1 = time.perf_counter()
    out = [policies.finish(ctx, p, res[3 * k: 3 * k + 3]) for k, p in enumerate(preps)]
    fin_s = time.perf_counter() - t1
    table = {}
    for N in sizes:
        rs = [o for (n, _, _), o in zip(cells, out) if n == N]
        row = {}
        for k in "bcd":
            v = np.array([o.ratio[k] for o in rs])
            fin = v[np.isfinite(v)]
            row[k] = {"median": float(np.median(v)) if len(v) else None,
                      "median_finite": float(np.median(fin)) if len(fin) else None,
                      "unstable": int((~np.isfinite(v)).sum())}
        table[str(N)] = row
    cells_iters = sum(x.C.shape[0] * x.C.shape[1] * r.iters for x, r in zip(insts, res))
    line = {"metric": "policy OT solves/s", "value": len(insts) / (ms / 1e3), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"policies_25rrh: N in {list(sizes)}, {len(seeds)} drops each, "
                                   f"{len(insts)} OT solves in one batched launch",
                       "load_target": 0.3, "eps": "0.01 x mean cheapest-link cost", "tol": TOL,
                       "max_iter": MAX_ITER},
            "cells_iters_per_s": cells_iters / (ms / 1e3),
            "completion_time_ratio_to_maxsinr": table,
            "prepare_s": prep_s, "finish_s": fin_s,
            "not_converged": int(sum(1 for r in res if not r.converged))}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_euclid(args):
    """The Euclidean cost of Sec. IV (cost choice (i)) on the 50,000 x 800 geometry: Algorithm 1
    with C formed inside every sweep from the coordinates (no matrix read), at eps = {0.1,
    0.03, 0.01} x median(C); against the same solves on the materialized matrix."""
    import torch

    from paper_1805_01559_gb300 import binding, instances as ins
    inst = ins.make_instance("c2_50000x800", 50_000, 800, 2000.0, 0, hotspot=True, traffic_sigma=1.5,
                             marginal="capacity", eps_rel=EPS_REL, dtype=np.float32, keep_geometry=True)
    I, J = inst.I, inst.J
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    dxy = torch.from_numpy(np.ascontiguousarray(inst.dev_xy, np.float32)).to(dev)
    rxy = torch.from_numpy(np.ascontiguousarray(inst.rrh_xy, np.float32)).to(dev)
    lam = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    C = ctx.euclid_cost(dxy, rxy)
    med = ctx.median_f32(C.contiguous().view(-1))
    s = torch.cuda.current_stream()

    def fly():
        return [ctx.solve_euclid(dxy, rxy, lam, q, er * med, tol=TOL, max_iter=MAX_ITER).iters for er in EPS_REL]

    def mat():
        return [ctx.solve_cost(C, lam, q, er * med, tol=TOL, max_iter=MAX_ITER).iters for er in EPS_REL]

    for _ in range(args.warmup):
        fly()
        mat()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = ctx.launch_count()
    ms_f = []
    its = None
    for _ in range(args.steps):
        its, ms, _ = _timed(fly, s)
        ms_f.append(ms)
    launches = (ctx.launch_count() - l0) / args.steps
    clk = clocks.stop()
    ms_m = []
    its_m = None
    for _ in range(max(1, args.steps // 2)):
        its_m, ms, _ = _timed(mat, s)
        ms_m.append(ms)
    ms = statistics.median(ms_f)
    ci = float(I) * J * sum(its)
    # two SFU operations a cell and sweep (the exponential and the square root's reciprocal
    # square root) against the device's measured exp2 rate; and the issue bound of the
    # kernel's instruction mix: 152 SMs x 4 schedulers x 1 warp instruction a clock x
    # 2.07 GHz / (warp instructions per cell and sweep, counted by ncu).  The lower binds.
    ex2_rate = ctx.measure_ex2_rate()
    sfu_cells = ex2_rate / 2
    wi = stored_euclid_inst()
    issue_cells = 152 * 4 * 2.07e9 / wi if wi else None
    if issue_cells and issue_cells < sfu_cells:
        peak_cells, peak_kind = issue_cells, (f"derived: issue bound, 152 SMs x 4 warp instructions/clk x 2.07 GHz / "
                                              f"{wi:.4f} warp instructions per cell and sweep (ncu count)")
    else:
        peak_cells, peak_kind = sfu_cells, (f"measured: {ex2_rate:.3g} exp2/s (ot_assoc_measure_ex2_rate) / 2 SFU "
                                            "ops per cell")
    sweeps = sum(it + 2 for it in its)
    achieved = float(I) * J * sweeps / (ms / 1e3)
    line = {"metric": METRIC, "value": ci / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "euclid_50000x800: Sinkhorn with C_ij = |x_i - x_j| formed in the sweep, "
                                   "eps = {0.1,0.03,0.01} x median(C)", "I": I, "J": J, "iters": its, "tol": TOL,
                       "l2": "no matrix is read"},
            "materialized": {"ms": statistics.median(ms_m), "iters": its_m,
                             "cells_iters_per_s": float(I) * J * sum(its_m) / (statistics.median(ms_m) / 1e3)},
            "roofline": {"bound": "alu", "kernel": "sk_solve_euclid (cost, ex2 and the square root formed per cell)",
                         "achieved": achieved, "peak": peak_cells, "unit": "cells*sweeps/s",
                         "frac": achieved / peak_cells, "traffic": None, "peak_kind": peak_kind,
                         "sfu_bound": sfu_cells, "issue_bound": issue_cells},
            "gpu_launches": launches, "clocks": clk}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args):
    """The row-sharded form of Algorithm 1 (ot_assoc_shard_*, sharded.solve_sharded) on the
    50,000 x 800 step's instance at eps = {0.1, 0.03, 0.01} x median(C): the rows split into
    --shards blocks, emulated in this process on the one GPU (each shard its own launches, the
    sum over the shards formed between launches), against the single-GPU persistent solve.
    One rank of a multi-GPU run does the work of one shard plus one all-reduce of J + 1
    doubles per iteration; here every shard runs on the same GPU, one after the other."""
    import torch

    from paper_1805_01559_gb300 import binding, sharded as S
    inst = make_inputs()
    I, J = inst.I, inst.J
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    G = torch.from_numpy(np.ascontiguousarray(inst.G, np.float32)).to(dev)
    P = torch.from_numpy(inst.P.astype(np.float32)).to(dev)
    lam = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    C, med = ctx.build_cost_from_gains(G, P, inst.N0, inst.W_hz, inst.mu, eps_rel=1.0)
    cuts = [round(I * k / args.shards) for k in range(args.shards + 1)]
    shards = [(C[cuts[k]:cuts[k + 1]], lam[cuts[k]:cuts[k + 1]]) for k in range(args.shards)]
    ops = S.DeviceOps(ctx)
    s = torch.cuda.current_stream()

    def sharded():
        return [S.solve_sharded(ops, shards, q, er * med, tol=TOL, max_iter=MAX_ITER).iters for er in EPS_REL]

    def single():
        return [ctx.solve_cost(C, lam, q, er * med, tol=TOL, max_iter=MAX_ITER).iters for er in EPS_REL]

    for _ in range(args.warmup):
        sharded()
        single()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = ctx.launch_count()
    ms_s, its = [], None
    for _ in range(args.steps):
        its, ms, _ = _timed(sharded, s)
        ms_s.append(ms)
    launches = (ctx.launch_count() - l0) / args.steps
    clk = clocks.stop()
    ms_1, its_1 = [], None
    for _ in range(args.steps):
        its_1, ms, _ = _timed(single, s)
        ms_1.append(ms)
    ms, ms1 = statistics.median(ms_s), statistics.median(ms_1)
    ci = float(I) * J * sum(its)
    peak, peak_kind = _peaks()
    # every iteration reads C once, plus iteration 1's and the finalize's reads
    sweeps = sum(it + 2 for it in its)
    achieved = 4.0 * I * J * sweeps / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": ci / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"sharded_50000x800: rows in {args.shards} shards on one GPU, "
                                   "eps = {0.1,0.03,0.01} x median(C)", "I": I, "J": J, "shards": args.shards,
                       "iters": its, "tol": TOL, "l2": "inputs larger than L2 (C 160 MB)"},
            "single_gpu_solve": {"ms": ms1, "iters": its_1, "cells_iters_per_s": float(I) * J * sum(its_1) / (ms1 / 1e3)},
            "roofline": {"bound": "hbm", "kernel": "k_shard_sweep (+ k_shard_reduce, k_shard_update per iteration)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": peak_kind,
                         "definition": "4 B x I x J x (iters + 2) over the call (every sweep reads C once)"},
            "gpu_launches": launches, "clocks": clk}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_oracle(args):
    """The FP64 oracle's own speed on the host cores, all of them and one (CPU only; run on the
    GPU machine's host so that the numbers describe the cores beside the GPU): the 1000 x 50
    instance solved to tol; the 50,000 x 800 step's instance at eps = 0.1 median(C), to tol on
    all cores and 2 iterations on one; a 20,000 x 512 sample of the 400,000 x 4,096
    configuration, to tol on all cores and 20 iterations on one; the whole 400,000 x 4,096
    instance, 2 iterations on all cores (its eps from a 1% row sample of C: only the timing
    matters).  Bounded so that the run takes a few minutes."""
    import oracle
    from paper_1805_01559_gb300 import instances as ins
    nall = oracle.num_threads()

    def solve(C, p, q, eps, tol, iters, threads):
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        _, _, it, _ = oracle.sinkhorn(C, p, q, eps, tol, iters)
        dt = time.perf_counter() - t0
        return {"threads": threads, "iters": int(it), "tol": tol, "s": dt,
                "cells_iters_per_s": float(C.shape[0]) * C.shape[1] * it / dt}

    def cost64(G, P, N0, W, mu):
        return oracle.cost(oracle.rates(np.asarray(G, np.float64), P, N0, W), mu)

    res = {}
    inst = ins.config1()
    C = cost64(inst.G, inst.P, inst.N0, inst.W_hz, inst.mu)
    eps = inst.eps_rel[0] * oracle.median(C)
    res["c1_1000x50"] = [solve(C, inst.lam, inst.q, eps, TOL, MAX_ITER, n) for n in (nall, 1)]
    inst = make_inputs()
    C = cost64(inst.G, inst.P, inst.N0, inst.W_hz, inst.mu)
    eps = 0.1 * oracle.median(C)
    res["c2_50000x800_eps0.1"] = [solve(C, inst.lam, inst.q, eps, TOL, MAX_ITER, nall),
                                  solve(C, inst.lam, inst.q, eps, 0.0, 2, 1)]
    inst = ins.make_instance("c4_sub", 20000, 512, 4000.0 * np.sqrt(20000 / 400000), 4, hotspot=True,
                             traffic_sigma=1.5, marginal="capacity", dtype=np.float32)
    C = cost64(inst.G, inst.P, inst.N0, inst.W_hz, inst.mu)
    eps = 0.05 * oracle.median(C)
    res["c4_sample_20000x512"] = [solve(C, inst.lam, inst.q, eps, TOL, MAX_ITER, nall),
                                  solve(C, inst.lam, inst.q, eps, 0.0, 20, 1)]
    del C
    I, J, block = args.c4_rows, 4096, 8192
    inst = ins.config4_blocked(0, I, J, block)
    C = np.empty((I, J), np.float64)
    oracle.set_threads(nall)
    t0 = time.perf_counter()
    pool = _pool(min(16, os.cpu_count() or 1))
    try:
        for b, G in pool.imap_unordered(_gen_c4_block, [(0, I, J, block, b) for b in range(inst.nblocks)]):
            C[b * block:b * block + G.shape[0]] = oracle.cost(oracle.rates_total(G, inst.P, inst.N0, inst.W_hz),
                                                              inst.mu)
    finally:
        pool.close()
    gen_s = time.perf_counter() - t0
    eps = 0.05 * oracle.median(C[::100])
    res[f"c4_{I}x{J}"] = [solve(C, inst.lam, inst.q, eps, 0.0, 2, nall)]
    del C
    oracle.set_threads(nall)
    c2 = res["c2_50000x800_eps0.1"][0]
    line = {"metric": "oracle cells*iters/s", "value": c2["cells_iters_per_s"], "unit": "cells*iters/s",
            "n_gpus": 0, "steps": 1, "warmup": 0, "ms_per_step": c2["s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "oracle timing: c1, the 50,000 x 800 step's first eps, a 20,000 x 512 sample "
                                   "and the whole 400,000 x 4,096 instance; all host cores and one",
                       "cores": nall, "c4_inputs_s": gen_s},
            "oracle_timing": res}
    print(json.dumps(line), flush=True)
    return 0


def run_epsscale(args):
    """eps-scaling on the 50,000 x 800 step's instance: Algorithm 1 at eps = e x median(C)
    from b = 1 (sk_solve) against the same eps reached through the stages 0.1 -> 0.03 -> ...
    -> e x median (sk_eps_scaling, one launch, each stage warm-started from the previous
    stage's g, intermediate stages to tol 1e-3, the last to the step's tol), for every e in
    --eps-final (the regime question: where do the stages pay)."""
    import torch

    from paper_1805_01559_gb300 import binding
    inst = make_inputs()
    I, J = inst.I, inst.J
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    G = torch.from_numpy(np.ascontiguousarray(inst.G, dtype=np.float32)).to(dev)
    P = torch.from_numpy(inst.P.astype(np.float32)).to(dev)
    lam = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    C, med = ctx.build_cost_from_gains(G, P, inst.N0, inst.W_hz, inst.mu, eps_rel=1.0)
    eps0, factor = 0.1 * med, 0.3
    s = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    peak, peak_kind = _peaks()
    regimes = []
    for e_rel in [float(x) for x in args.eps_final.split(",")]:
        eps = e_rel * med

        def direct():
            r = ctx.solve_cost(C, lam, q, eps, tol=TOL, max_iter=args.eps_max_iter)
            return [r.iters], r.transport_cost, r.status

        def staged():
            r, stages = ctx.solve_eps_scaling(C, lam, q, eps, eps0, factor=factor, tol_stage=1e-3, tol=TOL,
                                              max_iter=args.eps_max_iter)
            return stages, r.transport_cost, r.status

        for _ in range(args.warmup):
            direct()
            staged()
        out = {}
        for name, fn in (("direct", direct), ("eps_scaling", staged)):
            ms_all, its, cost, st = [], None, None, None
            for _ in range(args.steps):
                (its, cost, st), ms, _ = _timed(fn, s)
                ms_all.append(ms)
            ms = statistics.median(ms_all)
            sweeps = sum(it + 2 for it in its)  # each stage: its iterations, the first and the finalize sweep
            out[name] = {"ms": ms, "iters": its, "transport_cost": cost, "status": st,
                         "hbm_gbs": 4.0 * I * J * sweeps / (ms / 1e3) / 1e9}
        regimes.append({"eps_rel": e_rel, **out, "speedup_vs_direct": out["direct"]["ms"] / out["eps_scaling"]["ms"],
                        "cost_rel_diff": abs(out["direct"]["transport_cost"] - out["eps_scaling"]["transport_cost"])
                        / out["direct"]["transport_cost"]})
    clk = clocks.stop()
    st = regimes[0]["eps_scaling"]
    line = {"metric": METRIC, "value": float(I) * J * sum(st["iters"]) / (st["ms"] / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": st["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "epsscale_50000x800: eps = e x median(C), direct vs stages from 0.1 x median",
                       "I": I, "J": J, "tol": TOL, "tol_stage": 1e-3, "factor": factor,
                       "max_iter": args.eps_max_iter, "l2": "inputs larger than L2 (C 160 MB)"},
            "regimes": regimes,
            "roofline": {"bound": "hbm", "kernel": "sk_eps_scaling (whole call, CUDA events on its stream)",
                         "achieved": st["hbm_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": st["hbm_gbs"] / peak, "traffic": None, "peak_kind": peak_kind},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--multi", action="store_true",
                    help="c2: the two smaller eps in one launch sharing each read of C")
    ap.add_argument("--ref-rows", type=int, default=12_500)
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="only run this many rounds of the three solves of one step (for profiler captures)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "alg2", "policies", "euclid", "epsscale", "sharded", "oracle"],
                    help="c2: the headline line; c3 batched ragged; c4 stored-kernel precision; c5 serving; "
                         "alg2 adaptive association (Algorithm 2)")
    ap.add_argument("--alg2-outer", type=int, default=20)
    ap.add_argument("--policy-seeds", type=int, default=8)
    ap.add_argument("--c3-instances", type=int, default=256)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--c4-rows", type=int, default=400_000)
    ap.add_argument("--shards", type=int, default=2, help="sharded workload: row blocks on the one GPU")
    ap.add_argument("--c5-rate", type=float, default=2000.0)
    ap.add_argument("--c5-seconds", type=float, default=10.0)
    ap.add_argument("--c5-group", type=int, default=38)
    ap.add_argument("--c5-sweep", action="store_true")
    ap.add_argument("--eps-final", default="0.01", help="final eps / median(C) values of --workload epsscale")
    ap.add_argument("--eps-max-iter", type=int, default=MAX_ITER)
    ap.add_argument("--sub-records", type=int, default=1,
                    help="attach the batched and serving records to the default line (1) or not (0)")
    ap.add_argument("--sub-c3-instances", type=int, default=64)
    ap.add_argument("--sub-c5-seconds", type=float, default=2.0)
    args = ap.parse_args()
    if args.profile_solves > 0:
        return run_profile_solve(args)
    if args.workload != "c2" and args.impl != "reference":
        return {"c3": run_c3, "c4": run_c4, "c5": run_c5, "alg2": run_alg2,
                "policies": run_policies, "euclid": run_euclid, "epsscale": run_epsscale,
                "sharded": run_sharded, "oracle": run_oracle}[args.workload](args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
