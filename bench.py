#!/usr/bin/env python
"""Throughput of the Fullwave 2 time step on GB300 (one JSON line on stdout).

Workload: the 2D heterogeneous nonlinear abdominal-wall-like medium,
4096 x 4096 cells at lambda/12 for 3 MHz, N = 4 relaxation mechanisms,
fat / muscle / connective layers with beta 4-6, scatterers, 128-element
focused array source and element-mean traces (seeded, synthetic).  A bench
step is one full time step: velocity half step, sources, pressure half step,
recording.  The state (19 float32 arrays, 1.3 GB) plus the coefficient maps
exceed L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fw2|reference]

Under torchrun each rank simulates its own transmit event (independent
problems: weak scaling, no data-path collective); the barrier and the max
over ranks of the timed region follow the benchmark contract.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s (GPts/s) and % HBM roofline at ≤1e-4 rel-L2 vs FP64; p99 latency"
UNIT = "GPts/s"


# --------------------------------------------------------------------------
# algorithmic bytes
# --------------------------------------------------------------------------

def strip_cell_counts(shape, L):
    """Cells of each strip membership class: dict frozenset(axes in strip) -> count."""
    import itertools
    nd = len(shape)
    per_axis = []
    for n in shape:
        s = min(2 * L, n) if L > 0 else 0
        per_axis.append({True: s, False: n - s})
    out = {}
    for combo in itertools.product([False, True], repeat=nd):
        cnt = 1
        for q, inside in enumerate(combo):
            cnt *= per_axis[q][inside]
        out[frozenset(q for q in range(nd) if combo[q])] = cnt
    return out


def algorithmic_bytes(shape, N, L, nl, map_bytes=4):
    """Compulsory DRAM bytes of one launch of the velocity and of the pressure kernel.

    Every streamed array is read once and every updated array written once;
    the stencil operand (p, or v_q) is read once.  Coefficient a, b pairs of
    an axis come from its boundary strip inside the C-PML region, otherwise
    from the interior maps (read once per cell when any axis needs them).
    """
    nd = len(shape)
    classes = strip_cell_counts(shape, L)
    coef = 0
    for axes_in, cnt in classes.items():
        sets = len(axes_in) + (1 if len(axes_in) < nd else 0)
        coef += cnt * sets * 2 * N * map_bytes
    n = int(np.prod(shape))
    vel = n * (4 + map_bytes + map_bytes + nd * 8 + nd * N * 8) + coef
    prs = n * (nd * 4 + map_bytes + (map_bytes if nl else 0) + map_bytes + 8 + nd * N * 8) + coef
    return vel, prs


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("step2d.cu", "step3d.cu", "coef.cuh", "fw2_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2106_11476_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    entry = t.get(kernel)
    if not entry or entry.get("source_hash") != kernel_source_hash():
        return None
    return entry.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.device_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def device_id_for_smi():
    import torch
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis or "0"


def oracle_baseline(prob, steps, window):
    """The FP64 oracle, as it stands, on a window of the workload (host cores)."""
    from oracle.core import OracleSim
    orc = OracleSim(prob, round_to="f32", window=window)
    orc.run(2)
    t0 = time.perf_counter()
    orc.run(steps)
    dt = time.perf_counter() - t0
    pts = int(np.prod(orc.wshape))
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": pts * steps / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{orc.wshape[0]}x{orc.wshape[1]} window of the workload around the array "
                      f"(sources inside), {steps} steps, {dt:.1f} s"}


# --------------------------------------------------------------------------
# arms
# --------------------------------------------------------------------------

def run_fw2(args, rank, world, dist):
    import torch
    import synth
    from paper_2106_11476_gb300 import _build, fw2

    _build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n = args.n
    total_steps = args.warmup + args.steps
    prob = synth.abdominal_problem(n=n, n_steps=total_steps, seed=1 + rank)
    vel_b, prs_b = algorithmic_bytes(prob.shape, prob.nrelax, prob.pml_transition + prob.pml_bound,
                                     prob.nl_mode != "off")
    stream = torch.cuda.current_stream()
    sim = fw2.Simulation(prob, stream=stream)
    sim.step(args.warmup)
    sim.synchronize()
    fw2.fw2_profile(sim.ctx, True)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.launches
    with ClockSampler(device_id_for_smi()) as clk:
        for i in range(args.steps):
            events[i].record(stream)
            sim.step(1)
        events[-1].record(stream)
        torch.cuda.synchronize()
    launches = sim.launches - launches0
    if dist:
        dist.barrier()
    per_step = np.array([events[i].elapsed_time(events[i + 1]) for i in range(args.steps)])
    elapsed_ms = float(events[0].elapsed_time(events[-1]))
    vel_ms, nv, prs_ms, np_ = fw2.fw2_profile_read(sim.ctx)
    fw2.fw2_profile(sim.ctx, False)
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed_max = float(t.item())
    pts = prob.n_pts
    value = world * pts * args.steps / (elapsed_max * 1e-3) / 1e9
    # roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    dom = "vel2d" if vel_ms >= prs_ms else "prs2d"
    dom_ms = (vel_ms / nv) if dom == "vel2d" else (prs_ms / np_)
    dom_bytes = vel_b if dom == "vel2d" else prs_b
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    traffic = committed_traffic(dom)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": round(dom_ms, 5),
            "peak_source": f"{peak_kind} copy bandwidth hbm_gbs",
            "step_roofline_frac": round((vel_b + prs_b) / ((vel_ms / nv + prs_ms / np_) * 1e-3) / 1e9 / peak, 4),
            "vel_ms": round(vel_ms / nv, 5), "prs_ms": round(prs_ms / np_, 5)}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    # end to end through the C ABI with host buffers: medium, relaxation and
    # sources copied in from pinned host memory, K steps, traces copied out
    e2e = None
    if not args.no_e2e:
        pinned = {}
        def pin(a):
            if a is None:
                return None
            t_ = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            pinned[id(t_)] = t_
            return t_
        import dataclasses
        hp = dataclasses.replace(prob, c=pin(prob.c), rho=pin(prob.rho), beta=pin(prob.beta),
                                 kappa1=pin(prob.kappa1), kappa2=pin(prob.kappa2), d1=pin(prob.d1),
                                 alpha1=pin(prob.alpha1), d2=pin(prob.d2), alpha2=pin(prob.alpha2))
        h2d = sum(x.numel() * x.element_size() for x in (hp.c, hp.rho, hp.beta, hp.kappa1, hp.kappa2,
                                                          hp.d1, hp.alpha1, hp.d2, hp.alpha2) if x is not None)
        h2d += sum(s.idx.nbytes + s.group.nbytes + s.signal.nbytes for s in prob.sources)
        h2d += prob.sensors.idx.nbytes + prob.sensors.group.nbytes
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        s2 = fw2.Simulation(hp, stream=stream)
        s2.step(args.steps)
        trace_host = s2.trace[: args.steps].cpu()
        t1 = time.perf_counter()
        d2h = trace_host.numel() * 4
        s2.close()
        te = torch.tensor([t1 - t0], dtype=torch.float64, device="cuda")
        if dist:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * pts * args.steps / float(te.item()) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d // args.steps), "d2h_bytes_per_step": int(d2h // args.steps),
               "scope": "whole job through the C ABI from pinned host buffers: set_medium, set_relaxation, "
                        "add_source, record, coefficient build, K steps, trace read-back"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c0 = n // 2
        cpu = oracle_baseline(prob, args.cpu_steps, ((c0 - 256, c0 + 256), (0, 512)))
    if rank != 0:
        return
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(elapsed_max / args.steps, 5),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded abdominal-wall-like medium; stands in for the Visible Human phantom)",
           "config": {"workload": f"2D heterogeneous nonlinear abdominal wall, {n}x{n} cells at lambda/12 "
                                  f"for 3 MHz, N=4 mechanisms, beta 4-6, 128-element focused array, "
                                  f"element-mean traces, FP32 maps",
                      "grid": [n, n], "n_relax": 4, "nl_mode": prob.nl_mode, "map_precision": "f32",
                      "pml_cells": prob.pml_transition + prob.pml_bound,
                      "l2": "state and maps (>2.5 GB) exceed L2; no flush needed",
                      "parallelism": f"replicas x{world} (one transmit event per GPU)"},
           "latency": {"p50_ms_per_step": round(float(np.percentile(per_step, 50)), 5),
                       "p99_ms_per_step": round(float(np.percentile(per_step, 99)), 5)},
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on a bounded window of the same workload."""
    if rank != 0:
        return
    import synth
    from oracle.core import OracleSim
    n = args.n
    prob = synth.abdominal_problem(n=n, n_steps=args.warmup + args.steps + 2, seed=1)
    c0 = n // 2
    win = ((c0 - 128, c0 + 128), (0, 256))
    orc = OracleSim(prob, round_to="f32", window=win)
    orc.run(args.warmup)
    t0 = time.perf_counter()
    orc.run(args.steps)
    dt = time.perf_counter() - t0
    pts = int(np.prod(orc.wshape))
    value = pts * args.steps / dt / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"256x256 window of the {n}x{n} workload around the array, one oracle time step per bench step"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded abdominal-wall-like medium)",
           "config": {"workload": f"2D heterogeneous nonlinear abdominal wall, {n}x{n} cells, N=4 "
                                  f"(oracle on a 256x256 window)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fw2", choices=["fw2", "reference"])
    ap.add_argument("--n", type=int, default=4096, help="grid side of the workload")
    ap.add_argument("--cpu-steps", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_fw2(args, rank, world, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
