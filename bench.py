#!/usr/bin/env python
"""Throughput of the Fullwave 2 time step on GB300 (one JSON line on stdout).

Workload: the 2D heterogeneous nonlinear abdominal-wall-like medium,
4096 x 4096 cells at lambda/12 for 3 MHz, N = 4 relaxation mechanisms,
fat / muscle / connective layers with beta 4-6, scatterers, 128-element
focused array source and element-mean traces (seeded, synthetic).  A bench
step is one full time step: velocity half step, sources, pressure half step,
recording.  The state (19 float32 arrays, 1.3 GB) plus the coefficient maps
exceed L2, so no flush is needed between steps.

The line carries the roofline of the dominant kernel (compulsory bytes of
the step, charged to the half step that updates each array), the parity of
the reached state against the FP64 oracle on a window, the end-to-end rate
through the C ABI from host buffers, the oracle's own rate on host cores,
and, under `other_configs`, the plain 512^2 method (1000 steps), the 768^3
transcranial medium and the batch of 80 transmit events, each measured the
same way in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fw2|reference]
                  [--workload abdominal|abdominal-idx|skull|plain|batch|serve]
                  [--configs all|none|plain,skull,batch,serve] [--no-parity]
                  [--taps taylor|time-space] [--nl off|pressure|westervelt|literal]

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


def _strip_bytes(shape, N, L, map_bytes):
    """Bytes of the a, b pairs one half step reads for every cell: inside the
    C-PML strip of an axis that axis' set, the interior set when some axis
    is outside its strip."""
    nd = len(shape)
    coef = 0
    for axes_in, cnt in strip_cell_counts(shape, L).items():
        sets = len(axes_in) + (1 if len(axes_in) < nd else 0)
        coef += cnt * sets * 2 * N * map_bytes
    return coef


def algorithmic_bytes(shape, N, L, nl, map_bytes=4, nl_vel=False):
    """Compulsory DRAM bytes of one time step, split into the velocity and the
    pressure half step.

    The minimum for the whole step: every state array (p, v_q, psi1_q^nu,
    psi2_q^nu) read once and written once, every coefficient map read once,
    a, b pairs of an axis from its C-PML strip inside the boundary region.
    Each state array is charged to the half step that updates it: v_q and
    psi1 to the velocity half step (with rho, 1/kappa1, a1, b1 and, for the
    literal nonlinear system's momentum factor, K), p and psi2 to the
    pressure half step (with K, chi, 1/kappa2, a2, b2).  Reading p in the
    velocity half step and v_q in the pressure half step again, as stencil
    operands, is the cost of splitting the step into two launches:
    split_overhead_bytes."""
    nd = len(shape)
    coef = _strip_bytes(shape, N, L, map_bytes)
    n = int(np.prod(shape))
    vel = n * (nd * 8 + nd * N * 8 + map_bytes + map_bytes + (map_bytes if nl_vel else 0)) + coef
    prs = n * (8 + nd * N * 8 + map_bytes + (map_bytes if nl else 0) + map_bytes) + coef
    return vel, prs


def algorithmic_bytes_indexed(shape, N, L, nl, index_bytes=1):
    """As algorithmic_bytes for the tissue-index form: one index per cell
    (uint8, or uint16 with index_bytes = 2) replaces the interior maps (the
    tables live in shared memory or L2) and is charged to the velocity half
    step; cells inside a C-PML strip still read that axis' float a, b."""
    nd = len(shape)
    coef = sum(cnt * len(axes_in) * 2 * N * 4 for axes_in, cnt in strip_cell_counts(shape, L).items())
    n = int(np.prod(shape))
    vel = n * (index_bytes + nd * 8 + nd * N * 8) + coef
    prs = n * (8 + nd * N * 8) + coef
    return vel, prs


def split_overhead_bytes(shape, indexed=False, index_bytes=1):
    """Bytes per launch that the two-launch split reads beyond the step's
    minimum: p again in the velocity half step, v_q again in the pressure
    half step (and the tissue index again there)."""
    n = int(np.prod(shape))
    return 4 * n, 4 * len(shape) * n + (index_bytes * n if indexed else 0)


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

# GB300's nominal HBM3e bandwidth; the roofline's denominator is the measured
# copy bandwidth, this one is reported beside it
NOMINAL_HBM_GBS = 7900.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# sources of each kernel family: a committed traffic figure stays valid while
# the sources of its own family are unchanged
_COMMON_SOURCES = ("async.cuh", "maps.cuh", "tmap.h", "coef.cuh", "fw2_internal.cuh")
_FAMILY_SOURCES = {"pipe2d": ("step2d.cu", "step2d_pipe.cu", "tile2d.cuh"),
                   "pipe3d": ("step3d.cu", "step3d_pipe.cu", "tile2d.cuh")}


def kernel_source_hash(family="pipe2d"):
    h = hashlib.sha256()
    for f in _FAMILY_SOURCES[family] + _COMMON_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_11476_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the
    current sources of the kernel's family (pipe2d or pipe3d, from the key)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    entry = t.get(kernel)
    family = "pipe3d" if ":pipe3d" in kernel else "pipe2d"
    if not entry or entry.get("source_hash") != kernel_source_hash(family):
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


def _round_of(maps):
    """The oracle's model of the maps the kernels stream (the index form's
    coefficients are the float maps gathered from its tables)."""
    return "f32" if maps in ("idx", "idx16") else maps


def _openmp():
    """The OpenMP runtime the oracle's stepper runs its loops on, or None."""
    import ctypes
    try:
        return ctypes.CDLL("libgomp.so.1")
    except OSError:
        return None


def oracle_threads():
    """Threads the oracle's parallel loops use (the OpenMP runtime's count)."""
    omp = _openmp()
    if omp is not None:
        return int(omp.omp_get_max_threads())
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_single_core(orc, steps):
    """`steps` more steps of an oracle run on one thread: the per-core rate
    beside the all-core figure, or None without an OpenMP runtime."""
    omp = _openmp()
    if omp is None or steps < 1:
        return None
    old = int(omp.omp_get_max_threads())
    omp.omp_set_num_threads(1)
    try:
        t0 = time.perf_counter()
        orc.run(steps)
        dt = time.perf_counter() - t0
    finally:
        omp.omp_set_num_threads(old)
    pts = int(np.prod(orc.wshape))
    return {"value": pts * steps / dt / 1e9, "unit": UNIT, "cores": 1,
            "sample": f"the same window, {steps} steps, {dt:.1f} s"}


def oracle_baseline(prob, steps, window, maps="f32", media=True, single_core=True):
    """The FP64 oracle, as it stands, on a window of the workload (host
    cores).  With `media`, the same window is also run on the unrounded
    inputs: how far the stored (float32 or bf16) medium moves the result, a
    property of the input rather than of the kernels."""
    from oracle.core import OracleSim
    orc = OracleSim(prob, round_to=_round_of(maps), window=window)
    orc.run(2)
    t0 = time.perf_counter()
    orc.run(steps)
    dt = time.perf_counter() - t0
    pts = int(np.prod(orc.wshape))
    threads = oracle_threads()
    out = {"value": pts * steps / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{'x'.join(str(w) for w in orc.wshape)} window of the workload around the array "
                     f"(sources inside), {steps} steps, {dt:.1f} s"}
    if media:
        exact = OracleSim(prob, round_to=None, window=window)
        exact.run(2 + steps)
        p0, p1 = exact.field("p"), orc.field("p")
        dev = {"rel_l2": float(np.linalg.norm(p1 - p0) / max(np.linalg.norm(p0), 1e-300)),
               "max_over_peak": float(np.max(np.abs(p1 - p0)) / max(np.max(np.abs(p0)), 1e-300))}
        if orc.trace is not None and orc.trace.size:
            rows = slice(0, 2 + steps)
            e = np.max(np.abs(orc.trace[rows] - exact.trace[rows]))
            dev["trace_db"] = float(20 * math.log10(max(e, 1e-300) / max(np.max(np.abs(exact.trace[rows])), 1e-300)))
        dev["how"] = (f"oracle on the {maps} maps the kernels stream vs the oracle on the unrounded inputs, "
                      f"same window, {2 + steps} steps from rest")
        out["media_deviation"] = dev
    if single_core and threads > 1:
        # about 5 s on one core, estimated from the all-core rate (one core
        # runs at least 1/threads of it), at most half the sample's steps
        per_core = out["value"] * 1e9 / threads
        one = oracle_single_core(orc, max(1, min(steps // 2, int(5.0 * per_core / pts))))
        if one is not None:
            out["single_core"] = one
    return out


def exact_region(window, shape, margin):
    """Slices (numpy order) of the part of a window at least `margin` cells
    from every edge where the window cuts the grid (edges on the grid's own
    boundary need no margin)."""
    sl = []
    for (w0, w1), n in zip(window, shape):
        lo = w0 + (margin if w0 > 0 else 0)
        hi = w1 - (margin if w1 < n else 0)
        sl.append(slice(lo - w0, max(hi, lo) - w0))
    return tuple(reversed(sl)), [(w0 + s.start, w0 + s.stop) for (w0, _), s in zip(window, sl)]


def parity_after_run(sim, prob, maps, window, extra=4):
    """Parity of the timed run: the state the kernels reached is cut to
    `window`; the kernels then take `extra` more steps on the whole grid,
    and the FP64 oracle takes them on the window from the same state.
    Compared where the window is exact (8 cells per step from its cut
    edges): rel L2 and max |error| / peak of p and v_q, and the trace error
    [dB] of the sensor groups that lie entirely in that region."""
    from oracle.core import OracleSim
    from paper_2106_11476_gb300 import fw2
    names = ["p"] + ["v" + "xyz"[q] for q in range(prob.ndim)]
    if prob.nrelax:
        names += [f"psi{o}{'xyz'[q]}" for o in (1, 2) for q in range(prob.ndim)]
    sim.synchronize()
    n0 = fw2.fw2_get_step(sim.ctx)
    state = {nm: sim.field_window(nm, window) for nm in names}
    sim.step(extra)
    sim.synchronize()
    orc = OracleSim(prob, round_to=_round_of(maps), window=window)
    orc.set_state(state, step=n0)
    orc.run(extra)
    sl, region = exact_region(window, prob.shape, 8 * extra)
    err2 = ref2 = 0.0
    emax = peak = 0.0
    for nm in names[:1 + prob.ndim]:
        g = sim.field_window(nm, window)[sl].astype(np.float64)
        o = orc.field(nm)[sl]
        err2 += float(np.sum((g - o) ** 2))
        ref2 += float(np.sum(o ** 2))
        emax = max(emax, float(np.max(np.abs(g - o))) / max(float(np.max(np.abs(o))), 1e-300))
    out = {"rel_l2": math.sqrt(err2 / max(ref2, 1e-300)), "max_over_peak": emax, "trace_db": None,
           "steps_compared": extra, "window": [list(w) for w in window],
           "region": [list(r) for r in region]}
    sn = prob.sensors
    if sn is not None and sim.trace is not None and n0 + extra <= sim.trace.shape[0]:
        full = list(prob.shape) + [1] * (3 - prob.ndim)
        i = sn.idx % full[0]
        j = (sn.idx // full[0]) % full[1]
        k = sn.idx // (full[0] * full[1])
        rr = region + [(0, 1)] * (3 - prob.ndim)
        inside = ((i >= rr[0][0]) & (i < rr[0][1]) & (j >= rr[1][0]) & (j < rr[1][1])
                  & (k >= rr[2][0]) & (k < rr[2][1]))
        groups = [gi for gi in range(sn.n_groups) if np.all(inside[sn.group == gi]) and np.any(sn.group == gi)]
        if groups:
            tg = sim.trace[n0:n0 + extra].cpu().numpy()[:, groups].astype(np.float64)
            to = orc.trace[n0:n0 + extra][:, groups]
            e = float(np.max(np.abs(tg - to)))
            out["trace_db"] = 20 * math.log10(max(e, 1e-300) / max(float(np.max(np.abs(to))), 1e-300))
            out["trace_groups"] = len(groups)
    out["how"] = (f"state after the timed run cut to the window; {extra} further steps by the kernels on the "
                  f"whole grid and by the FP64 oracle on the window; compared {8 * extra} cells from its cut edges")
    return out


def parity_window(prob):
    """The window of the cpu_baseline sample and of the parity check: 512 x 512
    cells from the grid's y = 0 edge (2D), or the 128^3 box from its z = 0
    face (3D), centred in x (and y) on the source cell that fires first, so
    that the window holds a wavefield however few steps the run takes."""
    n = prob.shape
    x_c, y_c = n[0] // 2, n[1] // 2 if prob.ndim == 3 else 0
    first = None
    for s in prob.sources:
        sig = np.abs(np.asarray(s.signal))
        if sig.size == 0 or sig.max() == 0:
            continue
        on = sig >= 1e-3 * sig.max()
        t_on = np.where(on.any(axis=0), on.argmax(axis=0), sig.shape[0])   # first significant row per column
        col = int(np.argmin(t_on))
        cell = int(np.asarray(s.idx)[np.asarray(s.group) == col][0])
        if first is None or t_on[col] < first[0]:
            first = (int(t_on[col]), cell)
    if first is not None:
        x_c = first[1] % n[0]
        if prob.ndim == 3:
            y_c = (first[1] // n[0]) % n[1]

    def span(c, half, size):
        lo = min(max(c - half, 0), max(size - 2 * half, 0))
        return (lo, min(lo + 2 * half, size))
    if prob.ndim == 2:
        return (span(x_c, 256, n[0]), (0, min(512, n[1])))
    return (span(x_c, 64, n[0]), span(y_c, 64, n[1]), (0, min(128, n[2])))


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, cells: int, steps: int, seconds: float) -> float:
    """Whole-job GPts/s: every rank updates `cells` points `steps` times in the
    slowest rank's `seconds` (weak scaling)."""
    return world * cells * steps / seconds / 1e9


def workload_problem(args, name, n, total_steps, rank):
    """(problem, maps, description) of a single-grid workload."""
    import synth
    if name in ("abdominal-idx", "abdominal-idx16"):
        levels = 64 if name == "abdominal-idx" else 1024
        prob = synth.indexed_abdominal_problem(nx=n, ny=n, n_steps=total_steps, seed=1 + rank, n_elements=128,
                                               focus_mm=40.0, levels=levels)
        maps = args.maps or ("idx" if name == "abdominal-idx" else "idx16")
        desc = (f"2D heterogeneous nonlinear abdominal wall in tissue-index form (class x {levels} scatterer "
                f"levels), {n}x{n} cells at lambda/12 for 3 MHz, N=4, 128-element focused array, {maps} maps")
    elif name == "skull":
        prob = synth.skull_problem(n=n, n_steps=total_steps, seed=2 + rank)
        maps = "bf16"
        desc = (f"3D transcranial-like medium, {n}^3 cells at lambda/10 for 1 MHz, N=3, brain background "
                f"with an ellipsoidal skull shell, 16x16 planar array, bf16 maps")
    elif name == "plain":
        prob = synth.line_source_problem(n=n, n_steps=total_steps, seed=rank)
        maps = args.maps or "f32"
        desc = (f"2D plain method: homogeneous attenuating tissue (N=4, alpha0 0.5, y 1.1), {n}x{n} cells at "
                f"lambda/12 for 3 MHz, linear, line source, 256 point sensors, {maps} maps")
    else:
        prob = synth.abdominal_problem(n=n, n_steps=total_steps, seed=1 + rank)
        maps = args.maps or "f32"
        desc = abdominal_workload(n)
    return prob, maps, desc


def measure(args, prob, maps, desc, steps, warmup, rank, world, dist, want_e2e=True, want_cpu=True,
            want_parity=True, parity_steps=4, name=None):
    """One single-grid workload: warm-up, K timed steps (CUDA events on the
    library's stream, max over ranks), per-kernel event timing for the
    roofline, the parity of the reached state against the oracle, the end
    to end run through the C ABI from pinned host buffers, and the oracle
    baseline.  Returns the fields of a bench line (rank 0) or None."""
    import torch
    import synth
    from paper_2106_11476_gb300 import fw2
    total_steps = warmup + steps
    prob = synth.with_steps(prob, total_steps + (parity_steps if want_parity else 0))
    L = prob.pml_transition + prob.pml_bound
    ib = {"idx": 1, "idx16": 2}.get(maps, 0)
    if ib:
        vel_b, prs_b = algorithmic_bytes_indexed(prob.shape, prob.nrelax, L, prob.nl_mode != "off", index_bytes=ib)
    else:
        vel_b, prs_b = algorithmic_bytes(prob.shape, prob.nrelax, L, prob.nl_mode != "off",
                                         map_bytes={"f32": 4, "bf16": 2, "f16": 2}[maps],
                                         nl_vel=prob.nl_mode == "literal")
    vel_o, prs_o = split_overhead_bytes(prob.shape, indexed=ib > 0, index_bytes=max(ib, 1))
    stream = torch.cuda.current_stream()
    sim = fw2.Simulation(prob, stream=stream, map_precision=maps, kernel_path=args.kernel_path)
    sim.step(warmup)
    sim.synchronize()
    fw2.fw2_profile(sim.ctx, True)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.launches
    with ClockSampler(device_id_for_smi()) as clk:
        for i in range(steps):
            events[i].record(stream)
            sim.step(1)
        events[-1].record(stream)
        torch.cuda.synchronize()
    launches = sim.launches - launches0
    if dist:
        dist.barrier()
    per_step = np.array([events[i].elapsed_time(events[i + 1]) for i in range(steps)])
    elapsed_ms = float(events[0].elapsed_time(events[-1]))
    vel_ms, nv, prs_ms, np_ = fw2.fw2_profile_read(sim.ctx)
    fw2.fw2_profile(sim.ctx, False)
    nd = prob.ndim
    layout = fw2.fw2_pipe_layout(sim.ctx) if nd == 3 else None
    if fw2.fw2_kernel_path(sim.ctx) == "pipe":
        kv, kp = (f"pipe{nd}d_vel", f"pipe{nd}d_prs")
    else:
        kv, kp = (f"vel{nd}d", f"prs{nd}d")
    elapsed_max = max_over_ranks(elapsed_ms, dist)
    value = job_rate(world, prob.n_pts, steps, elapsed_max * 1e-3)
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    dom = kv if vel_ms / nv >= prs_ms / np_ else kp
    dom_ms = (vel_ms / nv) if dom == kv else (prs_ms / np_)
    dom_bytes, dom_over = (vel_b, vel_o) if dom == kv else (prs_b, prs_o)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    variant = ("" if args.taps == "taylor" else f":{args.taps}") + (f":{args.nl}" if args.nl else "")
    if layout is not None and dom.startswith("pipe3d"):
        variant += ":" + str(layout[0] if dom == kv else layout[1])
    traffic = committed_traffic(f"{name or args.workload}:{maps}:{prob.shape[0]}:{dom}{variant}")
    step_b = vel_b + prs_b
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": int(dom_bytes), "split_overhead_bytes_per_launch": int(dom_over),
            "bytes_basis": "compulsory bytes of the fused step (each state array read and written once, each "
                           "map read once, C-PML strips inside the boundary), charged to the half step that "
                           "updates each array; the second read of the stencil operand that the two-launch "
                           "split makes is split_overhead_bytes_per_launch, not counted",
            "algorithmic_bytes_per_cell_step": round(step_b / prob.n_pts, 2),
            "avg_launch_ms": round(dom_ms, 5),
            "peak_source": f"{peak_kind} copy bandwidth hbm_gbs",
            "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4), "nominal_gbs": NOMINAL_HBM_GBS,
            "step_frac": round(step_b / ((vel_ms / nv + prs_ms / np_) * 1e-3) / 1e9 / peak, 4),
            "step_frac_of_ms_per_step": round(step_b * steps / (elapsed_max * 1e-3) / 1e9 / peak, 4),
            "vel_ms": round(vel_ms / nv, 5), "prs_ms": round(prs_ms / np_, 5)}
    win = parity_window(prob)
    parity = None
    if want_parity and rank == 0 and maps != "f16":
        parity = parity_after_run(sim, prob, maps, win, extra=parity_steps)
    elif want_parity and rank == 0:
        parity = {"skipped": "the FP16 map scales come from the whole grid, which the oracle's window does not "
                             "hold; the tests compare whole grids"}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    e2e = None
    if want_e2e:
        e2e = end_to_end(args, prob, maps, steps, world, dist, stream)
    cpu = None
    if want_cpu and rank == 0 and world == 1:
        cpu = oracle_baseline(prob, args.cpu_steps, win, "f32" if maps == "f16" else maps)
    if rank != 0:
        return None
    return {"value": round(value, 4), "ms_per_step": round(elapsed_max / steps, 5),
            "config": {"workload": desc, "grid": list(prob.shape), "n_relax": prob.nrelax,
                       "nl_mode": prob.nl_mode, "map_precision": maps, "kernel_path": args.kernel_path,
                       "taps": args.taps, "pml_cells": L,
                       **({"pipe_layout": {"velocity": layout[0], "pressure": layout[1]}} if layout else {})},
            "latency": {"p50_ms_per_step": round(float(np.percentile(per_step, 50)), 5),
                        "p99_ms_per_step": round(float(np.percentile(per_step, 99)), 5)},
            "roofline": roof, "parity": parity, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk.summary()}


def end_to_end(args, prob, maps, steps, world, dist, stream):
    """The whole job through the C ABI with host buffers: medium, relaxation
    and sources copied in from pinned host memory, K steps, traces copied
    out, all inside the timed region."""
    import dataclasses
    import torch
    from paper_2106_11476_gb300 import fw2
    pinned = {}

    def pin(a):
        if a is None:
            return None
        t_ = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pinned[id(t_)] = t_
        return t_
    if maps in ("idx", "idx16"):
        tabs = {k: pin(v) for k, v in prob.tables.items()}
        hp = dataclasses.replace(prob, tissue=pin(prob.tissue.astype(np.uint16).view(np.int16)
                                                  if maps == "idx16" else prob.tissue), tables=tabs)
        used = [hp.tissue] + [tabs[k] for k in ("c", "rho", "kappa1", "kappa2", "d1", "alpha1", "d2", "alpha2")]
        if prob.nl_mode != "off":
            used.append(tabs["beta"])
    else:
        hp = dataclasses.replace(prob, c=pin(prob.c), rho=pin(prob.rho), beta=pin(prob.beta),
                                 kappa1=pin(prob.kappa1), kappa2=pin(prob.kappa2), d1=pin(prob.d1),
                                 alpha1=pin(prob.alpha1), d2=pin(prob.d2), alpha2=pin(prob.alpha2))
        used = [x for x in (hp.c, hp.rho, hp.beta, hp.kappa1, hp.kappa2, hp.d1, hp.alpha1, hp.d2, hp.alpha2)
                if x is not None]
    h2d = sum(x.numel() * x.element_size() for x in used)
    h2d += sum(s.idx.nbytes + s.group.nbytes + s.signal.nbytes for s in prob.sources)
    if prob.sensors is not None:
        h2d += prob.sensors.idx.nbytes + prob.sensors.group.nbytes
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    s2 = fw2.Simulation(hp, stream=stream, map_precision=maps, kernel_path=args.kernel_path)
    t_setup = time.perf_counter()
    s2.step(steps)
    trace_host = s2.trace[:steps].cpu() if s2.trace is not None else None
    t1 = time.perf_counter()
    d2h = trace_host.numel() * 4 if trace_host is not None else 0
    s2.close()
    return {"value": job_rate(world, prob.n_pts, steps, max_over_ranks(t1 - t0, dist)), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d // steps), "d2h_bytes_per_step": int(d2h // steps),
            "setup_s": round(t_setup - t0, 3), "steps_and_readback_s": round(t1 - t_setup, 3),
            "scope": "whole job through the C ABI from pinned host buffers: create, set_medium, set_relaxation, "
                     "add_source, record, coefficient build, K steps, trace read-back"}


def run_fw2(args, rank, world, dist):
    import torch
    from paper_2106_11476_gb300 import _build
    _build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = args.n if not (args.workload == "skull" and args.n == 4096) else 768
    if args.workload == "plain" and args.n == 4096:
        n = 512
    prob, maps, desc = workload_problem(args, args.workload, n, args.warmup + args.steps, rank)
    if args.nl:
        prob.nl_mode = args.nl
        desc += f", nonlinear mode {args.nl}"
        if args.nl != "off" and prob.beta is None:
            prob.beta = np.full(prob.grid_shape, 4.0, np.float32)
            desc += " (beta = 4 everywhere)"
    if args.taps == "time-space":
        from paper_2106_11476_gb300 import fw2
        r = float(np.max(prob.c)) * prob.dt / prob.h
        prob.taps = tuple(fw2.fw2_taps_time_space(r, prob.ndim))
        desc += f", time-space optimised taps at r = {r:.3f}"
    res = measure(args, prob, maps, desc, args.steps, args.warmup, rank, world, dist,
                  want_e2e=not args.no_e2e, want_cpu=not args.no_cpu_baseline, want_parity=not args.no_parity)
    del prob
    extras = None
    if args.workload == "abdominal" and args.configs != "none" and world == 1:
        extras = other_configs(args, rank)
    if rank != 0:
        return
    data = ("synthetic (seeded skull-like shell in a brain-like medium; stands in for the micro-CT rat skull)"
            if args.workload == "skull" else
            "synthetic (seeded homogeneous attenuating medium, line source)" if args.workload == "plain" else
            "synthetic (seeded abdominal-wall-like medium; stands in for the Visible Human phantom)")
    res["config"]["l2"] = ("working set within L2 (the HBM roofline is L2-distorted)"
                           if args.workload == "plain" and n <= 1024 else
                           "state and maps exceed L2 (129 MB); no flush needed")
    res["config"]["parallelism"] = f"replicas x{world} (one transmit event per GPU)"
    out = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": data}
    for k in ("config", "latency", "roofline", "parity", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        out[k] = res[k]
    if extras is not None:
        out["other_configs"] = extras
    print(json.dumps(out), flush=True)


def other_configs(args, rank):
    """The other configurations of the workload family, measured in the same
    run (rank 0 of a single-GPU run): the plain 512^2 method for its full
    1000 steps, the 768^3 transcranial medium for K steps, the batch of 80
    transmit events / uneven instances for K steps, and the serving loop on
    the first 16 arrivals of the full-scale request stream."""
    import torch
    out = {}
    sel = args.configs.split(",") if args.configs != "all" else ["plain", "skull", "batch", "serve"]
    if "plain" in sel:
        prob, maps, desc = workload_problem(args, "plain", 512, 1000, rank)
        r = measure(args, prob, maps, desc, 1000 - 20, 20, rank, 1, None, want_e2e=True, want_cpu=False,
                    name="plain")
        r["config"]["l2"] = "working set (about 70 MB) within L2: the HBM roofline is L2-distorted"
        out["plain_512"] = r
        torch.cuda.empty_cache()
    if "skull" in sel:
        prob, maps, desc = workload_problem(args, "skull", 768, args.steps + args.warmup, rank)
        r = measure(args, prob, maps, desc, args.steps, args.warmup, rank, 1, None, want_e2e=False,
                    want_cpu=True, name="skull")
        out["skull_768"] = r
        del prob
        torch.cuda.empty_cache()
    if "batch" in sel:
        out["batch"] = batch_measurement(args, rank, 1, None)
        torch.cuda.empty_cache()
    if "serve" in sel:
        # the first 16 arrivals of the full-scale stream (the whole 200-arrival
        # window runs with --workload serve)
        out["serve_16"] = serve_measurement(args, 16, [20.0], 1.0, rank, 1, None)
        torch.cuda.empty_cache()
    return out


def batch_problems(args, rank):
    """64 focused transmits over one 2048 x 1024 tissue-index medium (seeded
    lateral foci) and 16 tissue-index instances with sides in [512, 1536];
    step budgets: --batch-steps (4000) for every transmit, seeded uniform in
    [1000, 4000] scaled alike for the instances (the uneven lengths of a
    served mix)."""
    import synth
    rng = np.random.default_rng(100 + rank)
    K = args.batch_steps
    steps = max(args.warmup, 13) + K
    probs, budgets = [], []
    for e in range(64):
        probs.append(synth.indexed_abdominal_problem(nx=2048, ny=1024, n_steps=steps, seed=1 + rank,
                                                     n_elements=64, focus_mm=float(rng.uniform(15, 35)),
                                                     focus_x_mm=float(rng.uniform(-10, 10))))
        budgets.append(K)
    for e in range(16):
        nx, ny = (int(v) for v in rng.integers(512, 1537, 2))
        probs.append(synth.indexed_abdominal_problem(nx=nx, ny=ny, n_steps=steps, seed=200 + 16 * rank + e,
                                                     n_elements=16))
        budgets.append(max(1, int(round(K * rng.uniform(0.25, 1.0)))))
    return probs, budgets


def batch_order(probs, budgets):
    """Shortest work (cells x steps) first: the order both forms take the
    problems in, the one that minimises the mean time to result of a
    sequence run at a fixed rate."""
    return sorted(range(len(probs)), key=lambda i: (probs[i].n_pts * budgets[i], i))


def batch_measurement(args, rank, world, dist):
    """Batched tissue-index form vs the plain form (dense float maps, one
    context at a time) on the same 80 problems with the same uneven step
    budgets, both taking them shortest work first.  The batch admits
    problems in that order while at most --batch-cells cells are active
    (paused ones have a budget equal to their step counter): with the gang
    policy a group at a time (the next group once the last member of the
    previous one has left), with the continuous policy whenever the next one
    fits.  A problem leaves when its budget is spent; each one's time to
    result is taken when the batch step it finishes in completes."""
    import torch
    from paper_2106_11476_gb300 import fw2
    probs, budgets = batch_problems(args, rank)
    order = batch_order(probs, budgets)
    work = sum(p.n_pts * n for p, n in zip(probs, budgets))
    sims = [fw2.Simulation(p, map_precision="idx") for p in probs]
    batch = fw2.fw2_batch_create([s.ctx for s in sims])
    warm = max(args.warmup, 13)                          # includes the 13 tuning steps
    fw2.fw2_batch_step(batch, warm)
    fw2.fw2_batch_synchronize(batch)
    grid, tile_order, l0 = fw2.fw2_batch_info(batch)
    edge_weight = fw2.fw2_batch_edge_weight(batch)
    at = [warm] * len(sims)                              # each context's step counter
    last = [warm + n for n in budgets]
    queue, active = list(order), []

    def admit():
        # gang: a new group only when the previous one has left entirely;
        # continuous: whenever the next problem fits
        if args.batch_policy == "gang" and active:
            return
        cells = sum(probs[i].n_pts for i in active)
        while queue and (not active or cells + probs[queue[0]].n_pts <= args.batch_cells):
            i = queue.pop(0)
            active.append(i)
            cells += probs[i].n_pts
        live = set(active)
        fw2.fw2_batch_set_budget(batch, [last[i] if i in live else at[i] for i in range(len(sims))])

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    finish = [None] * len(sims)
    waves = 0
    with ClockSampler(device_id_for_smi()) as clk:
        t0 = time.perf_counter()
        admit()
        while active:
            nxt = min(last[i] - at[i] for i in active)
            fw2.fw2_batch_step(batch, nxt)
            fw2.fw2_batch_synchronize(batch)
            t = time.perf_counter() - t0
            for i in active:
                at[i] += nxt
            done = [i for i in active if at[i] >= last[i]]
            for i in done:
                finish[i] = t
                active.remove(i)
            waves += 1
            admit()
        t_batch = time.perf_counter() - t0
    _, _, l1 = fw2.fw2_batch_info(batch)
    fw2.fw2_batch_destroy(batch)
    for s in sims:
        s.close()
    del sims
    torch.cuda.empty_cache()
    # plain form: the same problems and budgets in the same order, dense
    # float maps, one after the other, each after a short warm-up of its own
    t_plain, plain_finish = 0.0, [None] * len(probs)
    for i in order:
        p, n = probs[i], budgets[i]
        s = fw2.Simulation(p, map_precision="f32")
        s.step(3)
        s.synchronize()
        t1 = time.perf_counter()
        s.step(n)
        s.synchronize()
        t_plain += time.perf_counter() - t1
        s.close()
        plain_finish[i] = t_plain
    t_batch = max_over_ranks(t_batch, dist)
    value = world * work / t_batch / 1e9
    if rank != 0:
        return None
    peaks, _ = measured_peaks()
    vb = sum(n * sum(algorithmic_bytes_indexed(p.shape, p.nrelax, p.pml_transition + p.pml_bound, True))
             for p, n in zip(probs, budgets))
    return {"value": round(value, 4), "unit": UNIT, "steps": args.batch_steps,
            "ms_per_step": round(t_batch / args.batch_steps * 1e3, 4),
            "config": {"workload": "batched: 64 focused transmits over one 2048x1024 tissue-index medium (%d steps "
                                   "each) + 16 instances 512^2..1536^2 (U(0.25, 1) x as many steps), shortest work first, "
                                   % args.batch_steps +
                                   "at most %d active cells (%s admission), contexts leave when their budget is "
                                   "spent, one persistent launch per half step, graph-captured step loop, "
                                   "autotuned launch" % (args.batch_cells, args.batch_policy), "cell_steps": work,
                       "active_cells_cap": args.batch_cells, "admission": args.batch_policy, "segments": waves,
                       "tuned_grid": grid, "tuned_order": tile_order, "tuned_edge_weight": edge_weight},
            "roofline": {"bound": "hbm", "kernel": "step (all kernels)", "unit": "GB/s",
                         "achieved": round(vb / t_batch / 1e9, 1), "peak": float(peaks["hbm_gbs"]),
                         "frac": round(vb / t_batch / 1e9 / float(peaks["hbm_gbs"]), 4),
                         "traffic": None},
            "plain_form": {"value": round(work / t_plain / 1e9, 4), "unit": UNIT,
                           "how": "same problems and budgets, dense float maps, one context at a time, "
                                  "shortest work first, each measured over its full budget"},
            "time_to_result_s": {"batched_p50": round(float(np.percentile(finish, 50)), 3),
                                 "batched_p99": round(float(np.percentile(finish, 99)), 3),
                                 "plain_p50": round(float(np.percentile(plain_finish, 50)), 3),
                                 "plain_p99": round(float(np.percentile(plain_finish, 99)), 3),
                                 "batched_per_context": [round(t, 3) for t in finish],
                                 "plain_per_context": [round(t, 3) for t in plain_finish]},
            "gpu_launches": int(l1 - l0), "clocks": clk.summary()}


def run_batch(args, rank, world, dist):
    import torch
    from paper_2106_11476_gb300 import _build
    _build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = batch_measurement(args, rank, world, dist)
    if rank != 0:
        return
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": r["steps"],
           "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded tissue-index abdominal media)"}
    for k in ("config", "roofline", "plain_form", "time_to_result_s", "gpu_launches", "clocks"):
        out[k] = r[k]
    print(json.dumps(out), flush=True)


def serve_requests(n_requests, scale, rank):
    """Seeded requests of a Poisson stream at one arrival per second (divide
    the arrival times by the rate): 70 % 2D tissue-index abdominal media with
    sides U[512, 4096] and U[1000, 4000] steps, 30 % 3D skull-like media
    (N = 3, bf16 maps) with sides U[256, 512] and U[1000, 2000] steps; `scale`
    < 1 shrinks sides and steps alike.  Each request carries its grid shape
    and a function that generates its problem (a 512^3 medium is 8.6 GB of
    host arrays, so problems are made when they are needed)."""
    import synth
    rng = np.random.default_rng(500 + rank)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0)
        if rng.random() < 0.7:
            side = max(int(rng.integers(512, 4097) * scale) // 4 * 4, 256)
            steps = int(rng.integers(1000, 4001) * scale)
            make = (lambda side=side, steps=steps, i=i: synth.indexed_abdominal_problem(
                nx=side, ny=side, n_steps=steps, seed=1000 + i, n_elements=min(64, side // 24)))
            out.append({"rid": i, "t": t, "shape": (side, side), "steps": steps, "maps": "idx", "make": make})
        else:
            side = max(int(rng.integers(256, 513) * scale), 96)
            steps = int(rng.integers(1000, 2001) * scale)
            make = (lambda side=side, steps=steps, i=i: synth.skull_problem(
                n=side, n_steps=steps, seed=2000 + i, pml_cells=16, array_elems=4))
            out.append({"rid": i, "t": t, "shape": (side, side, side), "steps": steps, "maps": "bf16",
                        "make": make})
    return out


class InputClock:
    """Wall clock that stops while a run waits for a request's problem to be
    generated on the host (input preparation is not the server's work)."""

    def __init__(self):
        self.stopped = 0.0

    def __call__(self):
        return time.perf_counter() - self.stopped


class ProblemFeed:
    """The requests' problems generated in arrival order on one host thread,
    up to `ahead` requests beyond the one asked for; the wait for a problem
    that is not ready yet stops `clock`."""

    def __init__(self, specs, clock, ahead=2):
        from concurrent.futures import ThreadPoolExecutor
        self.specs, self.clock, self.ahead = specs, clock, ahead
        self.pool = ThreadPoolExecutor(1)
        self.futs, self.next = {}, 0
        self.waited = 0.0

    def get(self, i):
        while self.next < len(self.specs) and self.next <= i + self.ahead:
            self.futs[self.next] = self.pool.submit(self.specs[self.next]["make"])
            self.next += 1
        t = time.perf_counter()
        prob = self.futs.pop(i).result()
        dt = time.perf_counter() - t
        self.waited += dt
        if self.clock is not None:
            self.clock.stopped += dt
        return prob

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)


def fcfs_plain(arrivals, durations):
    """Times to result of one-at-a-time service in arrival order."""
    t_free, ttr = 0.0, []
    for a, d in zip(arrivals, durations):
        t_free = max(t_free, a) + d
        ttr.append(t_free - a)
    return ttr, t_free - min(arrivals)


def serve_measurement(args, n_requests, rates, scale, rank, world, dist, sweep_requests=40):
    """The serving loop on a seeded request stream against the plain form
    (each request alone, in arrival order, dense float maps, setup and all
    its steps timed).  The first rate runs all `n_requests` arrivals; each
    further rate (the sweep) the first `sweep_requests`.  The plain form is
    run once; its per-request durations give its first-come first-served
    times to result at every rate.  Problem generation on the host is
    excluded from both forms' clocks."""
    from paper_2106_11476_gb300 import fw2
    from paper_2106_11476_gb300.serve import Request, Server, latency_stats
    specs = serve_requests(n_requests, scale, rank)
    runs = []
    with ClockSampler(device_id_for_smi()) as clk:
        for j, rate in enumerate(rates):
            sub = specs if j == 0 else specs[:min(sweep_requests, n_requests)]
            clock = InputClock()
            feed = ProblemFeed(sub, clock)
            reqs = [Request(q["rid"], q["t"] / rate, None, q["steps"], q["maps"], shape=q["shape"]) for q in sub]
            srv = Server(cap_bytes=160e9, slice_steps=args.slice, clock=clock,
                         prepare=lambda r, feed=feed: setattr(r, "problem", feed.get(r.rid)))
            t0 = clock()
            done = srv.run(reqs)
            makespan = clock() - t0
            feed.close()
            runs.append((rate, sub, done, makespan, feed.waited))
        # plain form: each request alone, in arrival order
        feed = ProblemFeed(specs, None)
        durations = []
        for i, q in enumerate(specs):
            prob = feed.get(i)
            s0 = time.perf_counter()
            sim = fw2.Simulation(prob, map_precision="f32")
            sim.step(q["steps"])
            sim.synchronize()
            sim.close()
            durations.append(time.perf_counter() - s0)
            del prob, sim
        feed.close()
    sweep = []
    for rate, sub, done, makespan, waited in runs:
        work = sum(int(np.prod(q["shape"])) * q["steps"] for q in sub)
        st = latency_stats(done)
        ttr, plain_makespan = fcfs_plain([q["t"] / rate for q in sub], durations[:len(sub)])
        sweep.append({"rate_per_s": rate, "requests": len(sub), "value": round(work / makespan / 1e9, 4),
                      "makespan_s": round(makespan, 3), "p50_s": round(st["p50_s"], 3),
                      "p99_s": round(st["p99_s"], 3),
                      "plain_value": round(work / plain_makespan / 1e9, 4),
                      "plain_p50_s": round(float(np.percentile(ttr, 50)), 3),
                      "plain_p99_s": round(float(np.percentile(ttr, 99)), 3),
                      "input_generation_wait_s": round(waited, 1)})
    head = sweep[0]
    n3 = sum(len(q["shape"]) == 3 for q in specs)
    work = sum(int(np.prod(q["shape"])) * q["steps"] for q in specs)
    return {"value": head["value"], "unit": UNIT,
            "config": {"workload": f"serving: {n_requests} Poisson arrivals at {rates[0]}/s, 70 % 2D tissue-index "
                                   f"(sides 512-4096, 1-4k steps) / 30 % 3D bf16 (sides 256-512, 1-2k steps), "
                                   f"scale {scale}, 160 GB admission cap, at most 32M cells advanced at once, "
                                   f"slices of {args.slice} steps",
                       "requests_2d": n_requests - n3, "requests_3d": n3,
                       "makespan_s": head["makespan_s"], "cell_steps": work,
                       "input_generation": "host problem generation excluded from both forms' clocks"},
            "latency": {"p50_time_to_result_s": head["p50_s"], "p99_time_to_result_s": head["p99_s"]},
            "plain_form": {"value": head["plain_value"], "unit": UNIT,
                           "p50_time_to_result_s": head["plain_p50_s"],
                           "p99_time_to_result_s": head["plain_p99_s"],
                           "how": "one request at a time in arrival order, float maps, each run in full "
                                  "(setup, all its steps); durations measured once, queueing computed per rate"},
            "rate_sweep": sweep[1:],
            "clocks": clk.summary()}


def run_serve(args, rank, world, dist):
    import torch
    from paper_2106_11476_gb300 import _build
    _build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rates = [float(x) for x in args.rates.split(",")]
    r = serve_measurement(args, args.requests, rates, args.serve_scale, rank, world, dist,
                          sweep_requests=args.sweep_requests)
    if rank != 0:
        return
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": None, "warmup": 0,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded request stream)"}
    for k in ("config", "latency", "plain_form", "rate_sweep", "clocks"):
        out[k] = r[k]
    print(json.dumps(out), flush=True)


def abdominal_workload(n):
    return (f"2D heterogeneous nonlinear abdominal wall, {n}x{n} cells at lambda/12 for 3 MHz, "
            f"N=4 mechanisms, beta 4-6, 128-element focused array, element-mean traces, FP32 maps")


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
    threads = oracle_threads()
    sample = f"256x256 window of the {n}x{n} workload around the array, one oracle time step per bench step"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded abdominal-wall-like medium)",
           "config": {"workload": abdominal_workload(n), "grid": [n, n], "n_relax": prob.nrelax,
                      "nl_mode": prob.nl_mode, "map_precision": "f32", "taps": "taylor",
                      "pml_cells": prob.pml_transition + prob.pml_bound,
                      "parallelism": f"replicas x{world} (rank 0 runs the oracle)"},
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
    ap.add_argument("--requests", type=int, default=200, help="serving: number of requests")
    ap.add_argument("--rates", default="20,1,0.5,0.25",
                    help="serving: mean arrivals per second; the first with all --requests arrivals, the others "
                         "(a sweep) with the first --sweep-requests")
    ap.add_argument("--sweep-requests", type=int, default=40, help="serving: arrivals of each sweep rate")
    ap.add_argument("--serve-scale", type=float, default=1.0, help="serving: size and step scale")
    ap.add_argument("--slice", type=int, default=100, help="serving: steps per slice")
    ap.add_argument("--batch-steps", type=int, default=4000, help="batch: steps of each transmit event")
    ap.add_argument("--batch-cells", type=int, default=32 << 20,
                    help="batch: most cells advanced at once (admission in shortest-work-first order)")
    ap.add_argument("--batch-policy", default="gang", choices=["gang", "continuous"],
                    help="batch: admit a group when the previous one has left, or whenever the next problem fits")
    ap.add_argument("--workload", default="abdominal",
                    choices=["abdominal", "abdominal-idx", "abdominal-idx16", "skull", "plain", "batch", "serve"],
                    help="abdominal: 2D 4096^2 nonlinear (default); abdominal-idx: the same in tissue-index "
                         "form; skull: 3D 768^3 with bf16 maps; plain: 2D 512^2 homogeneous line source")
    ap.add_argument("--maps", default=None, choices=["f32", "bf16", "f16", "idx", "idx16"],
                    help="override the map storage of the workload")
    ap.add_argument("--kernel-path", default="auto", choices=["auto", "tile", "pipe", "pipe-staged", "pipe-registers"],
                    help="half-step kernels (bitwise the same results); pipe-staged / pipe-registers fix the layout "
                         "of the 3D pipelined half steps, which auto and pipe choose by timing")
    ap.add_argument("--taps", default="taylor", choices=["taylor", "time-space"],
                    help="staggered taps: 8th-order Taylor, or the time-space optimised set with cross taps")
    ap.add_argument("--nl", default=None, choices=["off", "pressure", "westervelt", "literal"],
                    help="override the workload's nonlinear mode")
    ap.add_argument("--cpu-steps", type=int, default=300,
                    help="oracle steps of the cpu_baseline sample (about 10 s on 16 host cores)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--configs", default="all",
                    help="other configurations measured after the default workload: all, none, or a comma list "
                         "of plain, skull, batch, serve")
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
        if args.workload == "batch":
            run_batch(args, rank, world, dist)
        elif args.workload == "serve":
            run_serve(args, rank, world, dist)
        else:
            run_fw2(args, rank, world, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
