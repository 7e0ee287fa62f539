"""Continuous-batching serving loop over the C ABI.

Simulation requests (2D or 3D problems with a step count) arrive over time.
The server admits waiting requests in arrival order while their device
footprint fits under a memory cap and their cells under a cap on the cells
advanced at once (a few requests share the device, the rest keep their
place in the queue, so the time to result stays close to first-come
first-served at the batched rate), keeps their state resident, and advances
all active requests in slices: the 2D requests and the 3D requests with
bf16 maps together as one fw2 batch (one persistent launch per half step
and group for all of them, rebuilt when the set of active requests changes;
each request's remaining steps are its budget, so a slice is not cut short
for the others when one request ends inside it), other 3D requests each on
its own stream.  A request's result is its sensor trace;
it leaves when its last step is done, freeing memory for waiting requests.
Every request computes exactly what it would compute alone.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import fw2


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    problem: object                # a problem description (synth.Problem shape), or None
    steps: int
    maps: str = "f32"
    # the grid shape, for a request whose problem the server's `prepare`
    # fills in at admission
    shape: Optional[tuple] = None
    # filled by the server
    admitted: Optional[float] = None
    finished: Optional[float] = None
    trace: Optional[np.ndarray] = None

    @property
    def grid(self) -> tuple:
        return tuple(self.problem.shape if self.problem is not None else self.shape)

    @property
    def cells(self) -> int:
        return int(np.prod(self.grid))


def footprint_bytes(prob, maps: str) -> int:
    """Device bytes of a request as the library allocates them (up to
    alignment): the state, the coefficient maps (per cell in float, bf16 or
    FP16; or the index with its per-tissue tables of 21 fields) and the C-PML
    strips (4 arrays of N values per strip cell, in the maps' type; float for
    the index forms)."""
    nd = len(prob.shape)
    n = int(np.prod(prob.shape))
    N = prob.nrelax
    state = (1 + nd + 2 * nd * N) * 4 * n
    es = 2 if maps in ("bf16", "f16") else 4
    if maps in ("idx", "idx16"):
        if maps == "idx":
            tissues, index_bytes = 256, 1
        else:
            tables = getattr(prob, "tables", None)
            tissues = -(-len(tables["c"]) // 4) * 4 if tables else 65536
            index_bytes = 2
        mp = index_bytes * n + 21 * tissues * 4
    else:
        mp = (5 + 4 * N) * es * n
    L = prob.pml_transition + prob.pml_bound
    strips = sum(4 * N * es * 2 * L * n // s for s in prob.shape) if L else 0
    return state + mp + strips


def batchable(r: Request) -> bool:
    """2D requests, and the 3D requests the pipelined 3D half steps take
    (bf16 maps, at most 3 mechanisms, no periodic axis), join the batch; the
    others step on their own."""
    if len(r.grid) == 2:
        return True
    p = r.problem
    return (r.maps == "bf16" and p is not None and p.nrelax <= 3
            and all(b != "periodic" for b in getattr(p, "bc", ("zero",) * 3)))


class Server:
    def __init__(self, cap_bytes: float = 160e9, slice_steps: int = 100,
                 clock: Callable[[], float] = time.perf_counter, max_cells: Optional[int] = 32 << 20,
                 prepare: Optional[Callable[[Request], None]] = None):
        self.cap = cap_bytes
        self.max_cells = max_cells        # None: admission by memory alone
        self.slice = slice_steps
        self.clock = clock
        # called for a request about to be admitted, to fill in its problem;
        # with it, a request's problem is dropped again when it leaves
        self.prepare = prepare
        self.launch_log: List[dict] = []

    def run(self, requests: List[Request]) -> List[Request]:
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        active: List[tuple] = []          # (request, Simulation, remaining, bytes)
        used = 0.0
        batch = None
        batch_members: tuple = ()
        t0 = self.clock()
        done: List[Request] = []
        while pending or active:
            now = self.clock() - t0
            # admission by footprint and cells, in arrival order (one request
            # is always admitted when none is active)
            cells = sum(a[0].cells for a in active)
            while pending and pending[0].arrival <= now:
                r = pending[0]
                over_cells = self.max_cells is not None and cells + r.cells > self.max_cells
                if active and over_cells:
                    break
                if self.prepare is not None and r.problem is None:
                    self.prepare(r)
                fp = footprint_bytes(r.problem, r.maps)
                if active and used + fp > self.cap:
                    break
                pending.pop(0)
                stream = torch.cuda.current_stream() if batchable(r) else torch.cuda.Stream()
                sim = fw2.Simulation(r.problem, map_precision=r.maps, stream=stream)
                r.admitted = self.clock() - t0
                active.append((r, sim, r.steps, fp))
                used += fp
                cells += r.cells
            if not active:
                if pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            two = [a for a in active if batchable(a[0])]
            three = [a for a in active if not batchable(a[0])]
            step2 = min(self.slice, max([a[2] for a in two], default=0))
            members = tuple(a[0].rid for a in two)
            if two and members != batch_members:
                if batch is not None:
                    fw2.fw2_batch_destroy(batch)
                batch = fw2.fw2_batch_create([a[1].ctx for a in two])
                # every request stops at its own last step
                fw2.fw2_batch_set_budget(batch, [a[0].steps for a in two])
                batch_members = members
            if two and step2 > 0:
                fw2.fw2_batch_step(batch, step2)
            steps3 = []
            for a in three:
                k = min(self.slice, a[2])
                a[1].step(k)
                steps3.append(k)
            if two:
                fw2.fw2_batch_synchronize(batch)
            for a in three:
                a[1].synchronize()
            self.launch_log.append({"t": self.clock() - t0, "n_batch": len(two), "n_own": len(three), "steps": step2})
            # bookkeeping
            new_active = []
            i3 = 0
            for a in active:
                r, sim, rem, fp = a
                if batchable(r):
                    rem -= min(step2, rem)
                else:
                    rem -= steps3[i3]
                    i3 += 1
                if rem <= 0:
                    r.trace = sim.trace.cpu().numpy() if sim.trace is not None else None
                    r.finished = self.clock() - t0
                    sim.close()
                    if self.prepare is not None:
                        r.problem = None
                    used -= fp
                    done.append(r)
                else:
                    new_active.append((r, sim, rem, fp))
            active = new_active
        if batch is not None:
            fw2.fw2_batch_destroy(batch)
        return done


def latency_stats(reqs: List[Request]) -> dict:
    ttr = np.array([r.finished - r.arrival for r in reqs])
    return {"p50_s": float(np.percentile(ttr, 50)), "p99_s": float(np.percentile(ttr, 99)),
            "mean_s": float(ttr.mean()), "n": len(reqs)}
