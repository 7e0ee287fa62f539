"""One grid split into slabs along its slowest axis (y in 2D, z in 3D).

The time step is local: a cell's update reads the fields of its own cell and
of cells at most four away (the half-width of the 8th-order staggered
operator, Sec. 3.1), and the relaxation memory variables never leave their
cell.  A grid split into slabs therefore advances each slab as its own
context with four extra rows on every side where it borders another slab.
Before each velocity half step the extra rows of p are copied in from the
neighbours' own rows, before each pressure half step those of v_q; the
slabs' own rows then hold bitwise what one context of the whole grid holds
(the extra rows are computed too and overwritten by the next copy).  The
C-PML of each slab is placed by its position in the whole grid
(fw2_set_subdomain); dt and the C-PML speed c_p are those of the whole grid.

`SlabGroup` runs the slabs as contexts of one device and copies the rows on
that device.  `DistributedSlab` runs one slab per process (one GPU each) and
exchanges the rows with torch.distributed point-to-point messages (NCCL for
device tensors, or gloo through host memory); the partition and exchange
logic (`layout`, `slab_problem`, `exchange`) is plain host code.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

GHOST = 4   # extra rows per shared side: the half-width of the staggered operator


@dataclass
class SlabLayout:
    rank: int
    parts: int
    n_rows: int                 # rows of the whole grid along the slowest axis
    own: Tuple[int, int]        # rows this slab advances, [a, b)
    rows: Tuple[int, int]       # rows of its context, own rows and extra rows, [lo, hi)

    @property
    def ghost_lo(self) -> int:
        return self.own[0] - self.rows[0]

    @property
    def ghost_hi(self) -> int:
        return self.rows[1] - self.own[1]


def split_rows(n_rows: int, parts: int) -> List[Tuple[int, int]]:
    """Contiguous, balanced ranges of rows, one per slab."""
    if parts < 1 or n_rows < parts:
        raise ValueError(f"cannot split {n_rows} rows into {parts} slabs")
    cuts = [n_rows * i // parts for i in range(parts + 1)]
    return [(cuts[i], cuts[i + 1]) for i in range(parts)]


def layout(n_rows: int, parts: int, rank: int, ghost: int = GHOST) -> SlabLayout:
    a, b = split_rows(n_rows, parts)[rank]
    if parts > 1 and b - a < ghost:
        raise ValueError(f"slab {rank} has {b - a} rows, fewer than the {ghost} its neighbours need")
    lo = a - ghost if rank > 0 else 0
    hi = b + ghost if rank < parts - 1 else n_rows
    return SlabLayout(rank, parts, n_rows, (a, b), (lo, hi))


def _slow_coord(idx, shape):
    """Coordinate along the slowest axis of flat cell indices (x fastest)."""
    inner = int(np.prod(shape[:-1]))
    return np.asarray(idx, np.int64) // inner


def slab_problem(prob, lay: SlabLayout):
    """The problem description of one slab: media and relaxation maps cut to
    the context's rows, sources and sensor groups of the own rows only, with
    cell indices local to the slab; dt and c_p those of the whole grid.
    Returns (problem, global group index of each of its sensor groups)."""
    if prob.bc[prob.ndim - 1] == "periodic" and lay.parts > 1:
        raise ValueError("a periodic axis cannot be split into slabs")
    lo, hi = lay.rows
    a, b = lay.own
    shape = tuple(prob.shape)
    inner = int(np.prod(shape[:-1]))
    sub_shape = shape[:-1] + (hi - lo,)

    def cut(arr, lead=0):
        if arr is None:
            return None
        arr = np.asarray(arr)
        sl = (slice(None),) * lead + (slice(lo, hi),)
        return np.ascontiguousarray(arr[sl])
    dt = float(prob.dt)
    if not dt > 0:
        raise ValueError("slabs need the whole grid's time step: set prob.dt")
    cp = float(prob.pml_cp) if prob.pml_cp and prob.pml_cp > 0 else float(np.max(np.asarray(prob.c)))
    repl = dict(shape=sub_shape, dt=dt, pml_cp=cp, c=cut(prob.c), rho=cut(prob.rho), beta=cut(prob.beta),
                kappa1=cut(prob.kappa1), kappa2=cut(prob.kappa2), d1=cut(prob.d1, 1), alpha1=cut(prob.alpha1, 1),
                d2=cut(prob.d2, 1), alpha2=cut(prob.alpha2, 1), tissue=cut(prob.tissue))
    # sources: the entries whose cell is an own row, re-indexed to the slab
    srcs = []
    for s in prob.sources:
        k = _slow_coord(s.idx, shape)
        keep = (k >= a) & (k < b)
        if not np.any(keep):
            continue
        idx = np.asarray(s.idx, np.int64)[keep] - lo * inner
        srcs.append(dataclasses.replace(s, idx=np.ascontiguousarray(idx),
                                        group=np.ascontiguousarray(np.asarray(s.group, np.int32)[keep])))
    repl["sources"] = srcs
    # sensor groups lying in the own rows (a group across two slabs is refused)
    groups = []
    sens = prob.sensors
    if sens is not None:
        k = _slow_coord(sens.idx, shape)
        grp = np.asarray(sens.group, np.int32)
        idx_l, grp_l = [], []
        for g in range(sens.n_groups):
            m = grp == g
            if not np.any(m):
                continue
            inside = (k[m] >= a) & (k[m] < b)
            if np.all(inside):
                idx_l.append(np.asarray(sens.idx, np.int64)[m] - lo * inner)
                grp_l.append(np.full(int(m.sum()), len(groups), np.int32))
                groups.append(g)
            elif np.any(inside):
                raise ValueError(f"sensor group {g} spans two slabs")
        repl["sensors"] = (dataclasses.replace(sens, idx=np.concatenate(idx_l), group=np.concatenate(grp_l),
                                               n_groups=len(groups)) if groups else None)
    return dataclasses.replace(prob, **repl), groups


def velocity_fields(nd: int) -> List[str]:
    return ["v" + "xyz"[q] for q in range(nd)]


def exchange(lay: SlabLayout, fields: Sequence[str], get_rows: Callable, set_rows: Callable,
             send: Callable, recv: Callable):
    """Fill the slab's extra rows of `fields` from its neighbours.

    get_rows(field, r0, n) returns rows of the slab's context, set_rows(field,
    r0, data) writes them (rows local to the context); send(peer, data) and
    recv(peer, like) move one block of rows to or from a neighbouring slab.
    Each side sends its GHOST own rows next to the shared boundary and
    receives the neighbour's into its extra rows."""
    lo = lay.rows[0]
    a, b = lay.own
    g = GHOST
    out = []
    if lay.rank > 0:
        out.append((lay.rank - 1, a - lo, 0))                # own rows [a, a+g) -> lower neighbour
    if lay.rank < lay.parts - 1:
        out.append((lay.rank + 1, b - g - lo, b - lo))       # own rows [b-g, b) -> upper neighbour
    for f in fields:
        pending = []
        for peer, src, _ in out:
            data = get_rows(f, src, g)
            pending.append((send(peer, data), data))     # the block lives until its send completes
        for peer, _, dst in out:
            like = get_rows(f, dst, g)
            set_rows(f, dst, recv(peer, like))
        for w, _ in pending:
            if w is not None and hasattr(w, "wait"):
                w.wait()


class SlabGroup:
    """Slabs of one grid as contexts of one device, rows copied on the device."""

    def __init__(self, prob, parts: int, map_precision: str = "f32", kernel_path: str = "auto"):
        from . import fw2
        import torch
        self.fw2, self.torch = fw2, torch
        self.prob = prob
        self.nd = prob.ndim
        n_rows = prob.shape[-1]
        self.slabs = []
        for r in range(parts):
            lay = layout(n_rows, parts, r)
            sub, groups = slab_problem(prob, lay)
            off = [0] * (self.nd - 1) + [lay.rows[0]]
            sim = fw2.Simulation(sub, map_precision=map_precision, kernel_path=kernel_path,
                                 subdomain=(tuple(prob.shape), off))
            self.slabs.append((lay, sim, groups))
        self.row_cells = int(np.prod(prob.shape[:-1]))

    def _rows(self, sim, f, r0, n):
        t = self.torch.empty((n, self.row_cells), dtype=self.torch.float32, device="cuda")
        self.fw2.fw2_get_rows(sim.ctx, f, r0, n, t)
        return t

    def _exchange(self, fields):
        # every neighbour pair: upper ghost of i <- own rows of i+1, lower ghost of i+1 <- own rows of i
        for i in range(len(self.slabs) - 1):
            la, sa, _ = self.slabs[i]
            lb, sb, _ = self.slabs[i + 1]
            for f in fields:
                up = self._rows(sb, f, lb.own[0] - lb.rows[0], GHOST)
                dn = self._rows(sa, f, la.own[1] - GHOST - la.rows[0], GHOST)
                self.fw2.fw2_set_rows(sa.ctx, f, la.own[1] - la.rows[0], GHOST, up)
                self.fw2.fw2_set_rows(sb.ctx, f, 0, GHOST, dn)

    def step(self, n: int):
        for _ in range(n):
            self._exchange(["p"])
            for _, sim, _ in self.slabs:
                self.fw2.fw2_step_part(sim.ctx, 0)
            self._exchange(velocity_fields(self.nd))
            for _, sim, _ in self.slabs:
                self.fw2.fw2_step_part(sim.ctx, 1)
        return self

    def field(self, name: str) -> np.ndarray:
        """A state array of the whole grid (numpy order), from the own rows."""
        parts = []
        for lay, sim, _ in self.slabs:
            a = sim.field(name)
            lo = lay.rows[0]
            sl = (slice(lay.own[0] - lo, lay.own[1] - lo),)
            parts.append(a[(slice(None),) + sl] if name.startswith("psi") else a[sl])
        return np.concatenate(parts, axis=1 if name.startswith("psi") else 0)

    def trace(self) -> Optional[np.ndarray]:
        """The sensor traces of the whole grid [n_steps][n_groups]."""
        sens = self.prob.sensors
        if sens is None:
            return None
        out = None
        for _, sim, groups in self.slabs:
            if sim.trace is None or not groups:
                continue
            t = sim.trace.cpu().numpy()
            if out is None:
                out = np.zeros((t.shape[0], sens.n_groups), np.float32)
            out[:, groups] = t
        return out

    def close(self):
        for _, sim, _ in self.slabs:
            sim.close()


class DistributedSlab:
    """This process's slab of one grid, exchanging rows with torch.distributed
    (the default process group; NCCL moves device tensors, gloo host ones)."""

    def __init__(self, prob, map_precision: str = "f32", kernel_path: str = "auto", device_exchange: bool = True):
        from . import fw2
        import torch
        import torch.distributed as dist
        self.fw2, self.torch, self.dist = fw2, torch, dist
        self.rank, self.parts = dist.get_rank(), dist.get_world_size()
        self.prob = prob
        self.nd = prob.ndim
        self.lay = layout(prob.shape[-1], self.parts, self.rank)
        sub, self.groups = slab_problem(prob, self.lay)
        off = [0] * (self.nd - 1) + [self.lay.rows[0]]
        self.sim = fw2.Simulation(sub, map_precision=map_precision, kernel_path=kernel_path,
                                  subdomain=(tuple(prob.shape), off))
        self.row_cells = int(np.prod(prob.shape[:-1]))
        self.device = "cuda" if device_exchange else "cpu"

    def _get(self, f, r0, n):
        t = self.torch.empty((n, self.row_cells), dtype=self.torch.float32, device=self.device)
        self.fw2.fw2_get_rows(self.sim.ctx, f, r0, n, t)
        return t

    def _set(self, f, r0, t):
        self.fw2.fw2_set_rows(self.sim.ctx, f, r0, t.shape[0], t)

    def _exchange(self, fields):
        exchange(self.lay, fields, self._get, self._set,
                 lambda peer, t: self.dist.isend(t, peer),
                 lambda peer, like: (lambda buf: (self.dist.recv(buf, peer), buf)[1])(self.torch.empty_like(like)))

    def step(self, n: int):
        for _ in range(n):
            self._exchange(["p"])
            self.fw2.fw2_step_part(self.sim.ctx, 0)
            self._exchange(velocity_fields(self.nd))
            self.fw2.fw2_step_part(self.sim.ctx, 1)
        return self

    def close(self):
        self.sim.close()
