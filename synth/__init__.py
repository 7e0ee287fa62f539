"""Seeded synthetic workloads for the Fullwave 2 step.

This module is shared by the tests, the benchmark and the smoke check.  It
only *describes inputs*: grids, media (sound speed, density, nonlinearity,
relaxation parameters per point), sources, sensors and initial states.  It
holds none of the method's arithmetic (no relaxation coefficients, no PML
profiles, no time stepping); both the CUDA path and the oracle derive
everything else from a :class:`Problem` on their own.

Arrays are numpy, C-ordered as (nz, ny, nx) in 3D, (ny, nx) in 2D and (nx,)
in 1D, so the flat index of cell (i, j, k) is i + nx * (j + ny * k).
Relaxation arrays carry a leading mechanism axis: (N, ...grid).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# Table 2 of the paper: two mechanisms fitted to alpha0 = 0.5 dB/cm/MHz, y = 1
# (kappa_1, kappa_2, d_1^nu, d_2^nu, alpha_1^nu, alpha_2^nu).  Units: d and
# alpha in 1/s, with c = 1540 m/s.
TABLE2 = {
    "kappa1": 0.835, "kappa2": 1.19,
    "d1": [9.82e5, 3.26e6], "alpha1": [2.83e8, 3.54e9],
    "d2": [4.40e4, 1.68e5], "alpha2": [8.35e6, 5.10e7],
    "alpha0": 0.5, "y": 1.0, "c0": 1540.0,
}


def relaxation_sets() -> dict:
    """Fitted relaxation parameter sets (written by oracle/fit_relaxation.py)."""
    path = os.path.join(HERE, "relaxation_sets.json")
    with open(path) as f:
        return json.load(f)


@dataclass
class Source:
    kind: str                 # "p", "vx", "vy" or "vz"
    idx: np.ndarray           # int64 flat cell indices
    group: np.ndarray         # int32 signal column of each index
    signal: np.ndarray        # float32 [n_steps, n_groups]; row n is added at step n


@dataclass
class Sensors:
    idx: np.ndarray           # int64 flat cell indices
    group: np.ndarray         # int32 sensor of each cell (traces average a group)
    n_groups: int


@dataclass
class Problem:
    shape: Tuple[int, ...]    # (nx,), (nx, ny) or (nx, ny, nz); x fastest
    h: float                  # grid spacing [m]
    dt: float                 # time step [s]
    c: np.ndarray             # float32 sound speed [m/s]
    rho: np.ndarray           # float32 density [kg/m^3]
    beta: Optional[np.ndarray] = None   # float32 coefficient of nonlinearity
    nrelax: int = 0
    kappa1: Optional[np.ndarray] = None  # float32 grid
    kappa2: Optional[np.ndarray] = None
    d1: Optional[np.ndarray] = None      # float32 (N, grid)
    alpha1: Optional[np.ndarray] = None
    d2: Optional[np.ndarray] = None
    alpha2: Optional[np.ndarray] = None
    pml_transition: int = 0   # cells
    pml_bound: int = 0        # cells
    pml_rc: float = 1e-3
    pml_npow: float = 2.0
    pml_cp: float = 0.0       # 0: use the largest sound speed of the medium
    pml_reading: str = "C"
    nl_mode: str = "off"      # "off", "pressure", "westervelt" or "literal"
    memory_alignment: str = "centred"   # "centred" or "endpoint" time alignment of the memory term
    bc: Tuple[str, ...] = ("zero", "zero", "zero")
    taps: Optional[Tuple[float, ...]] = None   # (g1, g2, g3, g4, g11); None: 8th-order Taylor
    sources: List[Source] = field(default_factory=list)
    sensors: Optional[Sensors] = None
    n_steps: int = 0
    name: str = ""
    # tissue-index form of the same medium (optional): uint8 or uint16 index per cell
    # and per-tissue tables; the dense arrays above are these tables gathered
    tissue: Optional[np.ndarray] = None
    tables: Optional[dict] = None

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def n_pts(self) -> int:
        return int(np.prod(self.shape))

    @property
    def grid_shape(self) -> Tuple[int, ...]:
        """numpy shape of a field (slowest axis first)."""
        return tuple(reversed(self.shape))


# ----------------------------------------------------------------------------
# signals, sources, sensors
# ----------------------------------------------------------------------------

def gaussian_pulse(n_steps: int, dt: float, f0: float, ncycles: float, amp: float,
                   delay_cycles: Optional[float] = None) -> np.ndarray:
    """Gaussian-windowed sinusoid sampled at t = (n+1) dt, n = 0..n_steps-1."""
    t = (np.arange(n_steps, dtype=np.float64) + 1.0) * dt
    t0 = (delay_cycles if delay_cycles is not None else ncycles) / f0
    tau = ncycles / (2.0 * f0)
    s = amp * np.exp(-((t - t0) / tau) ** 2) * np.sin(2.0 * math.pi * f0 * (t - t0))
    return s.astype(np.float32)


def flat_index(shape: Sequence[int], i, j=0, k=0) -> np.ndarray:
    nx = shape[0]
    ny = shape[1] if len(shape) > 1 else 1
    return (np.asarray(i, np.int64) + nx * (np.asarray(j, np.int64) + ny * np.asarray(k, np.int64))).astype(np.int64)


def random_sensors(shape: Sequence[int], n: int, margin: int, rng: np.random.Generator) -> Sensors:
    """n single-cell sensors at uniform interior positions (inside `margin`)."""
    coords = [rng.integers(margin, s - margin, size=n) for s in shape]
    while len(coords) < 3:
        coords.append(np.zeros(n, np.int64))
    idx = flat_index(shape, coords[0], coords[1], coords[2])
    return Sensors(idx=idx, group=np.arange(n, dtype=np.int32), n_groups=n)


# ----------------------------------------------------------------------------
# media
# ----------------------------------------------------------------------------

def _fill_relaxation(prob: Problem, tissue_of: np.ndarray, sets: List[dict],
                     alpha0_map: Optional[np.ndarray] = None) -> None:
    """Per-point relaxation parameters from per-tissue parameter sets (float32).

    When `alpha0_map` is given, d^{nu=1} of each point is scaled by
    alpha0(x) / alpha0_ref of its tissue set: the paper's modulation rule for
    media with continuously varying attenuation (Eq. relaxation_parameter_
    modulation_y).  This is an input recipe, not part of the time step.
    """
    N = len(sets[0]["d1"])
    g = tissue_of.shape
    k1 = np.empty(g, np.float32); k2 = np.empty(g, np.float32)
    d1 = np.empty((N,) + g, np.float32); a1 = np.empty_like(d1)
    d2 = np.empty_like(d1); a2 = np.empty_like(d1)
    lut = lambda key, nu=None: np.asarray([s[key] if nu is None else s[key][nu] for s in sets], np.float64)
    flat_t = tissue_of.reshape(-1)
    # a few tissues: one mask per tissue and masked copies (much faster than
    # a gather over a large grid); many tissues: the gather
    masks = [flat_t == t for t in range(1, len(sets))] if len(sets) <= 8 else None

    def put(dst, values):
        v = values.astype(np.float32)
        d = dst.reshape(-1)
        if masks is None:
            d[:] = v[flat_t]
            return
        d.fill(v[0])
        for t, m in enumerate(masks, 1):
            np.copyto(d, v[t], where=m)
    put(k1, lut("kappa1")); put(k2, lut("kappa2"))
    for nu in range(N):
        put(d1[nu], lut("d1", nu)); put(a1[nu], lut("alpha1", nu))
        put(d2[nu], lut("d2", nu)); put(a2[nu], lut("alpha2", nu))
    if alpha0_map is not None:
        ref = lut("alpha0").astype(np.float32)[flat_t].reshape(g)
        scale = np.asarray(alpha0_map, np.float32) / ref
        d1[0] *= scale
        d2[0] *= scale
    prob.nrelax = N
    prob.kappa1, prob.kappa2 = k1, k2
    prob.d1, prob.alpha1, prob.d2, prob.alpha2 = d1, a1, d2, a2


def homogeneous(shape: Sequence[int], h: float, dt: float, c: float = 1540.0,
                rho: float = 1000.0, relax: Optional[dict] = None,
                beta: Optional[float] = None) -> Problem:
    g = tuple(reversed(tuple(shape)))
    prob = Problem(shape=tuple(shape), h=h, dt=dt,
                   c=np.full(g, c, np.float32), rho=np.full(g, rho, np.float32))
    if beta is not None:
        prob.beta = np.full(g, beta, np.float32)
    if relax is not None:
        _fill_relaxation(prob, np.zeros(g, np.int32), [relax])
    return prob


def line_source_problem(n: int = 512, n_steps: int = 1000, seed: int = 0,
                        relax_key: str = "N4_y1.1_a0.5", cfl: float = 0.4,
                        f0: float = 3e6, ppw: float = 12.0,
                        pml_lambda: Tuple[float, float] = (3.0, 1.0),
                        n_sensors: int = 256) -> Problem:
    """2D plain method: homogeneous tissue, line source, point sensors.

    n x n grid at lambda/ppw for f0 (c0 = 1540 m/s), rho = 1000 kg/m^3,
    power-law attenuation from a fitted N-mechanism set, beta = 0 (linear),
    CFL `cfl`, two-stage C-PML of (transition, bound) wavelengths, a
    3-cycle Gaussian-windowed line source across the grid and `n_sensors`
    seeded interior point sensors.
    """
    rng = np.random.default_rng(seed)
    c0 = 1540.0
    lam = c0 / f0
    h = lam / ppw
    dt = cfl * h / c0
    sets = relaxation_sets()
    prob = homogeneous((n, n), h, dt, c=c0, rho=1000.0, relax=sets[relax_key])
    lt = int(round(pml_lambda[0] * ppw)); lb = int(round(pml_lambda[1] * ppw))
    prob.pml_transition, prob.pml_bound = lt, lb
    L = lt + lb
    row = L + 4
    xs = np.arange(L, n - L, dtype=np.int64)
    sig = gaussian_pulse(n_steps, dt, f0, 3.0, 1.0e5)[:, None]
    prob.sources = [Source("p", flat_index((n, n), xs, row), np.zeros(xs.size, np.int32), sig)]
    prob.sensors = random_sensors((n, n), n_sensors, L, rng)
    prob.n_steps = n_steps
    prob.name = f"2d-homogeneous-{n}x{n}-N{prob.nrelax}-linear"
    return prob


# Abdominal-wall tissue classes: c [m/s], rho [kg/m^3], alpha0 [dB/cm/MHz^y].
ABDOMINAL_TISSUES = [
    ("fat", 1478.0, 950.0, 0.48),
    ("muscle", 1547.0, 1050.0, 1.09),
    ("connective", 1613.0, 1120.0, 1.57),
]


def abdominal_problem(n: int = 4096, n_steps: int = 8000, seed: int = 1,
                      f0: float = 3e6, ppw: float = 12.0, cfl: float = 0.4,
                      n_elements: int = 128, nl: str = "pressure",
                      scatterers_per_cell: float = 20.0,
                      pml_lambda: Tuple[float, float] = (3.0, 1.0),
                      ny: Optional[int] = None) -> Problem:
    """2D heterogeneous nonlinear abdominal-wall-like medium.

    Layers of fat / muscle / connective tissue 2-5 mm thick whose interfaces
    are perturbed by a seeded sum of random sinusoids; beta drawn in [4, 6]
    per layer; sub-resolution scatterers at `scatterers_per_cell` per
    resolution cell (lambda^2) with a 2 % Gaussian c / rho perturbation; a
    linear array of `n_elements` elements (pitch 12 cells, width 11) firing a
    focused 1 MPa, 3-cycle pulse; traces recorded as element means.
    Stands in for the segmented Visible Human abdominal wall (not available).
    """
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    lam_ref = 1540.0 / f0
    h = lam_ref / ppw
    lt = int(round(pml_lambda[0] * ppw)); lb = int(round(pml_lambda[1] * ppw))
    L = lt + lb
    # layer stack along y (depth), starting below the array
    y_mm = (np.arange(ny) * h) * 1e3
    x_mm = (np.arange(nx) * h) * 1e3
    top = (L + 8) * h * 1e3
    tissue = np.zeros((ny, nx), np.int32)
    beta = np.zeros((ny, nx), np.float32)
    depth = top
    layer_bounds = [depth]
    layer_kind = []
    while depth < y_mm[-1]:
        thick = rng.uniform(2.0, 5.0)
        depth += thick
        layer_bounds.append(depth)
        layer_kind.append(int(rng.integers(0, 3)))
    # perturbed interface depth(x) = bound + sum of 8 random sinusoids (+-0.5 mm)
    Y = y_mm[:, None]
    current = np.full((ny, nx), -1, np.int32)
    prev_surface = np.full(nx, -1e9)
    for li, kind in enumerate(layer_kind):
        amp = rng.uniform(0.0, 0.5 / 8, 8)
        k = rng.uniform(0.2, 2.0, 8)           # 1/mm
        ph = rng.uniform(0, 2 * math.pi, 8)
        pert = (amp[:, None] * np.sin(k[:, None] * x_mm[None, :] + ph[:, None])).sum(0)
        surface = layer_bounds[li + 1] + pert
        m = (Y >= prev_surface[None, :]) & (Y < surface[None, :]) & (current < 0)
        current[m] = li
        prev_surface = surface
    current[current < 0] = len(layer_kind) - 1
    kinds = np.asarray(layer_kind, np.int32)
    tissue = kinds[current]
    layer_beta = rng.uniform(4.0, 6.0, len(layer_kind)).astype(np.float32)
    beta = layer_beta[current]
    props = np.asarray([t[1:] for t in ABDOMINAL_TISSUES], np.float64)
    c = props[tissue, 0].copy()
    rho = props[tissue, 1].copy()
    alpha0 = props[tissue, 2]
    # water-like coupling layer above the tissue (under the array)
    above = Y < top
    above = np.broadcast_to(above, (ny, nx))
    c[above] = 1540.0; rho[above] = 1000.0
    tissue = tissue.copy(); tissue[above] = 0  # relaxation of fat set scaled below
    alpha0 = alpha0.copy(); alpha0[above] = 0.02
    # sub-resolution scatterers: scatterers_per_cell per lambda^2
    cells_per_res = ppw * ppw
    density = scatterers_per_cell / cells_per_res
    n_sc = int(density * nx * ny)
    sy = rng.integers(0, ny, n_sc); sx = rng.integers(0, nx, n_sc)
    pert = 1.0 + 0.02 * rng.standard_normal(n_sc)
    keep = ~above[sy, sx]
    c[sy[keep], sx[keep]] *= pert[keep]
    rho[sy[keep], sx[keep]] *= pert[keep]
    sets_all = relaxation_sets()
    sets = [sets_all["N4_y1.1_fat"], sets_all["N4_y1.1_muscle"], sets_all["N4_y1.1_connective"]]
    # time step at `cfl` of the fastest high-frequency speed c / sqrt(kappa1 kappa2)
    kmin = min(s["kappa1"] * s["kappa2"] for s in sets)
    dt = cfl * h * math.sqrt(kmin) / float(c.max())
    prob = Problem(shape=(nx, ny), h=h, dt=dt, c=c.astype(np.float32), rho=rho.astype(np.float32),
                   beta=beta if nl != "off" else None)
    _fill_relaxation(prob, tissue, sets, alpha0_map=alpha0)
    prob.pml_transition, prob.pml_bound = lt, lb
    prob.nl_mode = nl
    # 128-element linear array along x at depth row L+4, pitch 12, width 11,
    # focused at 40 mm below the centre: per-element delays
    pitch, width = 12, 11
    aperture = n_elements * pitch
    x0 = (nx - aperture) // 2
    row = L + 4
    el_x0 = x0 + pitch * np.arange(n_elements)
    idx = []; grp = []
    for e in range(n_elements):
        xs = np.arange(el_x0[e], el_x0[e] + width)
        xs = xs[(xs >= L) & (xs < nx - L)]
        idx.append(flat_index((nx, ny), xs, row)); grp.append(np.full(xs.size, e, np.int32))
    idx = np.concatenate(idx); grp = np.concatenate(grp)
    centre_mm = (x0 + aperture / 2) * h * 1e3
    el_mm = (el_x0 + width / 2) * h * 1e3
    focus_mm = 40.0
    dist = np.sqrt((el_mm - centre_mm) ** 2 + focus_mm ** 2)
    delays = (dist.max() - dist) / 1540.0 * 1e-3
    t = (np.arange(n_steps) + 1.0) * dt
    tau = 3.0 / (2.0 * f0); t0 = 3.0 / f0
    tt = t[:, None] - t0 - delays[None, :]
    sig = (1.0e6 * np.exp(-(tt / tau) ** 2) * np.sin(2 * math.pi * f0 * tt)).astype(np.float32)
    prob.sources = [Source("p", idx, grp, sig)]
    prob.sensors = Sensors(idx=idx.copy(), group=grp.copy(), n_groups=n_elements)
    prob.n_steps = n_steps
    prob.name = f"2d-abdominal-{nx}x{ny}-N4-{nl}"
    return prob


def _value_noise_3d(shape: Tuple[int, int, int], cell: int, rng: np.random.Generator) -> np.ndarray:
    """Smooth seeded noise in [0, 1): trilinear interpolation of a random
    lattice (smoothstep weights), built one z plane at a time in float32."""
    nz, ny, nx = shape
    lat = rng.random((nz // cell + 2, ny // cell + 2, nx // cell + 2)).astype(np.float32)
    def coords(n):
        u = np.arange(n) / cell
        i0 = np.floor(u).astype(np.int64)
        f = (u - i0).astype(np.float32)
        return i0, f * f * (3 - 2 * f)
    iz, fz = coords(nz); iy, fy = coords(ny); ix, fx = coords(nx)
    out = np.empty(shape, np.float32)
    for z in range(nz):
        acc = np.zeros((ny, nx), np.float32)
        for dz, wz in ((0, 1 - fz[z]), (1, fz[z])):
            layer = lat[iz[z] + dz]
            for dy, wy in ((0, 1 - fy), (1, fy)):
                rows = layer[iy + dy]                      # (ny, lx)
                for dx, wx in ((0, 1 - fx), (1, fx)):
                    acc += (wz * wy[:, None] * wx[None, :]) * rows[:, ix + dx]
        out[z] = acc
    return out


def skull_problem(n: int = 768, n_steps: int = 4000, seed: int = 2, f0: float = 1e6,
                  ppw: float = 10.0, cfl: float = 0.4, pml_cells: int = 40,
                  array_elems: int = 16, nl: str = "off") -> Problem:
    """3D transcranial-like medium: brain background and an ellipsoidal skull shell.

    Brain c = 1560 m/s, rho = 1040 kg/m^3, alpha0 = 0.6, y = 1.2 (N = 3);
    shell of semi-axes (50, 45, 40) mm scaled to the grid, 1-2 mm thick, with
    seeded smooth porosity mapped linearly to c 2400-3000 m/s, rho
    1700-2000 kg/m^3 and alpha0 4-8 dB/MHz^y/cm; a 16 x 16 planar array
    firing a plane wave.  Stands in for the micro-CT rat skull (not available).
    """
    rng = np.random.default_rng(seed)
    h = 1540.0 / f0 / ppw
    g = (n, n, n)
    span = (n - 2 * pml_cells) * h * 1e3 * 0.5  # mm radius available
    scale = min(1.0, span / 55.0)
    ax = np.array([50.0, 45.0, 40.0]) * scale
    thick = 1.0 + rng.random() * 1.0
    coord = (np.arange(n, dtype=np.float32) - (n - 1) / 2.0) * np.float32(h * 1e3)
    rx2 = (coord / ax[0]) ** 2
    ry2 = (coord / ax[1]) ** 2
    shell = np.empty(g, bool)
    for z in range(n):
        r = np.sqrt(rx2[None, :] + ry2[:, None] + (coord[z] / ax[2]) ** 2)
        shell[z] = (r >= 1.0) & (r < 1.0 + thick / ax.min())
    phi = _value_noise_3d(g, max(4, n // 48), rng)
    c = np.full(g, 1560.0, np.float32)
    rho = np.full(g, 1040.0, np.float32)
    alpha0 = np.full(g, 0.6, np.float32)
    c[shell] = 2400.0 + 600.0 * phi[shell]
    rho[shell] = 1700.0 + 300.0 * phi[shell]
    alpha0[shell] = 4.0 + 4.0 * phi[shell]
    del phi
    tissue = shell.astype(np.uint8)
    del shell
    sets_all = relaxation_sets()
    sets = [sets_all["N3_y1.2_brain"], sets_all["N3_y1.2_skull"]]
    # time step at `cfl` of the fastest high-frequency speed c / sqrt(kappa1 kappa2)
    kmin = min(s["kappa1"] * s["kappa2"] for s in sets)
    dt = cfl * h * math.sqrt(kmin) / float(c.max())
    prob = Problem(shape=g, h=h, dt=dt, c=c, rho=rho)
    _fill_relaxation(prob, tissue, sets, alpha0_map=alpha0)
    prob.pml_transition = pml_cells * 3 // 4
    prob.pml_bound = pml_cells - prob.pml_transition
    prob.nl_mode = nl
    if nl != "off":
        prob.beta = np.full(g, 4.5, np.float32)
    # 16 x 16 planar array in the plane z = pml_cells + 4, pitch lambda/2
    pitch = max(1, int(round(ppw / 2)))
    k0 = pml_cells + 4
    start = n // 2 - array_elems * pitch // 2
    idx = []; grp = []
    for ey in range(array_elems):
        for ex in range(array_elems):
            xs = np.arange(start + ex * pitch, start + ex * pitch + max(1, pitch - 1))
            ys = np.arange(start + ey * pitch, start + ey * pitch + max(1, pitch - 1))
            X, Y = np.meshgrid(xs, ys, indexing="xy")
            idx.append(flat_index(g, X.ravel(), Y.ravel(), k0))
            grp.append(np.full(X.size, ey * array_elems + ex, np.int32))
    idx = np.concatenate(idx); grp = np.concatenate(grp)
    sig = gaussian_pulse(n_steps, dt, f0, 3.0, 1.0e5)
    sig = np.repeat(sig[:, None], array_elems * array_elems, axis=1)
    prob.sources = [Source("p", idx, grp, sig)]
    prob.sensors = Sensors(idx=idx.copy(), group=grp.copy(), n_groups=array_elems * array_elems)
    prob.n_steps = n_steps
    prob.name = f"3d-skull-{n}^3-N3"
    return prob


# ----------------------------------------------------------------------------
# states
# ----------------------------------------------------------------------------

def random_state(prob: Problem, seed: int, amp_p: float = 1.0e5, n_waves: int = 6,
                 memory: bool = True) -> dict:
    """Smooth seeded fields for the state arrays (p, v_q and, with `memory`,
    psi1_q, psi2_q), float32.

    Each field is a sum of `n_waves` random plane waves with wavelengths of
    at least 8 cells, so the state looks like a propagating wavefield rather
    than white noise.  Velocities are scaled by 1/(rho c), memory variables by
    a small factor.
    """
    rng = np.random.default_rng(seed)
    g = prob.grid_shape
    axes = [np.arange(s, dtype=np.float32) for s in g]
    def field(scale):
        out = np.zeros(g, np.float32)
        for _ in range(n_waves):
            kvec = rng.uniform(-1.0, 1.0, len(g)) * (2 * math.pi / 8.0)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.standard_normal()
            arg = np.float32(ph)
            for d, ax in enumerate(axes):
                shape = [1] * len(g); shape[d] = g[d]
                arg = arg + (np.float32(kvec[d]) * ax).reshape(shape)
            out += np.float32(a * scale) * np.sin(arg)
        return out
    st = {"p": field(amp_p)}
    vscale = amp_p / (1000.0 * 1540.0)
    N = prob.nrelax
    names = "xyz"
    for q in range(prob.ndim):
        st["v" + names[q]] = field(vscale)
        if N and memory:
            st["psi1" + names[q]] = np.stack([field(0.01 * amp_p / prob.h * 1e-3) for _ in range(N)])
            st["psi2" + names[q]] = np.stack([field(0.01 * vscale / prob.h * 1e-3) for _ in range(N)])
    return st


def with_steps(prob: Problem, n_steps: int) -> Problem:
    """Same problem with the signal tables cut or zero-padded to n_steps."""
    srcs = []
    for s in prob.sources:
        sig = s.signal[:n_steps]
        if sig.shape[0] < n_steps:
            sig = np.concatenate([sig, np.zeros((n_steps - sig.shape[0], sig.shape[1]), np.float32)])
        srcs.append(replace(s, signal=np.ascontiguousarray(sig)))
    return replace(prob, sources=srcs, n_steps=n_steps)


# Tissue classes of the tissue-index abdominal medium: (name, c, rho, alpha0,
# beta, relaxation set).  beta is one value per class in this form.
INDEXED_TISSUES = [
    ("water", 1540.0, 1000.0, 0.02, 3.5, "N4_y1.1_fat"),
    ("fat", 1478.0, 950.0, 0.48, 6.0, "N4_y1.1_fat"),
    ("muscle", 1547.0, 1050.0, 1.09, 4.6, "N4_y1.1_muscle"),
    ("connective", 1613.0, 1120.0, 1.57, 5.0, "N4_y1.1_connective"),
]
LEVELS = 64   # quantised scatterer levels per class; level 0 is unperturbed


def indexed_abdominal_problem(nx: int = 2048, ny: int = 1024, n_steps: int = 4000, seed: int = 1,
                              f0: float = 3e6, ppw: float = 12.0, cfl: float = 0.4,
                              n_elements: int = 64, focus_mm: float = 30.0, focus_x_mm: float = 0.0,
                              nl: str = "pressure",
                              scatterers_per_cell: float = 20.0,
                              pml_lambda: Tuple[float, float] = (3.0, 1.0), transmit: int = -1,
                              levels: int = LEVELS) -> Problem:
    """Abdominal-wall-like medium in tissue-index form (reduced storage).

    Layered fat / muscle / connective tissue under a water coupling layer as
    in `abdominal_problem`, with one beta per tissue class, and sub-resolution
    scatterers whose +-2 % c / rho perturbation is quantised to `levels` - 1
    levels (63 by default): each cell stores index = class * levels + level
    into per-entry tables (uint8 while 4 * levels <= 256, else uint16).  The
    dense per-cell arrays are the tables gathered.  `transmit` >= 0 fires only that
    element (a full-synthetic-aperture transmit event); -1 fires the focused
    array, focused at depth `focus_mm` and lateral offset `focus_x_mm` from
    the array centre.
    """
    rng = np.random.default_rng(seed)
    h = 1540.0 / f0 / ppw
    lt = int(round(pml_lambda[0] * ppw)); lb = int(round(pml_lambda[1] * ppw))
    L = lt + lb
    y_mm = (np.arange(ny) * h) * 1e3
    x_mm = (np.arange(nx) * h) * 1e3
    top = (L + 8) * h * 1e3
    cls = np.zeros((ny, nx), np.uint8)
    depth = top
    surface_prev = np.full(nx, top)
    Y = y_mm[:, None]
    while depth < y_mm[-1]:
        kind = int(rng.integers(1, 4))
        depth += rng.uniform(2.0, 5.0)
        amp = rng.uniform(0.0, 0.5 / 8, 8); k = rng.uniform(0.2, 2.0, 8); ph = rng.uniform(0, 2 * math.pi, 8)
        surface = depth + (amp[:, None] * np.sin(k[:, None] * x_mm[None, :] + ph[:, None])).sum(0)
        m = (Y >= surface_prev[None, :]) & (Y < surface[None, :])
        cls[m] = kind
        surface_prev = surface
    cls[Y >= surface_prev[None, :]] = 1
    cls[np.broadcast_to(Y < top, (ny, nx))] = 0
    level = np.zeros((ny, nx), np.uint8)
    n_sc = int(scatterers_per_cell / (ppw * ppw) * nx * ny)
    sy = rng.integers(0, ny, n_sc); sx = rng.integers(0, nx, n_sc)
    pert = np.clip(0.02 * rng.standard_normal(n_sc), -0.0799, 0.0799)
    top_level = levels - 2
    lv = np.round((pert + 0.08) / 0.16 * top_level).astype(np.int64) + 1   # 1 .. levels - 1
    keep = cls[sy, sx] != 0
    level = level.astype(np.int64)
    level[sy[keep], sx[keep]] = lv[keep]
    T = len(INDEXED_TISSUES) * levels
    tissue = (cls.astype(np.int64) * levels + level).astype(np.uint8 if T <= 256 else np.uint16)
    sets_all = relaxation_sets()
    tab = {k: np.zeros(T, np.float32) for k in ("c", "rho", "beta", "kappa1", "kappa2")}
    N = len(sets_all["N4_y1.1_fat"]["d1"])
    for k in ("d1", "alpha1", "d2", "alpha2"):
        tab[k] = np.zeros((N, T), np.float32)
    for ci, (name, c0, r0, a0, beta, key) in enumerate(INDEXED_TISSUES):
        sset = sets_all[key]
        for lvl in range(levels):
            e = ci * levels + lvl
            f = 1.0 if lvl == 0 else 1.0 + (-0.08 + (lvl - 1) / top_level * 0.16)
            tab["c"][e] = c0 * f; tab["rho"][e] = r0 * f; tab["beta"][e] = beta
            tab["kappa1"][e] = sset["kappa1"]; tab["kappa2"][e] = sset["kappa2"]
            for nu in range(N):
                mod = a0 / sset["alpha0"] if nu == 0 else 1.0
                tab["d1"][nu, e] = sset["d1"][nu] * mod; tab["alpha1"][nu, e] = sset["alpha1"][nu]
                tab["d2"][nu, e] = sset["d2"][nu] * mod; tab["alpha2"][nu, e] = sset["alpha2"][nu]
    used_sets = [sets_all[t[5]] for t in INDEXED_TISSUES]
    kmin = min(s_["kappa1"] * s_["kappa2"] for s_ in used_sets)
    dt = cfl * h * math.sqrt(kmin) / float(tab["c"].max())
    ti = tissue.astype(np.int64)
    prob = Problem(shape=(nx, ny), h=h, dt=dt, c=tab["c"][ti], rho=tab["rho"][ti],
                   beta=tab["beta"][ti] if nl != "off" else None)
    prob.nrelax = N
    prob.kappa1 = tab["kappa1"][ti]; prob.kappa2 = tab["kappa2"][ti]
    prob.d1 = tab["d1"][:, ti]; prob.alpha1 = tab["alpha1"][:, ti]
    prob.d2 = tab["d2"][:, ti]; prob.alpha2 = tab["alpha2"][:, ti]
    prob.tissue = tissue
    prob.tables = tab
    prob.pml_transition, prob.pml_bound = lt, lb
    prob.nl_mode = nl
    pitch, width = 12, 11
    aperture = n_elements * pitch
    x0 = max(L, (nx - aperture) // 2)
    row = L + 4
    el_x0 = x0 + pitch * np.arange(n_elements)
    idx, grp = [], []
    for e in range(n_elements):
        xs = np.arange(el_x0[e], el_x0[e] + width)
        xs = xs[(xs >= L) & (xs < nx - L)]
        idx.append(flat_index((nx, ny), xs, row)); grp.append(np.full(xs.size, e, np.int32))
    idx = np.concatenate(idx); grp = np.concatenate(grp)
    t = (np.arange(n_steps) + 1.0) * dt
    tau = 3.0 / (2.0 * f0); t0 = 3.0 / f0
    if transmit >= 0:
        delays = np.full(n_elements, np.inf); delays[transmit % n_elements] = 0.0
    else:
        centre_mm = (x0 + aperture / 2) * h * 1e3 + focus_x_mm
        el_mm = (el_x0 + width / 2) * h * 1e3
        dist = np.sqrt((el_mm - centre_mm) ** 2 + focus_mm ** 2)
        delays = (dist.max() - dist) / 1540.0 * 1e-3
    tt = t[:, None] - t0 - np.where(np.isfinite(delays), delays, 0.0)[None, :]
    sig = 1.0e6 * np.exp(-(tt / tau) ** 2) * np.sin(2 * math.pi * f0 * tt)
    sig[:, ~np.isfinite(delays)] = 0.0
    prob.sources = [Source("p", idx, grp, sig.astype(np.float32))]
    prob.sensors = Sensors(idx=idx.copy(), group=grp.copy(), n_groups=n_elements)
    prob.n_steps = n_steps
    prob.name = f"2d-abdominal-indexed-{nx}x{ny}"
    return prob
