"""GPU path vs the FP64 oracle, element by element, through the C ABI.

The oracle runs on the same float32 inputs with its coefficient maps rounded
to float32 (the maps the kernels stream), in FP64 arithmetic.  Tolerances
(the accuracy target of the method's GPU port): relative L2 <= 1e-4 and
max |error| <= 1e-4 of the peak for the fields p and v_q; sensor traces within
-100 dB of their peak.  The memory variables meet 1e-4 outside the C-PML;
inside it they hold the slowly decaying memory of the absorbed wave, whose
float32 rounding grows relative to it, and the bound there is 1e-3.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

import synth
from oracle.core import OracleSim

pytestmark = pytest.mark.gpu

REL_L2 = 1e-4
MAX_REL = 1e-4
TRACE_DB = -100.0


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def rel_l2(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def max_rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    m = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / m if m > 0 else np.max(np.abs(a))


def trace_db(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    e = np.max(np.abs(a - b)); m = np.max(np.abs(b))
    return 20 * math.log10(max(e, 1e-300) / m)


def assert_field(name, g, o, rel=REL_L2, mx=MAX_REL):
    r, m = rel_l2(g, o), max_rel(g, o)
    assert r <= rel and m <= mx, f"{name}: rel L2 {r:.3e}, max/peak {m:.3e}"


PSI_PML = 1e-3


def pml_mask(prob, shape_np, window=None):
    """True on cells outside every C-PML strip (numpy order, optional window)."""
    L = prob.pml_transition + prob.pml_bound if prob.nrelax else 0
    m = np.ones(shape_np, bool)
    if L == 0:
        return m
    nd = prob.ndim
    win = window or [(0, s) for s in prob.shape]
    for q in range(nd):
        ax = nd - 1 - q
        coord = np.arange(win[q][0], win[q][0] + shape_np[ax])
        inside = (coord >= L) & (coord < prob.shape[q] - L)
        sh = [1] * nd
        sh[ax] = -1
        m = m & inside.reshape(sh)
    return m


def assert_state(prob, name, g, o, window=None):
    if not name.startswith("psi"):
        assert_field(name, g, o)
        return
    assert_field(name, g, o, PSI_PML, PSI_PML)
    m = pml_mask(prob, g.shape[1:], window)
    if m.any() and np.abs(o[:, m]).max() > 0:
        assert_field(name + "[outside C-PML]", g[:, m], o[:, m])


def state_names(prob):
    names = ["p"] + ["v" + "xyz"[q] for q in range(prob.ndim)]
    if prob.nrelax:
        names += ["psi1" + "xyz"[q] for q in range(prob.ndim)] + ["psi2" + "xyz"[q] for q in range(prob.ndim)]
    return names


def relax_set(N):
    """A fitted set of N <= 4 mechanisms; for N > 4 the four-mechanism set
    with N - 4 more mechanisms at rescaled rates (d / 2, alpha x 3: not a
    fit; the step computes whatever parameters it is given)."""
    if N <= 4:
        key = {1: "N2_y1.0_a0.5", 2: "N2_y1.0_a0.5", 3: "N3_y1.2_brain", 4: "N4_y1.1_a0.5"}[N]
        s = dict(synth.relaxation_sets()[key])
        if N == 1:
            s = {k: (v[:1] if isinstance(v, list) else v) for k, v in s.items()}
        return s
    s = dict(synth.relaxation_sets()["N4_y1.1_a0.5"])
    extra = N - 4
    for k, f in (("d1", 0.5), ("d2", 0.5), ("alpha1", 3.0), ("alpha2", 3.0)):
        s[k] = list(s[k]) + [v * f for v in s[k][:extra]]
    return s


def small_2d(nx=200, ny=136, N=2, nl="off", steps=300, seed=0, pml=(12, 4), alignment="centred",
             reading="C", vel_src=False, hetero=True, amp=None):
    rng = np.random.default_rng(seed)
    f0 = 3e6
    h = 1540.0 / f0 / 12
    relax = relax_set(N) if N else None
    prob = synth.homogeneous((nx, ny), h, 0.0, relax=relax)
    g = prob.grid_shape
    if hetero:
        prob.c = (1540.0 * (1 + 0.08 * rng.standard_normal(g).clip(-2, 2))).astype(np.float32)
        prob.rho = (1000.0 * (1 + 0.1 * rng.random(g))).astype(np.float32)
    prob.dt = 0.4 * h / float(prob.c.max()) * 0.95
    if nl != "off":
        prob.beta = rng.uniform(3.0, 8.0, g).astype(np.float32)
    prob.nl_mode = nl
    prob.memory_alignment = alignment
    prob.pml_reading = reading
    if N:
        prob.pml_transition, prob.pml_bound = pml
    L = sum(pml) if N else 0
    xs = np.arange(L + 2, nx - L - 2)
    sig = synth.gaussian_pulse(steps, prob.dt, f0, 3.0, amp or (2e6 if nl != "off" else 1e5))
    prob.sources = [synth.Source("p", synth.flat_index((nx, ny), xs, L + 6), np.zeros(xs.size, np.int32),
                                 sig[:, None])]
    if vel_src:
        ys = np.arange(L + 10, L + 20)
        sig2 = np.stack([sig * 1e-6, -sig * 2e-6], axis=1).astype(np.float32)
        prob.sources.append(synth.Source("vx", synth.flat_index((nx, ny), nx // 2, ys),
                                         (np.arange(ys.size) % 2).astype(np.int32), sig2))
        prob.sources.append(synth.Source("vy", synth.flat_index((nx, ny), ys, ny // 2),
                                         np.zeros(ys.size, np.int32), sig2[:, :1].copy()))
    sens = synth.random_sensors((nx, ny), 30, max(L, 4), rng)
    # two grouped sensors (element averaging) on top of the point sensors
    grp_idx = synth.flat_index((nx, ny), np.arange(L + 4, L + 15), ny // 2)
    sens = synth.Sensors(np.concatenate([sens.idx, grp_idx]),
                         np.concatenate([sens.group, np.full(grp_idx.size, 30, np.int32)]), 31)
    prob.sensors = sens
    prob.n_steps = steps
    return prob


def compare_run(fw2, prob, steps, state=None, check_trace=True, rel=REL_L2, mx=MAX_REL, maps="f32",
                kernel_path="auto"):
    sim = fw2.Simulation(prob, map_precision=maps, kernel_path=kernel_path)
    if state is not None:
        sim.set_state(state)
    sim.step(steps)
    sim.synchronize()
    orc = OracleSim(prob, round_to="f32" if maps in ("idx", "idx16") else maps)
    if state is not None:
        orc.set_state(state)
    orc.run(steps)
    for name in state_names(prob):
        assert_state(prob, name, sim.field(name), orc.field(name))
    if check_trace and prob.sensors is not None:
        tg = sim.trace.cpu().numpy()[:steps]
        to = orc.trace[:steps]
        db = trace_db(tg, to)
        assert db <= TRACE_DB, f"trace error {db:.1f} dB"
    sim.close()
    return sim, orc


CASES_2D = {
    "base": dict(),
    # more mechanisms than the pipelined kernels take (tile kernels)
    "N6-nonlinear": dict(N=6, nl="pressure", steps=250),
    "N8-literal": dict(N=8, nl="literal", vel_src=True, amp=2e7, steps=200),
    "nonlinear-pressure": dict(nl="pressure"),
    "westervelt-N4": dict(nl="westervelt", N=4),
    "endpoint-readingA": dict(alignment="endpoint", reading="A"),
    "readingA": dict(reading="A", N=4),
    "ragged-203x77": dict(nx=203, ny=77, pml=(8, 3)),
    "velocity-sources": dict(vel_src=True, N=4),
    "tiny-tile": dict(nx=24, ny=20, pml=(3, 1), steps=200),
    # grids with interior tiles: the persistent kernels' staged half tiles
    "interior-560x200-N4-nl": dict(nx=560, ny=200, N=4, nl="pressure", steps=250),
    "interior-430x170-N0": dict(nx=430, ny=170, N=0, steps=250),
    # both nonlinear factors (Eqs. general5-general6) at 2e7 Pa, where the
    # momentum factor moves the fields by ~1e-2, a hundred times the bound
    "literal-N4": dict(nl="literal", N=4, vel_src=True, amp=2e7),
    "literal-interior-560x200-N2": dict(nx=560, ny=200, N=2, nl="literal", steps=250, amp=2e7),
}


@pytest.mark.parametrize("case", list(CASES_2D))
def test_parity_2d(fw2, case):
    kw = dict(CASES_2D[case])
    steps = kw.get("steps", 300)
    prob = small_2d(**kw)
    compare_run(fw2, prob, steps)


@pytest.mark.parametrize("case", ["interior-560x200-N4-nl", "interior-430x170-N0", "ragged-203x77",
                                  "literal-interior-560x200-N2"])
def test_parity_2d_pipelined_path(fw2, case):
    kw = dict(CASES_2D[case])
    steps = kw.get("steps", 300)
    compare_run(fw2, small_2d(**kw), steps, kernel_path="pipe")


@pytest.mark.parametrize("path", ["tile", "pipe"])
def test_parity_2d_literal_tile_and_pipe(fw2, path):
    kw = dict(CASES_2D["literal-interior-560x200-N2"])
    compare_run(fw2, small_2d(**kw), kw["steps"], kernel_path=path)


def test_literal_momentum_factor_acts(fw2):
    """The literal system differs from the pressure-only factor with the same
    beta_eff by far more than the parity bound: the momentum factor runs."""
    out = {}
    for nl in ("pressure", "literal"):
        prob = small_2d(nx=300, ny=200, N=2, nl=nl, steps=250, amp=2e7)
        sim = fw2.Simulation(prob)
        sim.step(250)
        out[nl] = sim.field("p")
        sim.close()
    assert rel_l2(out["literal"], out["pressure"]) > 30 * REL_L2


@pytest.mark.parametrize("nl,N", [("off", 2), ("pressure", 4)])
def test_parity_2d_bf16_maps(fw2, nl, N):
    """bf16 coefficient maps against the oracle run on the same bf16-rounded maps."""
    prob = small_2d(N=N, nl=nl, steps=250)
    compare_run(fw2, prob, 250, maps="bf16")


def test_parity_2d_periodic_lossless_cross_taps(fw2):
    """N = 0, periodic on both axes, g11 != 0, from a random state (no sources)."""
    prob = synth.homogeneous((144, 96), 1e-4, 0.0)
    rng = np.random.default_rng(2)
    prob.c = (1500 + 200 * rng.random(prob.grid_shape)).astype(np.float32)
    prob.dt = 0.3 * 1e-4 / float(prob.c.max())
    prob.bc = ("periodic", "periodic", "zero")
    taps = [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]
    prob.taps = (taps[0] * 0.98, taps[1], taps[2], taps[3], 0.005)
    st = synth.random_state(prob, seed=7)
    compare_run(fw2, prob, 250, state=st, check_trace=False)


def test_parity_2d_random_state_all_fields(fw2):
    """Non-zero memory variables everywhere from the start (random state)."""
    prob = small_2d(N=4, nl="pressure", steps=60)
    st = synth.random_state(prob, seed=11)
    compare_run(fw2, prob, 60, state=st)


def small_3d(n=(70, 40, 36), N=3, nl="westervelt", steps=80, seed=3, pml=(6, 2)):
    rng = np.random.default_rng(seed)
    f0 = 1e6
    h = 1540.0 / f0 / 10
    relax = relax_set(N) if N else None
    prob = synth.homogeneous(n, h, 0.0, relax=relax)
    g = prob.grid_shape
    prob.c = (1560.0 * (1 + 0.1 * rng.random(g))).astype(np.float32)
    prob.rho = (1040.0 * (1 + 0.1 * rng.random(g))).astype(np.float32)
    prob.dt = 0.4 * h / float(prob.c.max())
    prob.beta = rng.uniform(3, 6, g).astype(np.float32)
    prob.nl_mode = nl
    prob.pml_transition, prob.pml_bound = pml if N else (0, 0)
    sig = synth.gaussian_pulse(steps, prob.dt, f0, 2.0, 1e6)
    X, Y = np.meshgrid(np.arange(20, 50), np.arange(12, 28), indexing="xy")
    idx = synth.flat_index(n, X.ravel(), Y.ravel(), 10)
    prob.sources = [synth.Source("p", idx, np.zeros(idx.size, np.int32), sig[:, None]),
                    synth.Source("vz", idx[:40], np.zeros(40, np.int32), (sig * 1e-6)[:, None])]
    prob.sensors = synth.random_sensors(n, 25, 8, rng)
    prob.n_steps = steps
    return prob


def test_parity_3d(fw2):
    prob = small_3d()
    compare_run(fw2, prob, 80)


def indexed_3d(n=(70, 40, 36), N=3, n_tissue=6, seed=11, nl="westervelt", steps=60):
    """small_3d's grid, sources and sensors over a seeded tissue-index medium:
    n_tissue tissues with their own c, rho, beta and relaxation rates (the
    brain set scaled per tissue), a random tissue per cell (uint8, or uint16
    beyond 256 tissues); the dense arrays are the tables gathered."""
    prob = small_3d(n=n, N=N, nl=nl, steps=steps, seed=seed)
    rng = np.random.default_rng(seed)
    base = relax_set(N)
    tab = {"c": (1500 + 120 * rng.random(n_tissue)).astype(np.float32),
           "rho": (1000 + 150 * rng.random(n_tissue)).astype(np.float32),
           "beta": rng.uniform(3, 6, n_tissue).astype(np.float32),
           "kappa1": np.full(n_tissue, base["kappa1"], np.float32),
           "kappa2": np.full(n_tissue, base["kappa2"], np.float32)}
    f = rng.uniform(0.8, 1.2, (4, N, n_tissue))
    for i, key in enumerate(("d1", "alpha1", "d2", "alpha2")):
        tab[key] = (np.asarray(base[key][:N], np.float64)[:, None] * f[i]).astype(np.float32)
    t = rng.integers(0, n_tissue, prob.grid_shape)
    prob.tissue = t.astype(np.uint8 if n_tissue <= 256 else np.uint16)
    prob.tables = tab
    prob.c, prob.rho, prob.beta = tab["c"][t], tab["rho"][t], tab["beta"][t]
    prob.kappa1, prob.kappa2 = tab["kappa1"][t], tab["kappa2"][t]
    prob.d1, prob.alpha1 = tab["d1"][:, t], tab["alpha1"][:, t]
    prob.d2, prob.alpha2 = tab["d2"][:, t], tab["alpha2"][:, t]
    prob.dt = 0.4 * prob.h / float(tab["c"].max()) * 0.95
    return prob


@pytest.mark.parametrize("maps,n_tissue,nl", [("idx", 6, "westervelt"), ("idx16", 300, "literal")])
def test_parity_3d_tissue_index(fw2, maps, n_tissue, nl):
    """The tissue index in 3D (tables through L2, tile kernels) against the
    oracle; the uint8 form also bitwise against the same medium as dense float
    maps (the tables gathered per cell)."""
    prob = indexed_3d(n_tissue=n_tissue, nl=nl)
    if nl == "literal":
        prob.sources[0].signal = prob.sources[0].signal * 20.0
    sim = fw2.Simulation(prob, map_precision=maps)
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "tile"
    sim.close()
    compare_run(fw2, prob, 60, maps=maps)
    if maps == "idx":
        out = {}
        for m in ("idx", "f32"):
            s = fw2.Simulation(prob, map_precision=m, kernel_path="tile")
            s.step(60)
            out[m] = ({n: s.field(n) for n in ("p", "vx", "vz")}, s.trace.cpu().numpy())
            s.close()
        for n in ("p", "vx", "vz"):
            np.testing.assert_array_equal(out["idx"][0][n], out["f32"][0][n], err_msg=n)
        np.testing.assert_array_equal(out["idx"][1], out["f32"][1])


@pytest.mark.parametrize("case", ["nonlinear-pressure", "literal-N4", "readingA", "ragged-203x77"])
def test_parity_2d_fp16_maps(fw2, case):
    """FP16 maps (each map divided by its power-of-two scale) on the tile
    kernels against the oracle on the same stored maps."""
    kw = dict(CASES_2D[case])
    steps = kw.get("steps", 300)
    compare_run(fw2, small_2d(**kw), steps, maps="f16")


@pytest.mark.parametrize("nl", ["westervelt", "literal"])
def test_parity_3d_fp16_maps(fw2, nl):
    prob = small_3d(n=(70, 40, 36), N=3, nl=nl, steps=60)
    if nl == "literal":
        prob.sources[0].signal = prob.sources[0].signal * 20.0     # the momentum factor acts
    sim = fw2.Simulation(prob, map_precision="f16")
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "tile"
    sim.close()
    compare_run(fw2, prob, 60, maps="f16")


def test_parity_2d_eight_mechanisms_bf16(fw2):
    compare_run(fw2, small_2d(N=8, nl="pressure", steps=250), 250, maps="bf16")


@pytest.mark.parametrize("N,maps", [(5, "f32"), (8, "bf16")])
def test_parity_3d_more_mechanisms(fw2, N, maps):
    """More mechanisms than the pipelined 3D half steps take: the tile
    kernels, float and bf16 maps."""
    prob = small_3d(n=(70, 40, 36), N=N, steps=60)
    sim = fw2.Simulation(prob, map_precision=maps)
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "tile"
    sim.close()
    compare_run(fw2, prob, 60, maps=maps)


@pytest.mark.parametrize("maps", ["f32", "bf16"])
def test_parity_3d_time_space_taps(fw2, maps):
    """The 3D time-space optimised operator (Sec. 3.1; cross taps over both
    transverse axes, library taps for a 3D grid at the problem's Courant
    number) against the oracle with the same taps: float maps on the tile
    kernels, bf16 maps on the pipelined half steps."""
    prob = small_3d(n=(70, 40, 36), steps=80)
    r = float(np.max(prob.c)) * prob.dt / prob.h
    prob.taps = tuple(fw2.fw2_taps_time_space(r, 3))
    assert prob.taps[4] > 0
    compare_run(fw2, prob, 80, maps=maps, kernel_path="pipe" if maps == "bf16" else "auto")
    sim = fw2.Simulation(prob, map_precision="bf16", kernel_path="pipe")
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "pipe"
    sim.close()


def test_parity_3d_periodic_lossless_cross_taps(fw2):
    """N = 0, periodic on all three axes, g11 != 0, from a random state: the
    cross taps wrap across every face of the grid."""
    prob = synth.homogeneous((52, 36, 28), 1e-4, 0.0)
    rng = np.random.default_rng(4)
    prob.c = (1500 + 200 * rng.random(prob.grid_shape)).astype(np.float32)
    prob.dt = 0.3 * 1e-4 / float(prob.c.max())
    prob.bc = ("periodic",) * 3
    prob.taps = tuple(fw2.fw2_taps_time_space(0.3, 3))
    compare_run(fw2, prob, 40, state=synth.random_state(prob, seed=8))


@pytest.mark.parametrize("maps", ["f32", "bf16"])
def test_parity_3d_literal(fw2, maps):
    """Both nonlinear factors in 3D: float maps on the tile kernels, bf16 maps
    on the pipelined half steps."""
    prob = small_3d(nl="literal", steps=80)
    for s in prob.sources:
        if s.kind == "p":
            s.signal = s.signal * 20
    compare_run(fw2, prob, 80, maps=maps, kernel_path="pipe" if maps == "bf16" else "auto")
    sim = fw2.Simulation(prob, map_precision="bf16", kernel_path="pipe")
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "pipe"
    sim.close()


def test_parity_3d_bf16_maps(fw2):
    prob = small_3d(nl="off")
    compare_run(fw2, prob, 80, maps="bf16")


def test_parity_3d_random_state(fw2):
    prob = small_3d(n=(36, 44, 40), steps=30)
    st = synth.random_state(prob, seed=5)
    compare_run(fw2, prob, 30, state=st)


@pytest.mark.parametrize("N,nl", [(0, "off"), (2, "pressure"), (3, "westervelt"), (3, "off"), (3, "literal")])
def test_pipelined_3d_equals_tile_path_bitwise(fw2, N, nl):
    """The persistent TMA-staged 3D half steps (bf16 maps) compute exactly what
    the tile kernels compute: interior and edge units, ragged x and y, C-PML
    strips on every axis."""
    prob = small_3d(n=(300, 70, 45), N=N, nl=nl, steps=40)
    _pipe_vs_tile(fw2, prob, 40, maps="bf16")


@pytest.mark.parametrize("N,nl", [(0, "off"), (3, "westervelt"), (2, "literal"), (3, "literal")])
def test_pipelined_3d_cross_taps_equal_tile_path_bitwise(fw2, N, nl):
    """The time-space taps (g11 != 0) on the pipelined 3D half steps: the
    velocity cross taps come from the operand ring's planes k +- 1, the
    pressure ones from the v_x, v_y rings and the haloed v_z ring; bitwise
    what the tile kernels compute, with and without the literal system."""
    prob = small_3d(n=(300, 70, 45), N=N, nl=nl, steps=40)
    r = float(np.max(prob.c)) * prob.dt / prob.h
    prob.taps = tuple(fw2.fw2_taps_time_space(r, 3))
    if nl == "literal":
        for s_ in prob.sources:
            if s_.kind == "p":
                s_.signal = s_.signal * 20
    _pipe_vs_tile(fw2, prob, 40, maps="bf16")


def test_pipelined_3d_cross_taps_from_random_state_equal_tile_path_bitwise(fw2):
    """Cross taps on a ragged grid from a random state, every field nonzero
    from the start (halo rows and planes at every edge carry values)."""
    prob = small_3d(n=(200, 45, 30), N=2, nl="pressure", steps=20)
    prob.taps = tuple(fw2.fw2_taps_time_space(0.35, 3))
    _pipe_vs_tile(fw2, prob, 20, maps="bf16", state=synth.random_state(prob, seed=21))


def test_pipelined_3d_x_strip_loaded_per_cell_equals_tile_path_bitwise(fw2):
    """A C-PML of 7 cells: the x strip's coefficient rows are not 16-byte
    multiples, so edge units read them per cell instead of by TMA."""
    prob = small_3d(n=(300, 70, 45), N=3, nl="pressure", steps=40, pml=(5, 2))
    _pipe_vs_tile(fw2, prob, 40, maps="bf16")


@pytest.mark.parametrize("shape,pml", [((100, 40, 20), (6, 2)), ((264, 30, 18), (6, 2)), ((200, 24, 17), (3, 1)),
                                       ((300, 36, 8), (1, 1)), ((200, 20, 20), (6, 2))])
def test_pipelined_3d_small_grids_equal_tile_path_bitwise(fw2, shape, pml):
    """Grids at the limits of the 3D pipeline from a random state: one x tile
    reaching both x strips (nx < 128 + L: the strip read per cell), a ragged
    last x tile holding the whole high strip (staged), a strip that is not a
    16-byte row (per cell; a y strip of 4 rows, staged), the fewest planes a
    grid may have, eight (most ring planes outside the grid; y strips of 2
    rows, read per cell), and units reaching both y strips (ny < 2 L + 8:
    read per cell)."""
    rng = np.random.default_rng(11)
    h = 1e-4
    prob = synth.homogeneous(shape, h, 0.0, relax=synth.relaxation_sets()["N2_y1.0_a0.5"])
    prob.c = (1540.0 * (1 + 0.05 * rng.random(prob.grid_shape))).astype(np.float32)
    prob.rho = (1000.0 * (1 + 0.1 * rng.random(prob.grid_shape))).astype(np.float32)
    prob.dt = 0.3 * h / float(prob.c.max())
    prob.pml_transition, prob.pml_bound = pml
    _pipe_vs_tile(fw2, prob, 20, maps="bf16", state=synth.random_state(prob, seed=12))


def test_pipelined_3d_many_columns_equals_tile_path_bitwise(fw2):
    """More columns of units than blocks: each block marches several items
    (columns and plane ranges), reloading its plane ring at each new one."""
    prob = small_3d(n=(300, 600, 20), N=3, nl="westervelt", steps=30)
    _pipe_vs_tile(fw2, prob, 30, maps="bf16")


def test_parity_3d_pipelined_path(fw2):
    prob = small_3d(n=(300, 70, 45), steps=60)
    compare_run(fw2, prob, 60, maps="bf16", kernel_path="pipe")


def test_parity_plain_2d_config_full(fw2):
    """The plain 2D configuration in full: 512 x 512, N = 4, y = 1.1, linear,
    4-wavelength C-PML, line source, 256 sensors, 1000 steps."""
    prob = synth.line_source_problem(n=512, n_steps=1000)
    compare_run(fw2, prob, 1000)


def _window_compare(sim, orc, prob, window, steps, rel=REL_L2, mx=MAX_REL):
    m = 8 * steps
    sl_g, sl_o = [], []
    for q in reversed(range(prob.ndim)):
        lo, hi = window[q]
        a = lo if lo == 0 else lo + m
        b = hi if hi == prob.shape[q] else hi - m
        sl_g.append(slice(a, b))
        sl_o.append(slice(a - lo, b - lo))
    for name in state_names(prob):
        g = sim.field(name)
        o = orc.field(name)
        gw = g[(Ellipsis,) + tuple(sl_g)]
        ow = o[(Ellipsis,) + tuple(sl_o)]
        w_eff = [(window[q][0] + sl_o[prob.ndim - 1 - q].start, 0) for q in range(prob.ndim)]
        assert_state(prob, name, gw, ow, window=w_eff)


def test_parity_abdominal_full_size_windows(fw2):
    """4096 x 4096 heterogeneous nonlinear medium, N = 4, in the launch
    configuration the benchmark times, from a seeded wavefield: after 4 steps
    the GPU matches the oracle on windows covering a C-PML corner, the array
    and the deep interior (sampled outputs the oracle computes exactly)."""
    prob = synth.abdominal_problem(n=4096, n_steps=8)
    st = synth.random_state(prob, seed=21)
    steps = 4
    sim = fw2.Simulation(prob)
    sim.set_state(st)
    sim.step(steps)
    sim.synchronize()
    for window in (((0, 160), (0, 160)), ((1900, 2200), (30, 200)), ((3000, 3200), (3900, 4096))):
        orc = OracleSim(prob, round_to="f32", window=window)
        orc.set_state(st)
        orc.run(steps)
        _window_compare(sim, orc, prob, window, steps)
    sim.close()


def test_parity_abdominal_tissue_index_full_size_windows(fw2):
    """The tissue-index workload the benchmark times (4096 x 4096, uint8
    index, 128-element focused array) from a seeded wavefield: after 4 steps
    the GPU matches the oracle (the gathered float tables) on windows covering
    a C-PML corner, the array and the deep interior."""
    prob = synth.indexed_abdominal_problem(nx=4096, ny=4096, n_steps=8, seed=1, n_elements=128, focus_mm=40.0)
    st = synth.random_state(prob, seed=22)
    steps = 4
    sim = fw2.Simulation(prob, map_precision="idx")
    sim.set_state(st)
    sim.step(steps)
    sim.synchronize()
    assert fw2.fw2_kernel_path(sim.ctx) == "pipe"
    for window in (((0, 160), (0, 160)), ((1900, 2200), (30, 200)), ((3000, 3200), (3900, 4096))):
        orc = OracleSim(prob, round_to="f32", window=window)
        orc.set_state(st)
        orc.run(steps)
        _window_compare(sim, orc, prob, window, steps)
    sim.close()


def test_parity_skull_full_size_windows(fw2):
    """768^3 transcranial-like medium with bf16 maps, N = 3, in the launch
    configuration the 3D benchmark times, from a seeded wavefield: after 2
    steps the GPU matches the oracle (same bf16 maps) on windows covering a
    C-PML corner, the skull shell and the brain interior."""
    prob = synth.skull_problem(n=768, n_steps=4)
    st = synth.random_state(prob, seed=31, memory=False)
    steps = 2
    sim = fw2.Simulation(prob, map_precision="bf16")
    sim.set_state(st)
    sim.step(steps)
    sim.synchronize()
    # shell crossing on the x axis through the centre
    xs = int(np.argmax(prob.c[384, 384, :] > 2000.0))
    for window in (((0, 56), (0, 56), (0, 56)), ((xs - 24, xs + 24), (360, 408), (360, 408)),
                   ((500, 548), (200, 248), (300, 348))):
        orc = OracleSim(prob, round_to="bf16", window=window)
        orc.set_state(st)
        orc.run(steps)
        _window_compare(sim, orc, prob, window, steps)
    sim.close()


@pytest.mark.parametrize("nl", ["pressure", "off", "literal"])
def test_tissue_index_form_equals_dense_form_bitwise(fw2, nl):
    """uint8 tissue index + per-tissue tables give bitwise the same fields and
    traces as the dense float maps of the same medium (ragged 203 x 150 grid)."""
    prob = synth.indexed_abdominal_problem(nx=203, ny=150, n_steps=150, n_elements=8, nl=nl,
                                           pml_lambda=(1.0, 0.5))
    dense = fw2.Simulation(prob, map_precision="f32"); dense.step(150)
    idx = fw2.Simulation(prob, map_precision="idx"); idx.step(150)
    for name in state_names(prob):
        np.testing.assert_array_equal(dense.field(name), idx.field(name), err_msg=name)
    np.testing.assert_array_equal(dense.trace.cpu().numpy(), idx.trace.cpu().numpy())


def _pipe_vs_tile(fw2, prob, steps, maps="f32", state=None):
    """Every pipelined path equals the tile kernels bitwise; in 3D each layout
    of the pipelined half steps alone, and the tuned choice (which runs both
    on its first four steps)."""
    out = {}
    paths = ("tile", "pipe") if prob.ndim == 2 else ("tile", "pipe-staged", "pipe-registers", "pipe")
    for path in paths:
        sim = fw2.Simulation(prob, map_precision=maps, kernel_path=path)
        if state is not None:
            sim.set_state(state)
        sim.step(steps)
        assert fw2.fw2_kernel_path(sim.ctx) == ("tile" if path == "tile" else "pipe")
        out[path] = ({n: sim.field(n) for n in state_names(prob)},
                     sim.trace.cpu().numpy() if sim.trace is not None else None)
        sim.close()
    for path in paths[1:]:
        for n in state_names(prob):
            np.testing.assert_array_equal(out[path][0][n], out["tile"][0][n], err_msg=f"{path}: {n}")
        if out["tile"][1] is not None:
            np.testing.assert_array_equal(out[path][1], out["tile"][1])


@pytest.mark.parametrize("N,nl", [(0, "off"), (2, "westervelt"), (2, "off"), (3, "pressure"), (4, "pressure"),
                                  (0, "literal"), (4, "literal")])
def test_pipelined_path_equals_tile_path_bitwise(fw2, N, nl):
    """The persistent pipelined half steps compute exactly what the one-block-
    per-tile kernels compute (same arithmetic, staged operands), edge and
    interior tiles alike, on a ragged grid with many interior tiles."""
    prob = small_2d(nx=717, ny=333, N=N, nl=nl, steps=120, vel_src=True)
    _pipe_vs_tile(fw2, prob, 120)


def test_pipelined_path_equals_tile_path_cross_taps(fw2):
    """g11 cross taps (Sec. 3.1) on a zero-outside grid from a random state."""
    prob = synth.homogeneous((520, 200), 1e-4, 0.0)
    rng = np.random.default_rng(5)
    prob.c = (1500 + 200 * rng.random(prob.grid_shape)).astype(np.float32)
    prob.dt = 0.3 * 1e-4 / float(prob.c.max())
    taps = [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]
    prob.taps = (taps[0] * 0.98, taps[1], taps[2], taps[3], 0.005)
    _pipe_vs_tile(fw2, prob, 100, state=synth.random_state(prob, seed=3))


def test_parity_2d_time_space_taps(fw2):
    """The time-space optimised operator of Sec. 3.1 (library taps at the
    problem's Courant number, g11 != 0) against the oracle with the same taps;
    the pipelined path equals the tile path bitwise with them."""
    prob = small_2d(nx=560, ny=200, N=4, nl="pressure", steps=200)
    r = float(np.max(prob.c)) * prob.dt / prob.h
    prob.taps = tuple(fw2.fw2_taps_time_space(r))
    assert prob.taps[4] > 0
    compare_run(fw2, prob, 200)
    _pipe_vs_tile(fw2, prob, 120)


def test_periodic_grids_take_the_tile_kernels(fw2):
    prob = synth.homogeneous((144, 96), 1e-4, 0.0)
    prob.dt = 0.3 * 1e-4 / 1540.0
    prob.bc = ("periodic", "zero", "zero")
    sim = fw2.Simulation(prob, kernel_path="pipe")
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "tile"
    sim.close()


@pytest.mark.parametrize("nl", ["pressure", "off", "literal"])
def test_pipelined_path_equals_tile_path_tissue_index(fw2, nl):
    prob = synth.indexed_abdominal_problem(nx=650, ny=300, n_steps=150, n_elements=16, nl=nl)
    _pipe_vs_tile(fw2, prob, 150, maps="idx")


def test_parity_tissue_index_form(fw2):
    prob = synth.indexed_abdominal_problem(nx=320, ny=256, n_steps=300, n_elements=16)
    compare_run(fw2, prob, 300, maps="idx")


def test_parity_wide_tissue_index_form(fw2):
    """The uint16 index with more than 256 tissues (scatterer levels of 1023
    steps per class), tables read through L2 by the tile kernels."""
    prob = synth.indexed_abdominal_problem(nx=320, ny=256, n_steps=300, n_elements=16, levels=1024)
    assert prob.tissue.dtype == np.uint16 and len(np.unique(prob.tissue)) > 256
    sim = fw2.Simulation(prob, map_precision="idx16")
    sim.step(1)
    assert fw2.fw2_kernel_path(sim.ctx) == "tile"
    sim.close()
    compare_run(fw2, prob, 300, maps="idx16")
    with pytest.raises(ValueError):
        fw2.Simulation(prob, map_precision="idx")        # beyond the uint8 form


@pytest.mark.parametrize("nl", ["pressure", "literal"])
def test_wide_tissue_index_equals_uint8_index_bitwise(fw2, nl):
    """The same medium of at most 256 tissues as a uint16 index: the same
    fields and traces as the uint8 form (tile and pipelined kernels)."""
    prob = synth.indexed_abdominal_problem(nx=650, ny=300, n_steps=150, n_elements=16, nl=nl)
    out = {}
    for maps, path in (("idx", "tile"), ("idx", "pipe"), ("idx16", "auto")):
        sim = fw2.Simulation(prob, map_precision=maps, kernel_path=path)
        sim.step(150)
        out[(maps, path)] = ({n: sim.field(n) for n in ("p", "vx", "vy")}, sim.trace.cpu().numpy())
        sim.close()
    ref = out[("idx16", "auto")]
    for key in (("idx", "tile"), ("idx", "pipe")):
        for n in ("p", "vx", "vy"):
            np.testing.assert_array_equal(out[key][0][n], ref[0][n], err_msg=f"{key}: {n}")
        np.testing.assert_array_equal(out[key][1], ref[1])


def test_deterministic_bitwise(fw2):
    prob = small_2d(N=4, nl="pressure", steps=120, vel_src=True)
    out = []
    for _ in range(2):
        sim = fw2.Simulation(prob)
        sim.step(120)
        out.append((sim.field("p"), sim.trace.cpu().numpy()))
        sim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_split_steps_equal_one_call(fw2):
    """fw2_step(a) + fw2_step(b) == fw2_step(a + b) (source and trace rows follow the step index)."""
    prob = small_2d(steps=100)
    s1 = fw2.Simulation(prob); s1.step(100)
    s2 = fw2.Simulation(prob); s2.step(37); s2.step(0); s2.step(63)
    np.testing.assert_array_equal(s1.field("p"), s2.field("p"))
    np.testing.assert_array_equal(s1.trace.cpu().numpy(), s2.trace.cpu().numpy())


def test_device_inputs_equal_host_inputs(fw2):
    prob = small_2d(steps=50, vel_src=True)
    a = fw2.Simulation(prob); a.step(50)
    b = fw2.Simulation(prob, device_inputs=True); b.step(50)
    np.testing.assert_array_equal(a.field("p"), b.field("p"))
    np.testing.assert_array_equal(a.trace.cpu().numpy(), b.trace.cpu().numpy())


def test_steps_past_signal_and_trace_rows(fw2):
    """Sources fall silent and recording stops past their tables; rows past
    n_steps of the trace buffer are never written."""
    import torch
    prob = small_2d(steps=40)
    sim = fw2.Simulation(prob)
    sn = prob.sensors
    buf = torch.full((50, sn.n_groups), 7.0, device="cuda")
    fw2.fw2_record(sim.ctx, sn.idx, sn.group, sn.n_groups, buf, 40)
    sim.step(80)
    sim.synchronize()
    assert torch.all(buf[40:] == 7.0)
    assert not torch.any(buf[:40] == 7.0)
    orc = OracleSim(replace(synth.with_steps(prob, 80), sensors=None), round_to="f32")
    orc.run(80)
    assert_field("p", sim.field("p"), orc.field("p"))


@pytest.mark.parametrize("dims", [2, 3])
def test_empty_inputs(fw2, dims):
    """No sources, no sensors, zero steps: a zero state stays exactly zero on
    every path (the memory variables and the C-PML included), and zero steps
    change nothing."""
    shape = (200, 72) if dims == 2 else (140, 40, 24)
    prob = synth.homogeneous(shape, 1e-4, 0.0, relax=synth.relaxation_sets()["N2_y1.0_a0.5"])
    prob.dt = 0.3e-4 / 1540.0
    prob.pml_transition, prob.pml_bound = 6, 2
    for maps in ("f32", "bf16"):
        sim = fw2.Simulation(prob, map_precision=maps)
        sim.step(0)
        assert fw2.fw2_get_step(sim.ctx) == 0
        sim.step(7)
        sim.synchronize()
        assert fw2.fw2_get_step(sim.ctx) == 7
        for name in state_names(prob):
            assert not np.any(sim.field(name)), name
        sim.close()


def test_checkpoint_restore_is_bitwise(fw2):
    """Snapshot at step 60 (fields + step counter), restore into a fresh
    context, continue 40 steps: identical to an uninterrupted 100-step run."""
    prob = small_2d(N=4, steps=100, vel_src=True)
    full = fw2.Simulation(prob); full.step(100)
    a = fw2.Simulation(prob); a.step(60)
    snap = {n: a.field(n) for n in state_names(prob)}
    b = fw2.Simulation(prob)
    b.set_state(snap)
    fw2.fw2_set_step(b.ctx, fw2.fw2_get_step(a.ctx))
    b.step(40)
    for n in state_names(prob):
        np.testing.assert_array_equal(full.field(n), b.field(n))
    np.testing.assert_array_equal(full.trace.cpu().numpy()[60:], b.trace.cpu().numpy()[60:])


def test_reset_and_field_roundtrip(fw2):
    prob = small_2d(steps=30)
    sim = fw2.Simulation(prob)
    sim.step(30)
    p = sim.field("p")
    assert np.abs(p).max() > 0
    fw2.fw2_reset(sim.ctx)
    assert np.abs(sim.field("p")).max() == 0 and fw2.fw2_get_step(sim.ctx) == 0
    sim.set_state({"p": p})
    np.testing.assert_array_equal(sim.field("p"), p)


def test_check_field_flags_nonfinite(fw2):
    """Failure detection without a GPU fault: a NaN planted from the host."""
    prob = small_2d(steps=10)
    sim = fw2.Simulation(prob)
    sim.step(10)
    st, m = fw2.fw2_check_field(sim.ctx, 1e9)
    assert st == fw2.OK and 0 < m < 1e9
    p = sim.field("p")
    p[5, 7] = np.nan
    sim.set_state({"p": p})
    st, m = fw2.fw2_check_field(sim.ctx, 1e9)
    assert st == fw2.EUNSTABLE and math.isinf(m)
    assert "max |p|" in fw2.fw2_last_error(sim.ctx)


def test_step_before_medium_is_a_state_error(fw2):
    prob = small_2d(steps=10)
    cfg = fw2.config_for(prob)
    ctx = fw2.fw2_create(cfg)
    try:
        with pytest.raises(fw2.Fw2Error) as e:
            fw2.fw2_step(ctx, 1)
        assert e.value.status == fw2.ESTATE
    finally:
        fw2.fw2_destroy(ctx)


def test_unstable_time_step_rejected(fw2):
    prob = small_2d(steps=10)
    prob.dt = prob.dt * 2.0
    with pytest.raises(fw2.Fw2Error) as e:
        fw2.Simulation(prob)
    assert e.value.status == fw2.EINVAL and "stability" in str(e.value)


def test_bad_medium_rejected(fw2):
    prob = small_2d(steps=10)
    prob.c = prob.c.copy()
    prob.c[3, 3] = -1.0
    with pytest.raises(fw2.Fw2Error) as e:
        fw2.Simulation(prob)
    assert e.value.status == fw2.EINVAL


def test_cfl_time_step_matches_oracle_rule(fw2):
    from oracle import coefficients as cf
    prob = small_2d(N=4, steps=10)
    prob.dt = 0.0
    sim = fw2.Simulation(prob)
    assert abs(sim.dt / cf.cfl_time_step(prob, 0.4) - 1) < 1e-15


def test_context_memory_is_reused_and_released(fw2):
    """Device memory comes from the library's pool: a context created after
    another of the same size was destroyed takes no new memory from the
    driver, and fw2_release_memory gives the pool's free memory back."""
    import torch
    prob = small_2d(nx=512, ny=400, N=4, steps=5)
    s = fw2.Simulation(prob)
    s.step(2)
    s.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = fw2.Simulation(prob)
    s.step(2)
    s.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    held = fw2.fw2_device_bytes(s.ctx)
    s.close()
    assert free1 == free0
    fw2.fw2_release_memory()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 >= free0 + held // 2
