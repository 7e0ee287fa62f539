"""Parity at the step counts the workloads are quoted on: crops of the 2D
abdominal-wall medium (nonlinear, N = 4, C-PML) for 8000 steps and of the 3D
transcranial medium (bf16 maps, N = 3, C-PML) for 4000 steps, element by
element against the FP64 oracle on the same stored maps, at checkpoints
along the run, and the whole sensor history.

The source fires a pulse every 1000 steps so that the field stays energetic
to the end (a single pulse leaves the crop within about a thousand steps and
only round-off would be compared after that)."""
import numpy as np
import pytest

import synth
from oracle.core import OracleSim
from tests.test_gpu_parity import MAX_REL, REL_L2, TRACE_DB, max_rel, rel_l2, trace_db

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def pulse_train(prob, period):
    """Each source signal replaced by its own first `period` rows repeated
    along the whole run."""
    for s in prob.sources:
        head = np.asarray(s.signal[:period], np.float32)
        reps = -(-prob.n_steps // period)
        s.signal = np.ascontiguousarray(np.tile(head, (reps, 1))[:prob.n_steps])
    return prob


def long_run(fw2, prob, maps, checkpoints, fields):
    sim = fw2.Simulation(prob, map_precision=maps)
    orc = OracleSim(prob, round_to=maps)
    done, worst = 0, {}
    for cp in checkpoints:
        sim.step(cp - done)
        orc.run(cp - done)
        sim.synchronize()
        done = cp
        for name in fields:
            g, o = sim.field(name), orc.field(name)
            r, m = rel_l2(g, o), max_rel(g, o)
            worst[name] = max(worst.get(name, (0, 0)), (r, m))
            assert r <= REL_L2 and m <= MAX_REL, f"step {cp}, {name}: rel L2 {r:.3e}, max/peak {m:.3e}"
    db = trace_db(sim.trace.cpu().numpy()[:done], orc.trace[:done])
    sim.close()
    assert db <= TRACE_DB, f"trace error over {done} steps: {db:.1f} dB"
    return worst, db


def test_abdominal_crop_8000_steps(fw2):
    """320 x 320 cells of the abdominal-wall medium (fat / muscle / connective
    layers, beta 4-6, scatterers, N = 4, pressure nonlinearity, float maps,
    3 + 1 wavelength C-PML), a 20-element focused array, 8000 steps."""
    prob = synth.abdominal_problem(n=320, n_steps=8000, seed=5, n_elements=20)
    pulse_train(prob, 1000)
    long_run(fw2, prob, "f32", (2000, 4000, 6000, 8000), ("p", "vx", "vy"))


def test_skull_crop_4000_steps(fw2):
    """96^3 cells of the transcranial medium (brain with the skull shell's
    porous bone where the crop reaches it, N = 3, bf16 maps, 16-cell C-PML
    on every face), a 4 x 4 planar array, 4000 steps."""
    prob = synth.skull_problem(n=96, n_steps=4000, seed=7, pml_cells=16, array_elems=4)
    pulse_train(prob, 1000)
    long_run(fw2, prob, "bf16", (1000, 2000, 3000, 4000), ("p", "vx", "vy", "vz"))
