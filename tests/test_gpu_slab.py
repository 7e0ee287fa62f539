"""One grid split into slabs (paper_2106_11476_gb300/slab.py): the slabs
advanced as contexts of one device, with their extra rows of p and v_q
copied from the neighbours between the half steps, hold bitwise what one
context of the whole grid holds -- fields, memory variables and traces --
with the C-PML placed by each slab's position in the whole grid."""
import numpy as np
import pytest

import synth
from paper_2106_11476_gb300 import slab
from tests.test_gpu_parity import small_3d, state_names

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def _compare(fw2, prob, parts, steps, maps="f32", kernel_path="auto"):
    whole = fw2.Simulation(prob, map_precision=maps, kernel_path=kernel_path)
    whole.step(steps)
    group = slab.SlabGroup(prob, parts, map_precision=maps, kernel_path=kernel_path)
    group.step(steps)
    try:
        for n in state_names(prob):
            np.testing.assert_array_equal(group.field(n), whole.field(n), err_msg=n)
        if prob.sensors is not None:
            np.testing.assert_array_equal(group.trace()[:steps], whole.trace.cpu().numpy()[:steps])
    finally:
        group.close()
        whole.close()


@pytest.mark.parametrize("parts", [2, 3])
def test_abdominal_slabs_equal_the_whole_grid(fw2, parts):
    """2D abdominal-wall medium (nonlinear, N = 4, float maps, C-PML on all
    faces, focused array), split along y across the array and the layers."""
    prob = synth.abdominal_problem(n=384, n_steps=120, n_elements=12, pml_lambda=(1.0, 0.5), ny=300)
    _compare(fw2, prob, parts, 120)


def test_tissue_index_slabs_equal_the_whole_grid(fw2):
    prob = synth.indexed_abdominal_problem(nx=300, ny=260, n_steps=90, n_elements=8, pml_lambda=(1.0, 0.5))
    _compare(fw2, prob, 2, 90, maps="idx")


@pytest.mark.parametrize("nl,taps", [("westervelt", False), ("literal", True)])
def test_3d_slabs_equal_the_whole_grid(fw2, nl, taps):
    """3D bf16 maps on the pipelined half steps, split along z; with the
    time-space cross taps and the literal system (whose momentum factor and
    cross taps read the neighbouring rows too)."""
    prob = small_3d(n=(140, 40, 60), N=3, nl=nl, steps=50)
    if taps:
        r = float(np.max(prob.c)) * prob.dt / prob.h
        prob.taps = tuple(fw2.fw2_taps_time_space(r, 3))
    _compare(fw2, prob, 3, 50, maps="bf16")


def test_step_parts_and_rows_reject_misuse(fw2):
    prob = synth.line_source_problem(n=96, n_steps=10, n_sensors=4, pml_lambda=(1.0, 0.5))
    sim = fw2.Simulation(prob)
    fw2.fw2_step_part(sim.ctx, 0)
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_step(sim.ctx, 1)                 # the step begun must be completed
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_step_part(sim.ctx, 0)
    fw2.fw2_step_part(sim.ctx, 1)
    assert fw2.fw2_get_step(sim.ctx) == 1
    buf = np.zeros((4, 96), np.float32)
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_get_rows(sim.ctx, "p", 94, 4, buf)   # past the last row
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_get_rows(sim.ctx, "psi1x", 0, 4, buf)
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_set_subdomain(sim.ctx, (96, 90), (0, 0))  # the grid does not fit
    sim.close()
