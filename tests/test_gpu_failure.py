"""Failure detection on the GPU without a GPU fault: the bounded wait that
guards every copy barrier of the pipelined kernels gives up on a barrier
nobody arrives on, returns an error status to the host, and the device stays
usable."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def test_bounded_wait_gives_up_and_device_stays_usable(fw2):
    import time
    t0 = time.perf_counter()
    assert fw2.fw2_selftest_bounded_wait(2_000_000) is True      # 2 ms limit
    assert time.perf_counter() - t0 < 5.0
    # the context after the timed-out wait still steps and synchronises cleanly
    prob = synth.homogeneous((256, 192), 1e-4, 0.0)
    prob.dt = 0.3 * 1e-4 / 1540.0
    prob.sources = [synth.Source("p", synth.flat_index((256, 192), [128], [96]), np.zeros(1, np.int32),
                                 np.ones((8, 1), np.float32))]
    sim = fw2.Simulation(prob, kernel_path="pipe")
    sim.step(20)
    fw2.fw2_synchronize(sim.ctx)
    assert np.isfinite(sim.field("p")).all() and np.abs(sim.field("p")).max() > 0
    sim.close()


def test_bounded_wait_rejects_bad_limits(fw2):
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_selftest_bounded_wait(0)


def _cpml_problem(reading, lt_lambda, lb_lambda, n_steps):
    """2D Table 2 tissue (N = 2) at 16 points per wavelength, CFL 0.4, a line
    source of one 1 MHz pulse, the two-stage C-PML of the given reading."""
    import math
    c0, f0, ppw = 1540.0, 1e6, 16
    h = c0 / f0 / ppw
    relax = synth.TABLE2
    keff = math.sqrt(float(np.float32(relax["kappa1"])) * float(np.float32(relax["kappa2"])))
    dt = 0.4 * h / (c0 / keff)
    shape = (300, 150)
    prob = synth.homogeneous(shape, h, dt, c=c0, rho=1000.0, relax=relax)
    prob.pml_transition, prob.pml_bound = int(lt_lambda * ppw), int(lb_lambda * ppw)
    prob.pml_reading = reading
    xs = np.arange(100, 200)
    sig = synth.gaussian_pulse(400, dt, f0, 3.0, 1.0)
    prob.sources = [synth.Source("p", synth.flat_index(shape, xs, 75), np.zeros(xs.size, np.int32), sig[:, None])]
    prob.n_steps = n_steps
    return prob


def test_watch_stops_the_multi_mechanism_cpml_without_transition_layer(fw2):
    """Sec. 3.3: with N = 2 mechanisms kept inside the C-PML (no transition
    layer) the scheme is unstable; with the watch on, fw2_step returns
    FW2_EUNSTABLE once |p| passes the bound, without a fault, and the
    context stays usable.  The same medium with the transition layer runs
    as many steps without tripping the same watch."""
    bad = fw2.Simulation(_cpml_problem("K", 0, 4, 400))
    bad.step(3000)
    bad.synchronize()
    _, m0 = fw2.fw2_check_field(bad.ctx, float("inf"))
    bound = 1e3 * max(m0, 1e-3)
    fw2.fw2_set_watch(bad.ctx, 1000, bound)
    steps_at_fail = None
    for _ in range(40):
        try:
            bad.step(20000)
        except fw2.Fw2Error as e:
            assert e.status == fw2.EUNSTABLE and "blew up" in str(e)
            steps_at_fail = fw2.fw2_get_step(bad.ctx)
            break
    assert steps_at_fail is not None, "the unstable C-PML never passed the bound"
    assert steps_at_fail % 1000 == 0
    st, m = fw2.fw2_check_field(bad.ctx, float("inf"))
    assert not (m <= bound)                        # the field that tripped the watch
    fw2.fw2_reset(bad.ctx)                         # still usable
    bad.step(10)
    fw2.fw2_synchronize(bad.ctx)
    bad.close()
    good = fw2.Simulation(_cpml_problem("C", 3, 1, 400))
    fw2.fw2_set_watch(good.ctx, 1000, bound)
    good.step(steps_at_fail)
    _, mg = fw2.fw2_check_field(good.ctx, float("inf"))
    assert mg < 1e-2 * m0
    good.close()


def test_watch_flags_a_planted_nonfinite_value(fw2):
    """A NaN written into p from the host is caught at the next scan; the
    steps before it are counted."""
    prob = synth.homogeneous((256, 192), 1e-4, 0.0)
    prob.dt = 0.3 * 1e-4 / 1540.0
    sim = fw2.Simulation(prob)
    fw2.fw2_set_watch(sim.ctx, 7, 1.0)
    sim.step(10)                                   # scans at 7: zero field passes
    p = sim.field("p")
    p[50, 60] = np.nan
    fw2.fw2_set_field(sim.ctx, "p", p)
    with pytest.raises(fw2.Fw2Error) as e:
        sim.step(10)
    assert e.value.status == fw2.EUNSTABLE
    assert fw2.fw2_get_step(sim.ctx) == 14
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_set_watch(sim.ctx, 5, 0.0)
    fw2.fw2_set_watch(sim.ctx, 0, 0.0)             # off: no scan, no error
    sim.step(3)
    sim.close()


def test_batch_watch_names_the_context_that_blew_up(fw2):
    """A batch with the watch on stops at the first scan after a NaN is
    planted in one context, names that context, and counts the steps taken
    on every context."""
    probs = [synth.indexed_abdominal_problem(nx=256, ny=160, n_steps=60, n_elements=4, seed=s,
                                             pml_lambda=(1.0, 0.5)) for s in (1, 2, 3)]
    sims = [fw2.Simulation(p, map_precision="idx") for p in probs]
    p = sims[1].field("p")
    p[80, 100] = np.inf
    fw2.fw2_set_field(sims[1].ctx, "p", p)
    batch = fw2.fw2_batch_create([s.ctx for s in sims])
    try:
        fw2.fw2_batch_set_watch(batch, 5, 1e12)
        with pytest.raises(fw2.Fw2Error) as e:
            fw2.fw2_batch_step(batch, 30)
        assert e.value.status == fw2.EUNSTABLE and "context 1" in str(e.value)
        for s in sims:
            assert fw2.fw2_get_step(s.ctx) == 5
    finally:
        fw2.fw2_batch_destroy(batch)
        for s in sims:
            s.close()
