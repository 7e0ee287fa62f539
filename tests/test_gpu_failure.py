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
