"""Serving loop: requests admitted as they arrive and stepped together give
the same traces as each request run alone."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def test_served_results_equal_alone(fw2):
    from paper_2106_11476_gb300.serve import Request, Server, latency_stats
    from tests.test_gpu_parity import small_2d, small_3d
    probs = [
        ("idx", synth.indexed_abdominal_problem(nx=200, ny=150, n_steps=70, n_elements=8, transmit=1,
                                                pml_lambda=(1.0, 0.5))),
        ("idx", synth.indexed_abdominal_problem(nx=150, ny=120, n_steps=45, n_elements=6, seed=5,
                                                pml_lambda=(1.0, 0.5))),
        ("f32", small_2d(nx=128, ny=96, N=4, steps=55, pml=(6, 2))),
        ("f32", small_3d(n=(40, 36, 32), steps=50)),
        ("bf16", small_3d(n=(140, 40, 30), N=2, nl="off", steps=40, seed=6)),   # joins the batch
    ]
    reqs = [Request(i, arrival=0.004 * i, problem=p, steps=p.n_steps, maps=m) for i, (m, p) in enumerate(probs)]
    done = Server(cap_bytes=2e9, slice_steps=16).run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3, 4]
    for r in done:
        alone = fw2.Simulation(r.problem, map_precision=r.maps)
        alone.step(r.steps)
        np.testing.assert_array_equal(r.trace, alone.trace.cpu().numpy(), err_msg=str(r.rid))
        alone.close()
        assert r.finished >= r.arrival
    st = latency_stats(done)
    assert st["p99_s"] >= st["p50_s"] > 0


def test_admission_respects_the_memory_cap(fw2):
    from paper_2106_11476_gb300.serve import Request, Server, footprint_bytes
    p = synth.indexed_abdominal_problem(nx=160, ny=128, n_steps=20, n_elements=4, pml_lambda=(1.0, 0.5))
    fp = footprint_bytes(p, "idx")
    reqs = [Request(i, 0.0, p, 20, "idx") for i in range(4)]
    srv = Server(cap_bytes=2.5 * fp, slice_steps=10)
    done = srv.run(reqs)
    assert len(done) == 4
    assert max(e["n_batch"] for e in srv.launch_log) <= 2
