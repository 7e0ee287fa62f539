"""Batched persistent stepping: every context in a batch computes exactly what
it computes alone (the same result alone and in the mix)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def _problems():
    probs = []
    for t in range(3):   # full-synthetic-aperture style: one element fires per event
        probs.append(("idx", synth.indexed_abdominal_problem(nx=260, ny=170, n_steps=95, n_elements=8,
                                                            transmit=t, pml_lambda=(1.0, 0.5))))
    probs.append(("idx", synth.indexed_abdominal_problem(nx=131, ny=97, n_steps=95, n_elements=4,
                                                        pml_lambda=(1.0, 0.5), seed=7)))
    from tests.test_gpu_parity import small_2d
    probs.append(("f32", small_2d(nx=200, ny=136, N=2, steps=95)))
    probs.append(("f32", small_2d(nx=150, ny=60, N=4, nl="pressure", steps=95, pml=(6, 2), vel_src=True)))
    probs.append(("bf16", small_2d(nx=96, ny=96, N=4, steps=95, pml=(6, 2))))
    # both nonlinear factors, grouped with the linear N = 2 context above
    probs.append(("f32", small_2d(nx=180, ny=100, N=2, nl="literal", steps=95, amp=2e7)))
    # more mechanisms than the pipelined kernels take: batched tile kernels
    probs.append(("f32", small_2d(nx=140, ny=90, N=6, steps=95, pml=(6, 2))))
    probs.append(("bf16", small_2d(nx=100, ny=70, N=8, nl="pressure", steps=95, pml=(6, 2))))
    # FP16 maps: batched tile kernels
    probs.append(("f16", small_2d(nx=120, ny=90, N=3, nl="pressure", steps=95, pml=(6, 2))))
    # the uint16 index with more than 256 tissues: batched tile kernels
    probs.append(("idx16", synth.indexed_abdominal_problem(nx=140, ny=100, n_steps=95, n_elements=4,
                                                          pml_lambda=(1.0, 0.5), seed=9, levels=300)))
    return probs


def test_batch_equals_each_context_alone(fw2):
    steps = 90                     # 13 tuning steps, four 16-step graphs, 13 plain
    probs = _problems()
    alone = []
    for maps, p in probs:
        s = fw2.Simulation(p, map_precision=maps)
        if maps == "f32" and p.nrelax == 4:
            s.step(5)              # a context that starts at another step
        s.step(steps)
        alone.append((s.field("p"), s.field("vx"), s.trace.cpu().numpy()))
        s.close()
    sims = []
    for maps, p in probs:
        s = fw2.Simulation(p, map_precision=maps)
        if maps == "f32" and p.nrelax == 4:
            s.step(5)
        sims.append(s)
    batch = fw2.fw2_batch_create([s.ctx for s in sims])
    try:
        fw2.fw2_batch_step(batch, steps)
        fw2.fw2_batch_synchronize(batch)
        grid, order, launches = fw2.fw2_batch_info(batch)
        assert grid > 0 and order in (0, 1) and launches > 0
        assert fw2.fw2_batch_edge_weight(batch) in (1.5, 2.5, 3.5, 5.0)
        for (p_ref, vx_ref, tr_ref), s in zip(alone, sims):
            np.testing.assert_array_equal(s.field("p"), p_ref)
            np.testing.assert_array_equal(s.field("vx"), vx_ref)
            np.testing.assert_array_equal(s.trace.cpu().numpy(), tr_ref)
        # the contexts' own counters advanced; a further single step continues
        for s in sims:
            assert fw2.fw2_get_step(s.ctx) in (steps, steps + 5)
    finally:
        fw2.fw2_batch_destroy(batch)
        for s in sims:
            s.close()


def test_batch_rejects_3d_contexts_off_the_pipelined_path(fw2):
    from tests.test_gpu_parity import small_3d
    s = fw2.Simulation(small_3d(steps=5))            # float maps: tile kernels only
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_batch_create([s.ctx])
    s.close()


def test_3d_contexts_in_a_batch_equal_each_alone(fw2):
    """3D contexts (bf16 maps) of different sizes, mechanism counts, with and
    without the cross taps and the literal system, batched with 2D ones and
    uneven budgets: each holds bitwise what it holds alone."""
    from tests.test_gpu_parity import small_2d, small_3d
    probs = [("bf16", small_3d(n=(150, 44, 40), N=3, nl="westervelt", steps=60)),
             ("bf16", small_3d(n=(90, 70, 30), N=2, nl="off", steps=60, seed=5)),
             ("bf16", small_3d(n=(130, 40, 36), N=3, nl="literal", steps=60, seed=7)),
             ("bf16", small_3d(n=(100, 50, 32), N=3, nl="pressure", steps=60, seed=9)),
             ("f32", small_2d(nx=200, ny=136, N=2, steps=60))]
    r = float(np.max(probs[3][1].c)) * probs[3][1].dt / probs[3][1].h
    probs[3][1].taps = tuple(fw2.fw2_taps_time_space(r, 3))
    budgets = [60, 41, 60, 52, 33]
    alone = []
    for (maps, p), n in zip(probs, budgets):
        s = fw2.Simulation(p, map_precision=maps)
        s.step(n)
        alone.append((s.field("p"), s.field("vx"), s.trace.cpu().numpy()[:n]))
        s.close()
    sims = [fw2.Simulation(p, map_precision=maps) for maps, p in probs]
    batch = fw2.fw2_batch_create([s.ctx for s in sims])
    try:
        fw2.fw2_batch_set_budget(batch, budgets)
        fw2.fw2_batch_step(batch, 100)
        fw2.fw2_batch_synchronize(batch)
        for s, n, (p_ref, vx_ref, tr_ref) in zip(sims, budgets, alone):
            assert fw2.fw2_get_step(s.ctx) == n
            np.testing.assert_array_equal(s.field("p"), p_ref)
            np.testing.assert_array_equal(s.field("vx"), vx_ref)
            np.testing.assert_array_equal(s.trace.cpu().numpy()[:n], tr_ref)
    finally:
        fw2.fw2_batch_destroy(batch)
        for s in sims:
            s.close()


def test_batch_full_size_equals_each_context_alone(fw2):
    """The benchmark's batch (64 focused transmits over one 2048 x 1024
    tissue-index medium and 16 uneven instances, 151 M cells) after the
    thirteen autotuning steps and three more: sampled contexts hold bitwise
    what they hold when stepped alone."""
    import types
    import bench
    probs, _ = bench.batch_problems(types.SimpleNamespace(warmup=8, steps=8, batch_steps=8), 0)
    steps = 16
    sims = [fw2.Simulation(p, map_precision="idx") for p in probs]
    batch = fw2.fw2_batch_create([s.ctx for s in sims])
    try:
        fw2.fw2_batch_step(batch, steps)
        fw2.fw2_batch_synchronize(batch)
        picked = [0, 31, 63, 64, 71, 79]
        got = {i: (sims[i].field("p"), sims[i].field("vy"), sims[i].trace.cpu().numpy()[:steps]) for i in picked}
    finally:
        fw2.fw2_batch_destroy(batch)
        for s in sims:
            s.close()
    for i in picked:
        s = fw2.Simulation(probs[i], map_precision="idx")
        s.step(steps)
        np.testing.assert_array_equal(got[i][0], s.field("p"))
        np.testing.assert_array_equal(got[i][1], s.field("vy"))
        np.testing.assert_array_equal(got[i][2], s.trace.cpu().numpy()[:steps])
        s.close()


def test_batch_budgets_let_contexts_leave_and_equal_each_context_alone(fw2):
    """Uneven step budgets: every context stops at its own budget (the batch
    rebuilds its launch tables as contexts leave) and holds bitwise what it
    holds when stepped alone for that many steps."""
    probs = _problems()
    budgets = [40, 95, 17, 70, 95, 33, 60, 81, 52, 29, 44, 66]
    alone = []
    for (maps, p), n in zip(probs, budgets):
        s = fw2.Simulation(p, map_precision=maps)
        s.step(n)
        alone.append((s.field("p"), s.field("vy"), s.trace.cpu().numpy()[:n]))
        s.close()
    sims = [fw2.Simulation(p, map_precision=maps) for maps, p in probs]
    batch = fw2.fw2_batch_create([s.ctx for s in sims])
    try:
        with pytest.raises(ValueError):
            fw2.fw2_batch_set_budget(batch, budgets[:-1])
        fw2.fw2_batch_set_budget(batch, budgets)
        assert fw2.fw2_batch_active(batch) == len(sims)
        fw2.fw2_batch_step(batch, 50)
        fw2.fw2_batch_synchronize(batch)
        assert fw2.fw2_batch_active(batch) == sum(b > 50 for b in budgets)
        fw2.fw2_batch_step(batch, 1000)
        fw2.fw2_batch_synchronize(batch)
        assert fw2.fw2_batch_active(batch) == 0
        for s, n, (p_ref, vy_ref, tr_ref) in zip(sims, budgets, alone):
            assert fw2.fw2_get_step(s.ctx) == n
            np.testing.assert_array_equal(s.field("p"), p_ref)
            np.testing.assert_array_equal(s.field("vy"), vy_ref)
            np.testing.assert_array_equal(s.trace.cpu().numpy()[:n], tr_ref)
    finally:
        fw2.fw2_batch_destroy(batch)
        for s in sims:
            s.close()
