"""Host logic of bench.py: the algorithmic bytes behind the roofline fraction
(counted by hand from the arrays each half step must read and write once)
and the committed DRAM traffic lookup."""
import json
import os

import pytest

import bench


def test_algorithmic_bytes_2d_by_hand():
    """2D, N = 4, nonlinear, float maps, no C-PML: the compulsory bytes of a
    step (each state array read and written once, each map read once) split
    by the array each half step updates.  Velocity: v_x, v_y and 8 memory
    variables read and written, rho, 1/kappa1 and a, b of 4 mechanisms:
    16 + 64 + 4 + 4 + 32 = 120 B per cell; pressure: p and 8 memory
    variables read and written, K, chi, 1/kappa2, a, b: 8 + 64 + 4 + 4 + 4
    + 32 = 116 B (236 B per cell-step)."""
    n = 1000 * 700
    vel, prs = bench.algorithmic_bytes((1000, 700), 4, 0, True, map_bytes=4)
    assert vel == 120 * n and prs == 116 * n
    vel, prs = bench.algorithmic_bytes((1000, 700), 4, 0, False, map_bytes=4)
    assert prs == 112 * n                                  # no chi
    vel, _ = bench.algorithmic_bytes((1000, 700), 4, 0, True, map_bytes=4, nl_vel=True)
    assert vel == 124 * n                                  # K in the velocity half step


def test_split_overhead_is_the_second_operand_read():
    """The two-launch split reads p again in the velocity half step and v_q
    again in the pressure half step: 4 and 4 D bytes per cell (and the
    tissue index again in the index form)."""
    n = 64 * 48
    assert bench.split_overhead_bytes((64, 48)) == (4 * n, 8 * n)
    assert bench.split_overhead_bytes((64, 48), indexed=True) == (4 * n, 9 * n)
    assert bench.split_overhead_bytes((8, 8, 8)) == (4 * 512, 12 * 512)


def test_algorithmic_bytes_3d_bf16_by_hand():
    """3D, N = 3, linear, bf16 maps, no C-PML: velocity 24 (v) + 72 (psi) + 2
    (rho) + 2 (1/kappa1) + 12 (a, b) = 112 B; pressure 8 (p) + 72 + 2 (K) + 2
    + 12 = 96 B per cell."""
    n = 64 * 48 * 40
    vel, prs = bench.algorithmic_bytes((64, 48, 40), 3, 0, False, map_bytes=2)
    assert vel == 112 * n and prs == 96 * n


def test_strip_bytes_count_each_axis_inside_its_strip():
    """A cell inside the C-PML of k axes reads k strip sets of a, b (one per
    axis) plus the interior set when some axis is outside its strip."""
    shape, N, L = (40, 30), 2, 5
    vel0, _ = bench.algorithmic_bytes(shape, N, 0, False)
    vel, _ = bench.algorithmic_bytes(shape, N, L, False)
    per_set = 2 * N * 4
    nx, ny = shape
    corner = (2 * L) * (2 * L)                           # both axes in a strip: 2 sets
    edge = (2 * L) * (ny - 2 * L) + (nx - 2 * L) * (2 * L)  # one axis: strip + interior
    assert vel - vel0 == (corner * 1 + edge * 1) * per_set


def test_index_form_bytes():
    """8 bytes per state array and one index byte per cell-step: 153 B."""
    n = 512 * 256
    vel, prs = bench.algorithmic_bytes_indexed((512, 256), 4, 0, True)
    assert vel == n * (1 + 16 + 64) and prs == n * (8 + 64)
    assert vel + prs == n * (8 * 19 + 1)


def test_exact_region_keeps_margins_only_at_cut_edges():
    """The parity region stays `margin` cells away from the window's edges
    inside the grid, but reaches the grid's own boundary."""
    sl, reg = bench.exact_region(((100, 612), (0, 512)), (4096, 4096), 32)
    assert reg == [(132, 580), (0, 480)]
    assert sl == (slice(0, 480), slice(32, 480))
    sl, reg = bench.exact_region(((0, 512), (0, 512)), (512, 512), 32)
    assert reg == [(0, 512), (0, 512)]


def test_committed_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The committed traffic is used only while the sources of its kernel
    family (2D or 3D pipeline) are the ones it was captured with."""
    real = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key in (k for k in real if not k.startswith("_")):
        family = "pipe3d" if ":pipe3d" in key else "pipe2d"
        if real[key]["source_hash"] == bench.kernel_source_hash(family):
            assert bench.committed_traffic(key) == real[key]["dram_bytes_per_launch"]
        else:
            assert bench.committed_traffic(key) is None
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "profiles" / "traffic.json").write_text(json.dumps({
        "w:f32:1:pipe2d_vel": {"dram_bytes_per_launch": 5, "source_hash": "stale"},
        "w:f32:1:pipe2d_prs": {"dram_bytes_per_launch": 7, "source_hash": "current2d"},
        "w:bf16:1:pipe3d_vel": {"dram_bytes_per_launch": 9, "source_hash": "current2d"}}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda family="pipe2d": "current" + family[-2:])
    assert bench.committed_traffic("w:f32:1:pipe2d_prs") == 7
    assert bench.committed_traffic("w:f32:1:pipe2d_vel") is None
    assert bench.committed_traffic("w:bf16:1:pipe3d_vel") is None   # another family's sources
    assert bench.committed_traffic("missing") is None


def test_fcfs_plain_queues_behind_earlier_requests():
    ttr, span = bench.fcfs_plain([0.0, 1.0, 10.0], [3.0, 2.0, 1.0])
    # the second waits for the first (free at 3), the third finds the device idle
    assert ttr == [3.0, 4.0, 1.0] and span == 11.0


def test_serve_requests_mix_and_rate_free_arrivals():
    specs = bench.serve_requests(200, 1.0, 0)
    assert len(specs) == 200 and [q["rid"] for q in specs] == list(range(200))
    t = [q["t"] for q in specs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert 150 < t[-1] < 250                                # one arrival per second on average
    n3 = sum(len(q["shape"]) == 3 for q in specs)
    assert 40 <= n3 <= 80                                   # about 30 % 3D
    for q in specs:
        side = q["shape"][0]
        if len(q["shape"]) == 2:
            assert 512 <= side <= 4096 and side % 4 == 0 and q["maps"] == "idx"
            assert 1000 <= q["steps"] <= 4000
        else:
            assert 256 <= side <= 512 and q["maps"] == "bf16" and 1000 <= q["steps"] <= 2000
    # the same seeded stream whatever the scale's effect on sizes
    small = bench.serve_requests(200, 0.25, 0)
    assert [q["t"] for q in small] == t


def test_problem_feed_hands_out_in_order_and_stops_the_clock():
    made = []

    def maker(i):
        def make():
            made.append(i)
            return i * 10
        return make
    specs = [{"make": maker(i)} for i in range(5)]
    clock = bench.InputClock()
    feed = bench.ProblemFeed(specs, clock, ahead=2)
    assert [feed.get(i) for i in range(5)] == [0, 10, 20, 30, 40]
    feed.close()
    assert made == [0, 1, 2, 3, 4]
    assert clock.stopped == pytest.approx(feed.waited) and clock.stopped >= 0.0


def test_oracle_baseline_reports_the_threads_used_and_a_single_core_rate():
    """The cpu_baseline leg states the OpenMP threads the oracle ran on and,
    beside the all-core rate, the rate on one core; the thread count is back
    to what it was afterwards."""
    import synth
    before = bench.oracle_threads()
    prob = synth.line_source_problem(n=160, n_steps=40, seed=0)
    out = bench.oracle_baseline(prob, 16, ((0, 160), (0, 160)), media=False)
    assert out["kind"] == "oracle" and out["value"] > 0
    assert out["cores"] == before >= 1
    if before > 1 and bench._openmp() is not None:
        one = out["single_core"]
        assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == out["unit"]
    assert bench.oracle_threads() == before
