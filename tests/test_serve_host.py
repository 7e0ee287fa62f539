"""Host logic of the serving loop (serve.py) on the CPU, with the library
calls replaced by fakes that count steps: admission in arrival order under
the memory cap, slices of at most `slice_steps`, 2D and bf16 3D requests
advanced together as one batch (rebuilt when the set changes), other 3D
requests on their own, every request stepped exactly its step count."""
import types

import numpy as np
import pytest

from paper_2106_11476_gb300 import serve


class _Trace:
    def __init__(self, steps):
        self.steps = steps

    def cpu(self):
        return self

    def numpy(self):
        return np.full(1, float(self.steps))


class _Sim:
    live = 0
    peak = 0

    def __init__(self, prob, map_precision="f32", stream=None):
        self.prob = prob
        self.maps = map_precision
        self.ctx = object()
        self.steps = 0
        self.closed = False
        _Sim.live += 1
        _Sim.peak = max(_Sim.peak, _Sim.live)

    def step(self, k):
        assert self.maps != "bf16" and len(self.prob.shape) == 3, "batchable requests advance through the batch"
        self.steps += k

    def synchronize(self):
        pass

    @property
    def trace(self):
        return _Trace(self.steps)

    def close(self):
        assert not self.closed
        self.closed = True
        _Sim.live -= 1


def _install_fakes(monkeypatch):
    sims = {}
    batches = []
    orig_init = _Sim.__init__

    def init(self, prob, map_precision="f32", stream=None):
        orig_init(self, prob, map_precision, stream)
        sims[id(self.ctx)] = self

    monkeypatch.setattr(_Sim, "__init__", init)
    _Sim.live = 0
    _Sim.peak = 0
    budgets = {}

    def bstep(b, n):
        for s, last in zip(batches[b], budgets.get(b, [None] * len(batches[b]))):
            s.steps += n if last is None else max(0, min(n, last - s.steps))
    fake = types.SimpleNamespace(
        Simulation=_Sim,
        fw2_batch_create=lambda ctxs: (batches.append([sims[id(c)] for c in ctxs]) or len(batches) - 1),
        fw2_batch_set_budget=lambda b, last: budgets.__setitem__(b, list(last)),
        fw2_batch_step=bstep,
        fw2_batch_synchronize=lambda b: None,
        fw2_batch_destroy=lambda b: None)
    monkeypatch.setattr(serve, "fw2", fake)
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    return batches


def _prob(shape, N=2, L=4):
    return types.SimpleNamespace(shape=shape, nrelax=N, pml_transition=L - 1, pml_bound=1)


def _clock():
    t = [0.0]

    def tick():
        t[0] += 1e-3
        return t[0]
    return tick


def test_every_request_runs_its_steps_in_slices(monkeypatch):
    batches = _install_fakes(monkeypatch)
    reqs = [serve.Request(0, 0.0, _prob((64, 48)), 250), serve.Request(1, 0.0, _prob((80, 40)), 120),
            serve.Request(2, 0.0, _prob((32, 32, 24)), 230), serve.Request(3, 0.0, _prob((40, 40)), 75)]
    srv = serve.Server(cap_bytes=1e12, slice_steps=100, clock=_clock())
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    for r in done:
        assert r.trace[0] == r.steps and r.finished >= r.admitted >= r.arrival
    assert all(e["steps"] <= 100 for e in srv.launch_log)
    # slices are not cut short by the request that ends first: batch slices of
    # 100, 100, 50 (rid 3 stops at 75, rid 1 at 120 inside them)
    assert [e["steps"] for e in srv.launch_log if e["n_batch"]] == [100, 100, 50]
    # the 2D set changed as requests finished: batches of 3, then 2 (rid 3 left), then 1
    assert [len(b) for b in batches] == [3, 2, 1]
    assert _Sim.live == 0


def test_admission_keeps_the_footprint_under_the_cap(monkeypatch):
    _install_fakes(monkeypatch)
    p = _prob((128, 128))
    fp = serve.footprint_bytes(p, "f32")
    reqs = [serve.Request(i, 0.0, _prob((128, 128)), 150) for i in range(5)]
    srv = serve.Server(cap_bytes=2.5 * fp, slice_steps=100, clock=_clock())
    done = srv.run(reqs)
    assert len(done) == 5 and _Sim.peak == 2
    order = [r.rid for r in sorted(done, key=lambda r: r.admitted)]
    assert order == [0, 1, 2, 3, 4]                        # arrival order


def test_admission_keeps_the_active_cells_under_their_cap(monkeypatch):
    """Three 128^2 requests fit the memory cap together but only two fit the
    cell cap: the third waits for the first to leave, then keeps its place
    ahead of a later small one."""
    _install_fakes(monkeypatch)
    reqs = [serve.Request(i, 0.0, _prob((128, 128)), 150 + 50 * i) for i in range(3)]
    reqs.append(serve.Request(3, 0.0, _prob((8, 8)), 50))
    srv = serve.Server(cap_bytes=1e12, slice_steps=100, clock=_clock(), max_cells=2 * 128 * 128 + 64)
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    assert all(e["n_batch"] <= 3 for e in srv.launch_log)
    for e in srv.launch_log:
        live = [r for r in reqs if r.admitted <= e["t"] and (r.finished is None or r.finished >= e["t"])]
        assert sum(r.cells for r in live) <= 2 * 128 * 128 + 64
    order = [r.rid for r in sorted(done, key=lambda r: r.admitted)]
    assert order == [0, 1, 2, 3]
    by = {r.rid: r for r in done}
    assert by[2].admitted >= by[0].finished


def test_a_request_larger_than_the_cap_still_runs_alone(monkeypatch):
    _install_fakes(monkeypatch)
    reqs = [serve.Request(0, 0.0, _prob((256, 256)), 50), serve.Request(1, 0.0, _prob((16, 16)), 50)]
    srv = serve.Server(cap_bytes=1.0, slice_steps=100, clock=_clock())
    done = srv.run(reqs)
    assert [r.rid for r in done] == [0, 1] and _Sim.peak == 1


@pytest.mark.parametrize("maps", ["f32", "bf16", "f16", "idx", "idx16"])
def test_footprint_counts_state_maps_and_strips(maps):
    """State 1 + D + 2DN float arrays; maps 5 + 4N values per cell (float,
    bf16 or FP16) or the index (1 or 2 bytes) plus tables of 21 fields; strips
    4 arrays of N x 2L cells per row of each axis, in the maps' type (float for
    the index forms)."""
    nx, ny, N, L = 200, 100, 3, 10
    p = types.SimpleNamespace(shape=(nx, ny), nrelax=N, pml_transition=L, pml_bound=0,
                              tables={"c": np.zeros(1157)})
    n = nx * ny
    state = (1 + 2 + 4 * N) * 4 * n
    mp = {"f32": (5 + 4 * N) * 4 * n, "bf16": (5 + 4 * N) * 2 * n, "f16": (5 + 4 * N) * 2 * n,
          "idx": n + 21 * 256 * 4, "idx16": 2 * n + 21 * 1160 * 4}[maps]
    es = 2 if maps in ("bf16", "f16") else 4
    strips = 4 * N * es * 2 * L * (ny + nx)
    assert serve.footprint_bytes(p, maps) == state + mp + strips


def test_only_3d_requests_of_the_pipelined_path_join_the_batch():
    """bf16 3D requests with at most 3 mechanisms and no periodic axis join
    the batch (fw2_batch_create takes 3D contexts on that path only); 2D
    requests always do."""
    def req(shape, maps, N=3, bc=("zero",) * 3):
        prob = types.SimpleNamespace(shape=shape, nrelax=N, pml_transition=3, pml_bound=1, bc=bc)
        return serve.Request(0, 0.0, prob, 10, maps=maps)
    assert serve.batchable(req((64, 48), "f32", N=8))
    assert serve.batchable(req((32, 32, 24), "bf16"))
    assert not serve.batchable(req((32, 32, 24), "bf16", N=4))
    assert not serve.batchable(req((32, 32, 24), "bf16", bc=("zero", "periodic", "zero")))
    assert not serve.batchable(req((32, 32, 24), "f32"))
    assert not serve.batchable(req((32, 32, 24), "idx"))


def test_prepare_fills_problems_at_admission_and_drops_them_after(monkeypatch):
    _install_fakes(monkeypatch)
    shapes = [(64, 48), (32, 32, 24), (40, 40)]
    reqs = [serve.Request(i, 0.0, None, 120, shape=s) for i, s in enumerate(shapes)]
    seen = []

    def prepare(r):
        assert r.problem is None
        seen.append(r.rid)
        r.problem = _prob(r.shape)
    srv = serve.Server(cap_bytes=1e12, slice_steps=100, clock=_clock(), prepare=prepare)
    done = srv.run(reqs)
    assert seen == [0, 1, 2]
    assert sorted(r.rid for r in done) == [0, 1, 2]
    assert all(r.problem is None and r.trace[0] == 120 for r in done)
    assert [r.cells for r in reqs] == [64 * 48, 32 * 32 * 24, 40 * 40]
