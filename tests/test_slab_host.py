"""Host logic of the slab decomposition (paper_2106_11476_gb300/slab.py) on
the CPU: the partition of the rows, the slab problems (media, sources,
sensor groups) and the exchange of extra rows between gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2106_11476_gb300 import slab


@pytest.mark.parametrize("n,parts", [(100, 1), (100, 2), (101, 3), (64, 8)])
def test_layout_covers_the_rows_once(n, parts):
    lays = [slab.layout(n, parts, r) for r in range(parts)]
    assert lays[0].own[0] == 0 and lays[-1].own[1] == n
    for a, b in zip(lays, lays[1:]):
        assert a.own[1] == b.own[0]
        assert a.rows[1] == a.own[1] + slab.GHOST and b.rows[0] == b.own[0] - slab.GHOST
    assert lays[0].rows[0] == 0 and lays[-1].rows[1] == n
    with pytest.raises(ValueError):
        slab.layout(12, 4, 1)                 # slabs of 3 rows cannot feed 4 extra rows


@pytest.mark.parametrize("dims", [2, 3])
def test_slab_problems_partition_the_problem(dims):
    if dims == 2:
        prob = synth.abdominal_problem(n=256, n_steps=10, n_elements=8, pml_lambda=(1.0, 0.5))
        # sensor groups along rows of the array plus point sensors at other depths
        parts = 3
    else:
        prob = synth.skull_problem(n=64, n_steps=10, pml_cells=8, array_elems=4)
        parts = 2
    shape = prob.shape
    inner = int(np.prod(shape[:-1]))
    subs = []
    for r in range(parts):
        lay = slab.layout(shape[-1], parts, r)
        sub, groups = slab.slab_problem(prob, lay)
        assert sub.shape == shape[:-1] + (lay.rows[1] - lay.rows[0],)
        assert sub.dt == prob.dt and sub.pml_cp == float(np.max(prob.c))
        subs.append((lay, sub, groups))
    lo_own = lambda lay, a: a[lay.own[0] - lay.rows[0]:lay.own[1] - lay.rows[0]]
    np.testing.assert_array_equal(np.concatenate([lo_own(l, s.c) for l, s, _ in subs]), prob.c)
    np.testing.assert_array_equal(np.concatenate([lo_own(l, s.d1.transpose(1, 0, *range(2, s.d1.ndim)))
                                                  for l, s, _ in subs]).transpose(1, 0, *range(2, prob.d1.ndim)),
                                  prob.d1)
    # every source entry in exactly one slab, at its global cell
    for k, src in enumerate(prob.sources):
        seen = []
        for lay, sub, _ in subs:
            for s in sub.sources:
                if s.kind == src.kind and s.signal is src.signal:
                    seen += list(zip(s.idx + lay.rows[0] * inner, s.group))
        assert sorted(seen) == sorted(zip(np.asarray(src.idx, np.int64), np.asarray(src.group)))
    # sensor groups: each in one slab, with the same cells
    got = {}
    for lay, sub, groups in subs:
        if sub.sensors is None:
            continue
        for local, g in enumerate(groups):
            cells = np.sort(sub.sensors.idx[sub.sensors.group == local] + lay.rows[0] * inner)
            assert g not in got
            got[g] = cells
    for g in range(prob.sensors.n_groups):
        np.testing.assert_array_equal(got[g], np.sort(prob.sensors.idx[prob.sensors.group == g]))


def test_a_sensor_group_across_slabs_is_refused():
    prob = synth.line_source_problem(n=64, n_steps=5, n_sensors=4, pml_lambda=(0.5, 0.25))
    k = np.array([30, 34]) * 64 + 10                          # one group on rows 30 and 34
    prob.sensors = synth.Sensors(k.astype(np.int64), np.zeros(2, np.int32), 1)
    with pytest.raises(ValueError):
        slab.slab_problem(prob, slab.layout(64, 2, 0))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_rows, cells = 30, 5
        lay = slab.layout(n_rows, world, rank)
        lo, hi = lay.rows
        # a stand-in context: p and v_x rows of the whole grid's values on the
        # own rows, NaN on the extra rows until the exchange fills them
        fields = {}
        for f, base in (("p", 0.0), ("vx", 0.5)):
            arr = np.full((hi - lo, cells), np.nan, np.float32)
            for r in range(lay.own[0], lay.own[1]):
                arr[r - lo] = base + 100.0 * r + np.arange(cells)
            fields[f] = arr
        get = lambda f, r0, n: torch.from_numpy(fields[f][r0:r0 + n].copy())
        def put(f, r0, t):
            fields[f][r0:r0 + t.shape[0]] = t.numpy()
        slab.exchange(lay, ["p", "vx"], get, put, lambda peer, t: dist.isend(t, peer),
                      lambda peer, like: (lambda b: (dist.recv(b, peer), b)[1])(torch.empty_like(like)))
        want = {f: np.stack([base + 100.0 * r + np.arange(cells) for r in range(lo, hi)]).astype(np.float32)
                for f, base in (("p", 0.0), ("vx", 0.5))}
        q.put((rank, all(np.array_equal(fields[f], want[f]) for f in fields)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_fill_each_others_extra_rows(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(r, True) for r in range(world)]
