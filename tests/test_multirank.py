"""The multi-rank host path of bench.py on CPU: two gloo ranks (one process
each, as torchrun launches them) take the slowest rank's time for the
whole-job rate, and simulate different transmit events (weak scaling: no
data-path collective, only the timing reduction)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
        rate = bench.job_rate(world, 1_000_000, 100, slowest)
        prob = synth.abdominal_problem(n=256, n_steps=5, seed=1 + rank, n_elements=16)
        q.put((rank, slowest, rate, float(np.asarray(prob.c, np.float64).sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_differ_in_transmits():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, c0), (r1, t1, v1, c1) = out
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 15.0                      # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 1e6 * 100 / 15.0 / 1e9)
    assert c0 != c1                              # each rank its own seeded medium


def test_job_rate_without_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 16_777_216, 1000, 0.7) == pytest.approx(16_777_216 * 1000 / 0.7 / 1e9)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """`bench.py --impl reference` launched as torchrun launches it (two
    ranks, 127.0.0.1): rank 0 times the oracle and prints the single JSON
    line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["steps"] == 3
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]
