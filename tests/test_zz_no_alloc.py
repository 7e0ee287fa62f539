"""The field scan that allocates nothing (fw2_field_absmax_noalloc).

It serves callers that cannot allocate device memory (applications that own
every device allocation, or loops that cannot afford cudaMalloc's
synchronisation).  Its result must equal the scan behind fw2_check_field on
the same field, call after call, although every call shares one static
scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw2(fw2lib):
    from paper_2106_11476_gb300 import fw2 as m
    return m


def test_noalloc_scan_matches_check_field_on_consecutive_calls(fw2):
    import torch
    prob = synth.line_source_problem(n=160, n_steps=200, relax_key="N2_y1.0_a0.5",
                                     pml_lambda=(1.0, 0.5), n_sensors=8)
    sim = fw2.Simulation(prob)
    ny, nx = prob.grid_shape
    stream = torch.cuda.current_stream().cuda_stream
    for call, (steps, rows) in enumerate(((60, ny), (45, ny - 37))):
        sim.step(steps)
        p = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        fw2.fw2_get_field(sim.ctx, "p", p)
        # reference: the context's own scan (rows limited by zeroing the rest)
        field = p.clone()
        field[rows:] = 0.0
        fw2.fw2_set_field(sim.ctx, "p", field)
        st, ref = fw2.fw2_check_field(sim.ctx, 1e30)
        assert st == fw2.OK and ref > 0
        out = torch.full((1,), -1.0, device="cuda")
        assert fw2.fw2_field_absmax_noalloc(p, nx, rows, nx, out, stream) == fw2.OK, fw2.fw2_last_error(None)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-7 * ref, (call, got, ref)
        assert got == float(p[:rows].abs().max().item())
        fw2.fw2_set_field(sim.ctx, "p", p)
    sim.close()


def test_noalloc_scan_flags_nonfinite_and_rejects_oversize(fw2):
    import torch
    x = torch.zeros((64, 40), device="cuda")
    x[10, 3] = float("nan")
    out = torch.zeros((1,), device="cuda")
    assert fw2.fw2_field_absmax_noalloc(x, 40, 64, 40, out) == fw2.OK
    torch.cuda.synchronize()
    assert np.isinf(out.item())
    assert fw2.fw2_field_absmax_noalloc(x, 40, (1 << 20) + 1, 40, out) == fw2.EINVAL
    assert "static scratch" in fw2.fw2_last_error(None)
    assert fw2.fw2_field_absmax_noalloc(x, 40, 64, 39, out) == fw2.EINVAL
