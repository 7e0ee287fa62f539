"""The field scan that allocates nothing (fw2_field_absmax_noalloc).

It serves callers that cannot allocate device memory (applications that own
every device allocation, or loops that cannot afford cudaMalloc's
synchronisation).  Its result must equal the scan behind fw2_check_field on
the same field, call after call, although every call shares one static
scratch array.  This file is collected last on purpose.
"""
import ctypes

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


def test_noalloc_scan_leaves_device_memory_unchanged(fw2):
    """After a first call (which may load the library's device code), further
    calls take no device memory: the driver's free-memory count is the same
    before and after them."""
    import torch
    x = torch.randn((300, 200), device="cuda")
    out = torch.zeros((2,), device="cuda")
    assert fw2.fw2_field_absmax_noalloc(x, 200, 300, 200, out[:1]) == fw2.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert fw2.fw2_field_absmax_noalloc(x, 200, 300, 200, out[:1]) == fw2.OK
    assert fw2.fw2_field_absmax_noalloc(x, 150, 299, 200, out[1:]) == fw2.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert float(out[0]) == float(x.abs().max())
    assert float(out[1]) == float(x[:299, :150].abs().max())


def test_noalloc_scan_flags_nonfinite_and_rejects_bad_arguments(fw2):
    import torch
    x = torch.zeros((64, 40), device="cuda")
    x[10, 3] = float("nan")
    out = torch.zeros((1,), device="cuda")
    assert fw2.fw2_field_absmax_noalloc(x, 40, 64, 40, out) == fw2.OK
    torch.cuda.synchronize()
    assert np.isinf(out.item())
    # more rows than the static scratch holds: refused by the library itself
    tall = torch.zeros(((1 << 20) + 1, 1), device="cuda")
    assert fw2.fw2_field_absmax_noalloc(tall, 1, (1 << 20) + 1, 1, out) == fw2.EINVAL
    assert "static scratch" in fw2.fw2_last_error(None)
    assert fw2.fw2_field_absmax_noalloc(x, 40, 64, 39, out) == fw2.EINVAL
    # the binding refuses what would reach outside the tensors
    for bad in (lambda: fw2.fw2_field_absmax_noalloc(x.cpu(), 40, 64, 40, out),
                lambda: fw2.fw2_field_absmax_noalloc(x, 40, 65, 40, out),
                lambda: fw2.fw2_field_absmax_noalloc(x.double(), 40, 64, 40, out),
                lambda: fw2.fw2_field_absmax_noalloc(x, 40, 64, 40, out[:0])):
        with pytest.raises(ValueError):
            bad()
    # host memory given straight to the C entry point is refused before any
    # launch (the buffer is large enough for every row the call names)
    host = np.zeros(64 * 40, dtype=np.float32)
    st = fw2.lib().fw2_field_absmax_noalloc(ctypes.c_void_p(host.ctypes.data), 40, 64, 40,
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert st == fw2.EINVAL
    assert "device memory" in fw2.fw2_last_error(None)
