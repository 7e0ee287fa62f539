"""The C ABI library: loads, exports what include/fw2.h declares, validates
its inputs before touching a device (runs without a GPU)."""
import ctypes as C
import os
import re

import numpy as np

import pytest

from paper_2106_11476_gb300 import fw2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fw2.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fw2_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    syms = declared_symbols()
    for name in ("fw2_create", "fw2_set_medium", "fw2_set_relaxation", "fw2_add_source",
                 "fw2_step", "fw2_record", "fw2_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(fw2lib):
    for name in declared_symbols():
        assert hasattr(fw2lib, name), name
    assert set(declared_symbols()) == set(fw2.EXPORTS), "binding and header disagree"


def test_struct_layout_matches_header(fw2lib):
    # fw2_config_init writes the whole struct; the sentinel after it must survive
    class Guarded(C.Structure):
        _fields_ = [("cfg", fw2.Config), ("guard", C.c_uint64)]
    g = Guarded()
    g.guard = 0xDEADBEEFCAFEF00D
    assert fw2lib.fw2_config_init(C.byref(g.cfg)) == 0
    assert g.guard == 0xDEADBEEFCAFEF00D
    assert g.cfg.ndim == 2 and abs(g.cfg.cfl - 0.4) < 1e-15 and abs(g.cfg.pml_rc - 1e-3) < 1e-18
    assert g.cfg.pml_npow == 2.0 and g.cfg.mem_alignment == 0 and g.cfg.pml_reading == 2


def test_abi_version(fw2lib):
    assert fw2.fw2_abi_version() == 1


@pytest.mark.parametrize("patch,status", [
    ({"ndim": 4}, fw2.EINVAL),
    ({"n": (4, 64, 1)}, fw2.EINVAL),
    ({"n_relax": 9}, fw2.EUNSUPPORTED),
    ({"n_relax": -1}, fw2.EINVAL),
    ({"h": 0.0}, fw2.EINVAL),
    ({"pml_transition": 30, "pml_bound": 10, "n_relax": 2}, fw2.EINVAL),   # 2 * 40 > 64
    ({"pml_transition": 4, "n_relax": 0}, fw2.EINVAL),                     # PML needs N >= 1
    ({"nl_mode": 7}, fw2.EINVAL),
    ({"nl_mode": 4}, fw2.EINVAL),                                          # past LITERAL
    ({"kernel_path": 5}, fw2.EINVAL),
    ({"mem_alignment": 2}, fw2.EINVAL),
    ({"map_precision": 5}, fw2.EINVAL),
    ({"map_precision": 2, "n_relax": 5}, fw2.EUNSUPPORTED),                # index tables: N <= 4
    ({"map_precision": 3, "n_relax": 5}, fw2.EUNSUPPORTED),
    ({"ndim": 3, "n": (64, 64, 64), "map_precision": 2, "n_relax": 6}, fw2.EUNSUPPORTED),
    ({"pml_reading": 1}, fw2.EINVAL),                                      # withdrawn reading
    ({"pml_reading": 4}, fw2.EINVAL),
])
def test_create_rejects_bad_configs(fw2lib, patch, status):
    cfg = fw2.fw2_config_init()
    cfg.n[0], cfg.n[1], cfg.n[2] = 64, 64, 1
    cfg.h = 1e-4
    for k, v in patch.items():
        if k in ("n", "g"):
            for i, x in enumerate(v):
                getattr(cfg, k)[i] = x
        else:
            setattr(cfg, k, v)
    h = C.c_void_p()
    st = fw2lib.fw2_create(C.byref(cfg), C.byref(h))
    assert st == status, fw2.fw2_last_error(None)
    assert h.value is None
    assert len(fw2.fw2_last_error(None)) > 0


def test_create_without_device_fails_cleanly(fw2lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    cfg = fw2.fw2_config_init()
    cfg.n[0], cfg.n[1] = 64, 64
    cfg.h = 1e-4
    h = C.c_void_p()
    assert fw2lib.fw2_create(C.byref(cfg), C.byref(h)) == fw2.ECUDA
    assert "device" in fw2.fw2_last_error(None)


def test_null_context_calls_are_rejected(fw2lib):
    assert fw2lib.fw2_step(None, 1) == fw2.EINVAL
    assert fw2lib.fw2_destroy(None) == 0
    assert fw2.fw2_last_error(None)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("r", [0.0, 0.1, 0.35, 0.4, 0.7])
def test_time_space_taps_match_the_oracle(fw2lib, r, ndim):
    """The library's time-space optimised taps (a host computation) equal the
    oracle's independent derivation."""
    import numpy as np
    from oracle import coefficients as cf
    got = np.array(fw2.fw2_taps_time_space(r, ndim))
    want = np.array(cf.time_space_taps(r, D=ndim))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("r,ndim", [(-0.1, 2), (1.0, 2), (float("nan"), 3), (0.3, 1), (0.3, 4)])
def test_time_space_taps_reject_bad_arguments(fw2lib, r, ndim):
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_taps_time_space(r, ndim)


def test_binding_checks_buffers_against_the_grid_before_calling(monkeypatch):
    """The C ABI takes bare pointers whose extents follow the grid; the
    binding rejects a buffer of the wrong type, a short one, or a
    non-contiguous output before it calls into the library (every case
    below raises before any C call: the handle is not a real context)."""
    import torch
    h = 0x5EED
    monkeypatch.setitem(fw2._GRIDS, h, (64, 48, 1, 2, 4))
    n = 64 * 48
    one = np.ones(n, np.float32)
    with pytest.raises(ValueError):
        fw2.fw2_set_medium(h, one[:-1], one)                      # short c
    with pytest.raises(ValueError):
        fw2.fw2_set_medium(h, one, torch.ones(n, dtype=torch.float64))   # wrong dtype
    with pytest.raises(ValueError):
        fw2.fw2_set_relaxation(h, one, one, one, one, one, one)   # d, alpha are [N][cells]
    with pytest.raises(ValueError):
        fw2.fw2_set_medium_indexed(h, np.zeros(n - 1, np.uint8), 3, *([np.ones(3, np.float32)] * 5),
                                   *([np.ones(12, np.float32)] * 4))
    with pytest.raises(ValueError):
        fw2.fw2_set_medium_indexed(h, np.zeros(n, np.uint8), 3, *([np.ones(3, np.float32)] * 5),
                                   *([np.ones(11, np.float32)] * 4))   # tables of N x n_tissue
    with pytest.raises(ValueError):
        fw2.fw2_get_field(h, "p", np.empty(n - 1, np.float32))
    with pytest.raises(ValueError):
        fw2.fw2_get_field(h, "psi1x", np.empty(n, np.float32))   # N planes
    with pytest.raises(ValueError):
        fw2.fw2_get_field(h, "p", np.empty(n, np.float64))
    with pytest.raises(ValueError):
        fw2.fw2_get_field(h, "p", np.empty((48, 128), np.float32)[:, ::2])   # a copy would take the writes
    with pytest.raises(ValueError):
        fw2.fw2_set_field(h, "p", np.empty(n + 1, np.float32))
    with pytest.raises(ValueError):
        fw2.fw2_get_rows(h, "p", 0, 4, np.empty((3, 64), np.float32))
    with pytest.raises(ValueError):
        fw2.fw2_set_rows(h, "p", 0, 4, np.empty((3, 64), np.float32))
    idx = np.arange(8, dtype=np.int64)
    with pytest.raises(ValueError):
        fw2.fw2_record(h, idx, np.zeros(7, np.int32), 1, torch.empty(100), 10)   # group per point
    with pytest.raises(ValueError):
        fw2.fw2_record(h, idx, None, 8, torch.empty(79), 10)                      # 10 x 8 outputs
    with pytest.raises(ValueError):
        fw2.fw2_record(h, idx, None, 8, torch.empty(80), 10)                      # host tensor
    with pytest.raises(ValueError):
        fw2.fw2_record(h, idx, None, 8, np.empty(80, np.float32), 10)             # host array
    with pytest.raises(ValueError):
        fw2.fw2_add_source(h, "p", idx, np.zeros(9, np.int32), np.zeros((10, 1), np.float32))
    with pytest.raises(ValueError):
        fw2.fw2_add_source(h, "p", idx, None, np.zeros(10, np.float32))           # [n_steps][n_groups]
