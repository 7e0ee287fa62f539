"""ctypes binding of libfw2.so (include/fw2.h): argument marshalling only.

Every function named ``fw2_*`` here forwards to the C entry point of the same
name; all compute runs in the library's CUDA kernels.  Arrays are numpy
(host) or torch CUDA tensors (device); torch provides device memory and the
stream.  Loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfw2.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, EUNSTABLE, ETIMEOUT, EUNSUPPORTED = range(8)
STATUS_NAMES = ["FW2_OK", "FW2_EINVAL", "FW2_ENOMEM", "FW2_ECUDA", "FW2_ESTATE", "FW2_EUNSTABLE",
                "FW2_ETIMEOUT", "FW2_EUNSUPPORTED"]
MEM_HOST, MEM_DEVICE = 0, 1
BC = {"zero": 0, "periodic": 1}
NL = {"off": 0, "pressure": 1, "westervelt": 2, "literal": 3}
MAP = {"f32": 0, "bf16": 1, "idx": 2, "idx16": 3, "f16": 4}
PML_READING = {"A": 0, "C": 2, "K": 3}
MEM_ALIGN = {"centred": 0, "endpoint": 1}
SRC_KIND = {"p": 0, "vx": 1, "vy": 2, "vz": 3}
FIELD = {"p": 0, "vx": 1, "vy": 2, "vz": 3, "psi1x": 4, "psi1y": 5, "psi1z": 6,
         "psi2x": 7, "psi2y": 8, "psi2z": 9}


class Fw2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("n_relax", C.c_int32), ("n", C.c_int64 * 3), ("h", C.c_double),
                ("dt", C.c_double), ("cfl", C.c_double), ("g", C.c_double * 5),
                ("pml_transition", C.c_int32), ("pml_bound", C.c_int32), ("pml_reading", C.c_int32),
                ("map_precision", C.c_int32), ("pml_rc", C.c_double), ("pml_npow", C.c_double),
                ("pml_cp", C.c_double), ("nl_mode", C.c_int32), ("mem_alignment", C.c_int32),
                ("bc", C.c_int32 * 3), ("kernel_path", C.c_int32), ("stream", C.c_void_p)]


FIT_MAX_RELAX = 4


class FitRequest(C.Structure):
    _fields_ = [("alpha0", C.c_double), ("y", C.c_double), ("n_relax", C.c_int32), ("c0", C.c_double),
                ("f_ref", C.c_double), ("f_lo", C.c_double), ("f_hi", C.c_double), ("n_freq", C.c_int32),
                ("w_alpha", C.c_double), ("kappa_bounds", C.c_double * 2), ("log_d_bounds", C.c_double * 2),
                ("log_alpha_bounds", C.c_double * 2), ("grid_points", C.c_int32), ("refinements", C.c_int32),
                ("shrink", C.c_double), ("polish_iterations", C.c_int32), ("threads", C.c_int32)]


class FitResult(C.Structure):
    _fields_ = [("kappa1", C.c_double), ("kappa2", C.c_double), ("d1", C.c_double * FIT_MAX_RELAX),
                ("alpha1", C.c_double * FIT_MAX_RELAX), ("d2", C.c_double * FIT_MAX_RELAX),
                ("alpha2", C.c_double * FIT_MAX_RELAX), ("J", C.c_double), ("J_grid", C.c_double),
                ("f_ref", C.c_double), ("max_att_rel_err", C.c_double), ("max_phase_rel_err", C.c_double),
                ("evaluations", C.c_int64)]


class RelaxDesc(C.Structure):
    _fields_ = [("kappa1", C.c_void_p), ("kappa2", C.c_void_p), ("d1", C.c_void_p), ("alpha1", C.c_void_p),
                ("d2", C.c_void_p), ("alpha2", C.c_void_p), ("mem_space", C.c_int32)]


EXPORTS = {
    "fw2_config_init": (C.c_int, [C.POINTER(Config)]),
    "fw2_create": (C.c_int, [C.POINTER(Config), C.POINTER(C.c_void_p)]),
    "fw2_set_medium": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fw2_set_relaxation": (C.c_int, [C.c_void_p, C.POINTER(RelaxDesc)]),
    "fw2_set_medium_indexed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(RelaxDesc), C.c_int32]),
    "fw2_add_source": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int64, C.c_int64, C.c_int32]),
    "fw2_record": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                             C.c_int64, C.c_int32]),
    "fw2_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "fw2_destroy": (C.c_int, [C.c_void_p]),
    "fw2_set_watch": (C.c_int, [C.c_void_p, C.c_int64, C.c_float]),
    "fw2_set_subdomain": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "fw2_step_part": (C.c_int, [C.c_void_p, C.c_int32]),
    "fw2_get_rows": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_void_p, C.c_int32]),
    "fw2_set_rows": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_void_p, C.c_int32]),
    "fw2_get_dt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "fw2_get_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "fw2_set_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "fw2_get_field": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "fw2_set_field": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "fw2_reset": (C.c_int, [C.c_void_p]),
    "fw2_synchronize": (C.c_int, [C.c_void_p]),
    "fw2_check_field": (C.c_int, [C.c_void_p, C.c_float, C.POINTER(C.c_float)]),
    "fw2_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "fw2_release_memory": (C.c_int, []),
    "fw2_kernel_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "fw2_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "fw2_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "fw2_field_absmax_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                           C.c_void_p]),
    "fw2_selftest_bounded_wait": (C.c_int, [C.c_int64, C.POINTER(C.c_int32)]),
    "fw2_kernel_path": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "fw2_pipe_layout": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "fw2_taps_time_space": (C.c_int, [C.c_double, C.c_int32, C.POINTER(C.c_double)]),
    "fw2_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "fw2_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "fw2_batch_synchronize": (C.c_int, [C.c_void_p]),
    "fw2_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "fw2_batch_edge_weight": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "fw2_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "fw2_batch_set_watch": (C.c_int, [C.c_void_p, C.c_int64, C.c_float]),
    "fw2_batch_set_budget": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fw2_batch_active": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "fw2_batch_destroy": (C.c_int, [C.c_void_p]),
    "fw2_last_error": (C.c_char_p, [C.c_void_p]),
    "fw2_abi_version": (C.c_int32, []),
    "fw2_fit_request_init": (C.c_int, [C.POINTER(FitRequest)]),
    "fw2_fit_relaxation": (C.c_int, [C.POINTER(FitRequest), C.POINTER(FitResult)]),
    "fw2_relaxation_curves": (C.c_int, [C.POINTER(FitResult), C.c_int32, C.c_double, C.c_void_p, C.c_int64,
                                        C.c_void_p, C.c_void_p]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded libfw2.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfw2.so not found at {LIB_PATH}: build it with "
                               "paper_2106_11476_gb300._build.build() (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != OK:
        raise Fw2Error(status, fw2_last_error(ctx))


def _ptr(a):
    """(pointer, mem_space, keepalive) of a numpy array or torch tensor (float32/int64/int32)."""
    if a is None:
        return None, MEM_HOST, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, MEM_HOST, a
    import torch
    if isinstance(a, torch.Tensor):
        t = a.contiguous()
        return t.data_ptr(), (MEM_DEVICE if t.is_cuda else MEM_HOST), t
    raise TypeError(type(a))


# Grid of every context created through this binding, by handle: (nx, ny,
# nz, ndim, n_relax).  The C ABI takes bare pointers whose extents follow the
# grid, so the binding checks each buffer against it before the call (a short
# buffer would let the library read or write past it).
_GRIDS = {}


def _grid_cells(ctx):
    """(cells of the grid, cells of one row along the slowest axis, n_relax),
    or None for a context this binding did not create."""
    g = _GRIDS.get(ctx)
    if g is None:
        return None
    nx, ny, nz, nd, N = g
    return nx * ny * (nz if nd == 3 else 1), nx * (ny if nd == 3 else 1), N


def _want(a, dtype, count, name, out=False, exact=False):
    """Check one buffer of a call.  Host inputs (numpy) are converted to
    `dtype`; tensors must already hold it.  Output buffers must be contiguous
    (a copy would take the library's writes) and, numpy ones, writable.
    `count` (None: unknown) is the number of elements the library reads or
    writes through the buffer: it must hold at least that many (exactly
    that many with `exact`)."""
    if a is None:
        return None
    dt = np.dtype(dtype)
    if isinstance(a, np.ndarray):
        if out:
            if a.dtype != dt or not a.flags.c_contiguous or not a.flags.writeable:
                raise ValueError(f"{name} must be a writable C-contiguous {dt.name} array")
        else:
            a = np.ascontiguousarray(a, dt)
        n = a.size
    else:
        import torch
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"{name}: a numpy array or a torch tensor, not {type(a).__name__}")
        if a.dtype != getattr(torch, dt.name):
            raise ValueError(f"{name} must hold {dt.name}, not {a.dtype}")
        if out and not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        n = a.numel()
    if count is not None and (n != count if exact else n < count):
        raise ValueError(f"{name} holds {n} elements; the call {'writes' if out else 'reads'} {count}")
    return a


def _same_space(*arrays):
    spaces = {_ptr(a)[1] for a in arrays if a is not None}
    if len(spaces) > 1:
        raise ValueError("all arrays of one call must live in the same memory space")
    return spaces.pop() if spaces else MEM_HOST


# ---------------------------------------------------------------- C names ---

def fw2_config_init() -> Config:
    """Defaults of fw2_config (fw2_config_init in include/fw2.h)."""
    cfg = Config()
    _check(lib().fw2_config_init(C.byref(cfg)))
    return cfg


def fw2_create(cfg: Config) -> int:
    """Create a context for one grid (fw2_create); returns the handle."""
    h = C.c_void_p()
    _check(lib().fw2_create(C.byref(cfg), C.byref(h)))
    _GRIDS[h.value] = (int(cfg.n[0]), int(cfg.n[1]), int(cfg.n[2]), int(cfg.ndim), int(cfg.n_relax))
    return h.value


def fw2_set_medium(ctx, c, rho, beta=None):
    """c, rho and beta of every cell, host or device arrays (fw2_set_medium)."""
    g = _grid_cells(ctx)
    n = g[0] if g else None
    c, rho, beta = (_want(a, np.float32, n, nm, exact=True) for a, nm in ((c, "c"), (rho, "rho"), (beta, "beta")))
    space = _same_space(c, rho, beta)
    pc, _, kc = _ptr(c)
    pr, _, kr = _ptr(rho)
    pb, _, kb = _ptr(beta)
    _check(lib().fw2_set_medium(ctx, pc, pr, pb, space), ctx)


def fw2_set_relaxation(ctx, kappa1, kappa2, d1, alpha1, d2, alpha2):
    """Interior relaxation parameters of every cell (fw2_set_relaxation)."""
    g = _grid_cells(ctx)
    counts = (g[0], g[0]) + (g[2] * g[0],) * 4 if g else (None,) * 6
    names = ("kappa1", "kappa2", "d1", "alpha1", "d2", "alpha2")
    arrs = [_want(x, np.float32, k, nm, exact=True)
            for x, k, nm in zip((kappa1, kappa2, d1, alpha1, d2, alpha2), counts, names)]
    space = _same_space(*arrs)
    ptrs = [_ptr(a) for a in arrs]
    desc = RelaxDesc(*[p[0] for p in ptrs], space)
    _check(lib().fw2_set_relaxation(ctx, C.byref(desc)), ctx)


def fw2_set_medium_indexed(ctx, tissue, n_tissue: int, c, rho, beta, kappa1, kappa2, d1, alpha1, d2, alpha2,
                           wide: bool = False):
    """Tissue-index medium: uint8 (wide: uint16) index per cell, per-tissue
    tables (fw2_set_medium_indexed)."""
    size = 2 if wide else 1
    if isinstance(tissue, np.ndarray):
        if wide and tissue.dtype == np.int16:
            tissue = tissue.view(np.uint16)
        if tissue.size and (tissue.min() < 0 or tissue.max() >= (1 << (8 * size))):
            raise ValueError(f"tissue index outside the range of {8 * size} bits")
        tissue = np.asarray(tissue, np.uint16 if wide else np.uint8)
    elif tissue.element_size() != size:
        raise ValueError(f"the tissue tensor must hold {size}-byte indices")
    g = _grid_cells(ctx)
    if g is not None:
        n_idx = tissue.size if isinstance(tissue, np.ndarray) else tissue.numel()
        if n_idx != g[0]:
            raise ValueError(f"tissue holds {n_idx} indices; the grid has {g[0]} cells")
    nt = int(n_tissue)
    counts = (nt,) * 5 + ((g[2] * nt,) * 4 if g else (None,) * 4)
    names = ("c", "rho", "beta", "kappa1", "kappa2", "d1", "alpha1", "d2", "alpha2")
    tabs = [_want(x, np.float32, k, nm)
            for x, k, nm in zip((c, rho, beta, kappa1, kappa2, d1, alpha1, d2, alpha2), counts, names)]
    space = _same_space(tissue, *tabs)
    pt, _, kt = _ptr(tissue)
    ptrs = [_ptr(a) for a in tabs]
    desc = RelaxDesc(*[p[0] for p in ptrs[3:]], space)
    _check(lib().fw2_set_medium_indexed(ctx, pt, int(n_tissue), ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                        C.byref(desc), space), ctx)


def fw2_add_source(ctx, kind: str, idx, group, signal):
    """Add an additive source of kind FW2_SRC_* (fw2_add_source)."""
    idx = _want(idx, np.int64, None, "idx")
    n = int(idx.shape[0])
    group = _want(group, np.int32, n, "group", exact=True)
    signal = _want(signal, np.float32, None, "signal")
    if signal.ndim != 2:
        raise ValueError("signal is [n_steps][n_groups]")
    space = _same_space(idx, group, signal)
    pi, _, ki = _ptr(idx)
    pg, _, kg = _ptr(group)
    ps, _, ks = _ptr(signal)
    n_steps, n_groups = signal.shape
    _check(lib().fw2_add_source(ctx, SRC_KIND[kind], int(idx.shape[0]), pi, pg, ps, int(n_groups),
                                int(n_steps), space), ctx)


def fw2_record(ctx, idx, group, n_groups: int, out, n_steps: int):
    """Record p after every step into a caller-owned device buffer (fw2_record).

    `out` is a contiguous float32 CUDA tensor of at least n_steps x n_groups
    elements (n_groups = the number of sensor points without `group`)."""
    idx = _want(idx, np.int64, None, "idx")
    n = int(idx.shape[0])
    group = _want(group, np.int32, n, "group", exact=True)
    if out is not None:
        rows = max(int(n_steps), 0) * (int(n_groups) if group is not None else n)
        _want(out, np.float32, rows if n else None, "out", out=True)
        if isinstance(out, np.ndarray) or not out.is_cuda:
            raise ValueError("out must be a CUDA tensor: the recording kernel writes it")
    space = _same_space(idx, group)
    pi, _, ki = _ptr(idx)
    pg, _, kg = _ptr(group)
    _check(lib().fw2_record(ctx, int(idx.shape[0]), pi, pg, int(n_groups),
                            C.c_void_p(out.data_ptr() if out is not None else 0), int(n_steps), space), ctx)


def fw2_step(ctx, n_steps: int):
    """Advance n_steps time steps, asynchronously on the context stream (fw2_step)."""
    _check(lib().fw2_step(ctx, int(n_steps)), ctx)


def fw2_destroy(ctx):
    """Release the context (fw2_destroy)."""
    if ctx:
        _GRIDS.pop(ctx, None)
        lib().fw2_destroy(ctx)


def fw2_get_dt(ctx) -> float:
    """The time step in use; builds the coefficient maps if needed (fw2_get_dt)."""
    v = C.c_double()
    _check(lib().fw2_get_dt(ctx, C.byref(v)), ctx)
    return v.value


def fw2_set_watch(ctx, every: int, bound: float):
    """Scan p every `every` steps inside fw2_step and stop with EUNSTABLE
    beyond `bound` (fw2_set_watch; every = 0 switches it off)."""
    _check(lib().fw2_set_watch(ctx, int(every), float(bound)), ctx)


def fw2_set_subdomain(ctx, global_shape, offset):
    """Declare the context's grid as a box of a larger grid (fw2_set_subdomain)."""
    g = (C.c_int64 * 3)(*(list(global_shape) + [1] * (3 - len(global_shape))))
    o = (C.c_int64 * 3)(*(list(offset) + [0] * (3 - len(offset))))
    _check(lib().fw2_set_subdomain(ctx, g, o), ctx)


def fw2_step_part(ctx, part: int):
    """Velocity (0) or pressure (1) part of a time step (fw2_step_part)."""
    _check(lib().fw2_step_part(ctx, int(part)), ctx)


def fw2_get_rows(ctx, field: str, row0: int, n_rows: int, out):
    """Rows along the slowest axis of p or v_q into `out` (fw2_get_rows)."""
    g = _grid_cells(ctx)
    _want(out, np.float32, max(int(n_rows), 0) * g[1] if g else None, "out", out=True)
    p, space, keep = _ptr(out)
    _check(lib().fw2_get_rows(ctx, FIELD[field], int(row0), int(n_rows), p, space), ctx)
    return out


def fw2_set_rows(ctx, field: str, row0: int, n_rows: int, arr):
    """Rows along the slowest axis of p or v_q from `arr` (fw2_set_rows)."""
    g = _grid_cells(ctx)
    arr = _want(arr, np.float32, max(int(n_rows), 0) * g[1] if g else None, "arr")
    p, space, keep = _ptr(arr)
    _check(lib().fw2_set_rows(ctx, FIELD[field], int(row0), int(n_rows), p, space), ctx)


def fw2_get_step(ctx) -> int:
    """Index of the next time step (fw2_get_step)."""
    v = C.c_int64()
    _check(lib().fw2_get_step(ctx, C.byref(v)), ctx)
    return v.value


def fw2_set_step(ctx, step: int):
    """Set the index of the next time step, for restore (fw2_set_step)."""
    _check(lib().fw2_set_step(ctx, int(step)), ctx)


def _field_cells(ctx, field: str):
    """Elements of a state array (N per cell for the memory variables)."""
    g = _grid_cells(ctx)
    if g is None:
        return None
    return g[0] * (g[2] if field.startswith("psi") else 1)


def fw2_get_field(ctx, field: str, out):
    """Copy a state array out (fw2_get_field)."""
    _want(out, np.float32, _field_cells(ctx, field), "out", out=True)
    p, space, keep = _ptr(out)
    _check(lib().fw2_get_field(ctx, FIELD[field], p, space), ctx)
    return out


def fw2_set_field(ctx, field: str, arr):
    """Copy a state array in (fw2_set_field)."""
    arr = _want(arr, np.float32, _field_cells(ctx, field), "arr", exact=True)
    p, space, keep = _ptr(arr)
    _check(lib().fw2_set_field(ctx, FIELD[field], p, space), ctx)


def fw2_reset(ctx):
    """Zero the state and the step counter (fw2_reset)."""
    _check(lib().fw2_reset(ctx), ctx)


def fw2_synchronize(ctx):
    """Wait for the context stream; raises on a device-side wait that gave up (fw2_synchronize)."""
    _check(lib().fw2_synchronize(ctx), ctx)


def fw2_check_field(ctx, bound: float):
    """Scan p for non-finite values or a bound (fw2_check_field)."""
    m = C.c_float()
    st = lib().fw2_check_field(ctx, C.c_float(bound), C.byref(m))
    return st, m.value


def fw2_release_memory():
    """Give the free memory of the library's device pool back (fw2_release_memory)."""
    _check(lib().fw2_release_memory())


def fw2_device_bytes(ctx) -> int:
    """Device bytes the context holds (fw2_device_bytes)."""
    v = C.c_int64()
    _check(lib().fw2_device_bytes(ctx, C.byref(v)), ctx)
    return v.value


def fw2_kernel_launches(ctx) -> int:
    """Kernels the context has launched (fw2_kernel_launches)."""
    v = C.c_int64()
    _check(lib().fw2_kernel_launches(ctx, C.byref(v)), ctx)
    return v.value


def fw2_profile(ctx, enable: bool):
    """Switch per-kernel event timing on or off (fw2_profile)."""
    _check(lib().fw2_profile(ctx, 1 if enable else 0), ctx)


def fw2_profile_read(ctx):
    """(vel_ms, vel_launches, prs_ms, prs_launches) since profiling was enabled."""
    tv, nv, tp, np_ = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
    _check(lib().fw2_profile_read(ctx, C.byref(tv), C.byref(nv), C.byref(tp), C.byref(np_)), ctx)
    return tv.value, nv.value, tp.value, np_.value


def fw2_taps_time_space(r: float, ndim: int = 2) -> tuple:
    """(g_1..g_4, g_11) of the time-space optimised operator of an ndim-D grid
    at Courant number r."""
    g = (C.c_double * 5)()
    _check(lib().fw2_taps_time_space(float(r), int(ndim), g))
    return tuple(g)


def fw2_kernel_path(ctx) -> str:
    """'tile' or 'pipe' once the context has stepped ('auto' before)."""
    v = C.c_int32(0)
    _check(lib().fw2_kernel_path(ctx, C.byref(v)), ctx)
    return {0: "auto", 1: "tile", 2: "pipe"}[v.value]


def fw2_pipe_layout(ctx) -> tuple:
    """(velocity, pressure) layout of the 3D pipelined half steps:
    'staged', 'registers' or None before the choice (fw2_pipe_layout)."""
    v, p = C.c_int32(0), C.c_int32(0)
    _check(lib().fw2_pipe_layout(ctx, C.byref(v), C.byref(p)), ctx)
    names = {0: None, 1: "staged", 2: "registers"}
    return names[v.value], names[p.value]


def fw2_selftest_bounded_wait(limit_ns: int) -> bool:
    """True when a wait on a barrier nobody arrives on gave up after limit_ns."""
    t = C.c_int32(-1)
    _check(lib().fw2_selftest_bounded_wait(int(limit_ns), C.byref(t)))
    return bool(t.value)


def fw2_field_absmax_noalloc(field, row_len: int, n_rows: int, row_pitch: int, out, stream=None) -> int:
    """max |field| over n_rows rows into the one-element device tensor `out`,
    without allocating (fw2_field_absmax_noalloc; returns the status).

    `field` and `out` must be float32 CUDA tensors of one device, `field`
    contiguous and holding every row that the call reads.  The call is
    enqueued on `stream` (a cudaStream_t handle), by default on torch's
    current stream of the field's device, so that it follows the work that
    produced the field.  Arguments that would make the kernel reach outside
    the tensors raise ValueError before any call."""
    import torch
    for name, t in (("field", field), ("out", out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
            raise ValueError(f"{name} must be a float32 CUDA tensor")
    if out.device != field.device:
        raise ValueError("field and out must be on the same device")
    if out.numel() < 1:
        raise ValueError("out needs one element")
    if not field.is_contiguous():
        raise ValueError("field must be contiguous")
    row_len, n_rows, row_pitch = int(row_len), int(n_rows), int(row_pitch)
    if row_len >= 1 and n_rows >= 1 and (n_rows - 1) * row_pitch + row_len > field.numel():
        raise ValueError("rows reach past the field's storage")
    if stream is None:
        stream = torch.cuda.current_stream(field.device).cuda_stream
    return lib().fw2_field_absmax_noalloc(C.c_void_p(field.data_ptr()), row_len, n_rows, row_pitch,
                                          C.c_void_p(out.data_ptr()), C.c_void_p(stream if stream else 0))


def fw2_fit_relaxation(alpha0: float, y: float, n_relax: int, **options) -> dict:
    """Relaxation parameters for a power-law tissue (fw2_fit_relaxation, Sec.
    4.1).  Keyword options are fields of fw2_fit_request (c0, f_ref, f_lo,
    f_hi, n_freq, w_alpha, grid_points, refinements, shrink,
    polish_iterations, threads, and the bounds as 2-tuples).  Returns the
    parameter set in the layout of a relaxation description (kappa1,
    kappa2, d1, alpha1, d2, alpha2) with the cost and the errors."""
    req = FitRequest()
    _check(lib().fw2_fit_request_init(C.byref(req)))
    req.alpha0, req.y, req.n_relax = float(alpha0), float(y), int(n_relax)
    for k, v in options.items():
        if k.endswith("_bounds"):
            getattr(req, k)[0], getattr(req, k)[1] = float(v[0]), float(v[1])
        else:
            setattr(req, k, v)
    res = FitResult()
    _check(lib().fw2_fit_relaxation(C.byref(req), C.byref(res)))
    N = int(n_relax)
    return {"kappa1": res.kappa1, "kappa2": res.kappa2, "d1": list(res.d1[:N]), "alpha1": list(res.alpha1[:N]),
            "d2": list(res.d2[:N]), "alpha2": list(res.alpha2[:N]), "J": res.J, "J_grid": res.J_grid,
            "f_ref": res.f_ref, "max_att_rel_err_2_20MHz": res.max_att_rel_err,
            "max_phase_rel_err": res.max_phase_rel_err, "evaluations": res.evaluations}


def fw2_relaxation_curves(params: dict, c0: float, freqs) -> tuple:
    """(attenuation dB/cm, phase velocity m/s) of a parameter set at freqs [Hz]
    (fw2_relaxation_curves)."""
    N = len(params["d1"])
    res = FitResult()
    res.kappa1, res.kappa2 = float(params["kappa1"]), float(params["kappa2"])
    for n in range(N):
        res.d1[n], res.alpha1[n] = float(params["d1"][n]), float(params["alpha1"][n])
        res.d2[n], res.alpha2[n] = float(params["d2"][n]), float(params["alpha2"][n])
    f = np.ascontiguousarray(freqs, np.float64)
    att, c = np.empty_like(f), np.empty_like(f)
    _check(lib().fw2_relaxation_curves(C.byref(res), N, float(c0), f.ctypes.data, f.size, att.ctypes.data,
                                       c.ctypes.data))
    return att, c


def _bcheck(status: int, batch):
    if status != OK:
        r = lib().fw2_batch_last_error(batch)
        raise Fw2Error(status, r.decode() if r else "")


# contexts per live batch handle (the budget array must have one entry each)
_batch_sizes = {}


def fw2_batch_create(ctxs) -> int:
    """One batch over several contexts (fw2_batch_create); returns the handle."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    h = C.c_void_p()
    st = lib().fw2_batch_create(arr, len(ctxs), C.byref(h))
    if st != OK:
        raise Fw2Error(st, "fw2_batch_create failed")
    _batch_sizes[h.value] = len(ctxs)
    return h.value


def fw2_batch_step(batch, n_steps: int):
    """Advance every context of the batch n_steps (fw2_batch_step)."""
    _bcheck(lib().fw2_batch_step(batch, int(n_steps)), batch)


def fw2_batch_synchronize(batch):
    """Wait for the batch (fw2_batch_synchronize)."""
    _bcheck(lib().fw2_batch_synchronize(batch), batch)


def fw2_batch_info(batch):
    """(grid, order, launches) chosen by the batch autotuner (fw2_batch_info)."""
    g, o, n = C.c_int32(), C.c_int32(), C.c_int64()
    _bcheck(lib().fw2_batch_info(batch, C.byref(g), C.byref(o), C.byref(n)), batch)
    return g.value, o.value, n.value


def fw2_batch_set_watch(batch, every: int, bound: float):
    """Scan every context's p every `every` batch steps (fw2_batch_set_watch)."""
    _bcheck(lib().fw2_batch_set_watch(batch, int(every), float(bound)), batch)


def fw2_batch_set_budget(batch, last_steps):
    """Step count at which each context leaves the batch (fw2_batch_set_budget;
    None clears, a negative entry means no budget)."""
    if last_steps is None:
        _bcheck(lib().fw2_batch_set_budget(batch, None), batch)
        return
    arr = np.ascontiguousarray(last_steps, np.int64)
    n = _batch_sizes.get(batch)
    if arr.ndim != 1 or (n is not None and arr.size != n):
        raise ValueError(f"one budget per context of the batch: got {arr.size}, the batch has {n}")
    _bcheck(lib().fw2_batch_set_budget(batch, arr.ctypes.data), batch)


def fw2_batch_active(batch) -> int:
    """Contexts still short of their budget (fw2_batch_active)."""
    n = C.c_int32()
    _bcheck(lib().fw2_batch_active(batch, C.byref(n)), batch)
    return n.value


def fw2_batch_edge_weight(batch) -> float:
    """Tuned edge-unit cost of the pipelined groups' runs, 0 before tuning
    (fw2_batch_edge_weight)."""
    w = C.c_double()
    _bcheck(lib().fw2_batch_edge_weight(batch, C.byref(w)), batch)
    return w.value


def fw2_batch_destroy(batch):
    """Release the batch (fw2_batch_destroy); the contexts remain."""
    if batch:
        _batch_sizes.pop(batch, None)
        lib().fw2_batch_destroy(batch)


def fw2_last_error(ctx=None) -> str:
    """Text of the last error of a context (or of the library with None)."""
    r = lib().fw2_last_error(ctx)
    return r.decode() if r else ""


def fw2_abi_version() -> int:
    """Version of the C ABI."""
    return lib().fw2_abi_version()


# ------------------------------------------------------------ convenience ---

KERNEL_PATH = {"auto": 0, "tile": 1, "pipe": 2, "pipe-staged": 3, "pipe-registers": 4}


def config_for(prob, stream: Optional[int] = None, map_precision: str = "f32", kernel_path: str = "auto") -> Config:
    """A Config for a problem description (any object with the attributes of
    synth.Problem: shape, h, dt, nrelax, pml_*, nl_mode, memory_alignment, bc, taps)."""
    cfg = fw2_config_init()
    nd = len(prob.shape)
    cfg.ndim = nd
    cfg.n_relax = int(prob.nrelax)
    full = list(prob.shape) + [1] * (3 - nd)
    for q in range(3):
        cfg.n[q] = int(full[q])
        cfg.bc[q] = BC[prob.bc[q]] if q < nd else 0
    cfg.h = float(prob.h)
    cfg.dt = float(prob.dt) if prob.dt else 0.0
    if prob.taps is not None:
        for i in range(5):
            cfg.g[i] = float(prob.taps[i])
    cfg.pml_transition = int(prob.pml_transition)
    cfg.pml_bound = int(prob.pml_bound)
    cfg.pml_reading = PML_READING[prob.pml_reading]
    cfg.pml_rc = float(prob.pml_rc)
    cfg.pml_npow = float(prob.pml_npow)
    cfg.pml_cp = float(prob.pml_cp)
    cfg.nl_mode = NL[prob.nl_mode]
    cfg.mem_alignment = MEM_ALIGN[prob.memory_alignment]
    cfg.map_precision = MAP[map_precision]
    cfg.kernel_path = KERNEL_PATH[kernel_path]
    cfg.stream = stream
    return cfg


class Simulation:
    """One fw2 context built from a problem description.

    Traces land in a torch CUDA tensor ``self.trace`` of [n_steps, n_groups].
    """

    def __init__(self, prob, map_precision: str = "f32", device_inputs: bool = False, stream=None,
                 kernel_path: str = "auto", subdomain=None):
        import torch
        self.prob = prob
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.cfg = config_for(prob, stream=stream.cuda_stream, map_precision=map_precision,
                              kernel_path=kernel_path)
        self.ctx = fw2_create(self.cfg)
        try:
            if subdomain is not None:          # (shape of the whole grid, offset of this one)
                fw2_set_subdomain(self.ctx, subdomain[0], subdomain[1])
            conv = (lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()) \
                if device_inputs else (lambda a: a)
            if map_precision in ("idx", "idx16"):
                t = prob.tables
                wide = map_precision == "idx16"
                if isinstance(prob.tissue, np.ndarray):
                    tissue = prob.tissue
                    if tissue.size and tissue.max() >= (65536 if wide else 256):
                        raise ValueError(f"tissue index beyond the {map_precision} form")
                    tissue = tissue.astype(np.uint16) if wide else tissue.astype(np.uint8)
                    # uint16 indices travel to the device as the same bits in int16
                    targ = conv(tissue.view(np.int16)) if (wide and device_inputs) else conv(tissue)
                else:                          # a tensor of 1- or 2-byte indices, passed as it is
                    targ = prob.tissue
                fw2_set_medium_indexed(self.ctx, targ, len(t["c"]), conv(t["c"]), conv(t["rho"]),
                                       conv(t["beta"]) if prob.nl_mode != "off" else None,
                                       conv(t["kappa1"]), conv(t["kappa2"]), conv(t["d1"]), conv(t["alpha1"]),
                                       conv(t["d2"]), conv(t["alpha2"]), wide=wide)
            else:
                fw2_set_medium(self.ctx, conv(prob.c), conv(prob.rho),
                               conv(prob.beta) if prob.nl_mode != "off" else None)
                if prob.nrelax:
                    fw2_set_relaxation(self.ctx, conv(prob.kappa1), conv(prob.kappa2), conv(prob.d1),
                                       conv(prob.alpha1), conv(prob.d2), conv(prob.alpha2))
            for s in prob.sources:
                fw2_add_source(self.ctx, s.kind, conv(s.idx), conv(s.group), conv(s.signal))
            self.trace = None
            if prob.sensors is not None and prob.n_steps > 0:
                sn = prob.sensors
                self.trace = torch.zeros((prob.n_steps, sn.n_groups), dtype=torch.float32, device="cuda")
                fw2_record(self.ctx, conv(sn.idx), conv(sn.group), sn.n_groups, self.trace, prob.n_steps)
            self.dt = fw2_get_dt(self.ctx)
        except Exception:
            fw2_destroy(self.ctx)
            self.ctx = None
            raise

    def step(self, n: int):
        fw2_step(self.ctx, n)
        return self

    def synchronize(self):
        fw2_synchronize(self.ctx)

    def field(self, name: str) -> np.ndarray:
        g = tuple(reversed(self.prob.shape))
        if name.startswith("psi"):
            out = np.empty((self.prob.nrelax,) + g, np.float32)
        else:
            out = np.empty(g, np.float32)
        return fw2_get_field(self.ctx, name, out)

    def field_window(self, name: str, window) -> np.ndarray:
        """A state array cut to `window` ((x0, x1), (y0, y1)[, (z0, z1)]):
        copied out into device memory, cut there, and only the window copied
        to the host (numpy order, memory variables [N, ...])."""
        torch = self.torch
        g = tuple(reversed(self.prob.shape))
        shape = ((self.prob.nrelax,) + g) if name.startswith("psi") else g
        buf = torch.empty(shape, dtype=torch.float32, device="cuda")
        fw2_get_field(self.ctx, name, buf)
        sl = tuple(slice(int(w[0]), int(w[1])) for w in reversed(list(window)))
        out = buf[(Ellipsis,) + sl].cpu().numpy()
        del buf
        return out

    def set_state(self, st: dict):
        for k, v in st.items():
            fw2_set_field(self.ctx, k, v)

    @property
    def launches(self) -> int:
        return fw2_kernel_launches(self.ctx)

    def close(self):
        if self.ctx:
            fw2_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
