"""ctypes front end of the FP64 C stepper (test infrastructure only).

``OracleSim(problem)`` builds the coefficients with ``oracle.coefficients``
and advances the state with ``fw2_oracle.c``; the result is FP64.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Optional

import numpy as np

from . import coefficients as coef
from .build import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        _lib.orc_run.restype = None
        _lib.orc_derivative_face.restype = None
        _lib.orc_derivative_centre.restype = None
    return _lib


DP = C.POINTER(C.c_double)


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("nrelax", C.c_int32), ("n", C.c_int64 * 3),
                ("bc", C.c_int32 * 3), ("centred", C.c_int32), ("dt", C.c_double),
                ("h", C.c_double), ("g", C.c_double * 4), ("g11", C.c_double)]


class Coef(C.Structure):
    _fields_ = [("K", DP), ("chi", DP), ("buoy", DP * 3), ("ik1", DP * 3), ("a1", DP * 3),
                ("b1", DP * 3), ("ik2", DP * 3), ("a2", DP * 3), ("b2", DP * 3), ("k0f", DP * 3)]


class State(C.Structure):
    _fields_ = [("p", DP), ("v", DP * 3), ("psi1", DP * 3), ("psi2", DP * 3)]


class Sources(C.Structure):
    _fields_ = [("n_pts", C.c_int64), ("kind", C.POINTER(C.c_int32)), ("idx", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int32)), ("signal", DP), ("n_cols", C.c_int64), ("n_rows", C.c_int64)]


class Record(C.Structure):
    _fields_ = [("n_pts", C.c_int64), ("idx", C.POINTER(C.c_int64)), ("group", C.POINTER(C.c_int32)),
                ("n_groups", C.c_int64), ("trace", DP), ("n_rows", C.c_int64)]


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return DP()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(DP)


_KIND = {"p": 0, "vx": 1, "vy": 2, "vz": 3}
_STATE_NAMES = ("p", "vx", "vy", "vz")


def make_grid(shape, bc, dt, h, taps, nrelax, centred=True) -> Grid:
    nd = len(shape)
    G = Grid()
    G.ndim = nd
    G.nrelax = nrelax
    full = list(shape) + [1] * (3 - nd)
    for q in range(3):
        G.n[q] = int(full[q])
        G.bc[q] = 1 if (q < nd and bc[q] == "periodic") else 0
    G.centred = 1 if centred else 0
    G.dt = dt
    G.h = h
    for i in range(4):
        G.g[i] = taps[i]
    G.g11 = taps[4]
    return G


class OracleSim:
    """FP64 simulation of a synth.Problem with the paper's method."""

    def __init__(self, prob, round_to: Optional[str] = None, coefficients: Optional[Dict] = None,
                 window=None):
        """`window` = ((x0, x1), (y0, y1)[, (z0, z1)]) simulates only that sub-box
        of the grid (fields zero outside it); its values are exact at cells
        farther than 8 cells per step from every cut edge."""
        self.prob = prob
        nd = prob.ndim
        self.window = [tuple(w) for w in window] if window is not None else [(0, s) for s in prob.shape]
        self.wshape = tuple(w[1] - w[0] for w in self.window)
        for q in range(nd):
            if prob.bc[q] == "periodic" and self.window[q] != (0, prob.shape[q]):
                raise ValueError("a window cannot cut a periodic axis")
        self.cf = coefficients if coefficients is not None else coef.build(prob, round_to=round_to,
                                                                            window=self.window)
        self.dt = self.cf["dt"]
        n = int(np.prod(self.wshape))
        N = prob.nrelax
        self.G = make_grid(self.wshape, prob.bc, self.dt, prob.h, self.cf["taps"], N,
                           centred=(prob.memory_alignment == "centred"))
        self.p = np.zeros(n)
        self.v = [np.zeros(n) for _ in range(nd)]
        self.psi1 = [np.zeros((N, n)) for _ in range(nd)]
        self.psi2 = [np.zeros((N, n)) for _ in range(nd)]
        self.step_index = 0
        cf = self.cf
        self._keep = []
        self.C = Coef()
        self.C.K = _dp(cf["K"])
        self.C.chi = _dp(cf["chi"])
        for q in range(nd):
            for name in ("buoy", "ik1", "ik2", "a1", "b1", "a2", "b2", "k0f"):
                if f"{name}{q}" not in cf:
                    continue                   # k0f: only with the momentum factor
                arr = np.ascontiguousarray(cf[f"{name}{q}"], np.float64)
                self._keep.append(arr)
                getattr(self.C, name)[q] = _dp(arr)
        self.S = State()
        self._bind_state()
        # sources: one entry per (point, column)
        kinds, idxs, cols, sigs = [], [], [], []
        col0 = 0
        for s in prob.sources:
            li, keep = self._localise(s.idx)
            kinds.append(np.full(li.size, _KIND[s.kind], np.int32))
            idxs.append(li)
            cols.append(np.asarray(s.group, np.int32)[keep] + col0)
            sigs.append(np.asarray(s.signal, np.float64))
            col0 += s.signal.shape[1]
        self.src = Sources()
        if kinds:
            self._src_arrays = (np.concatenate(kinds), np.concatenate(idxs), np.concatenate(cols),
                                np.ascontiguousarray(np.concatenate(sigs, axis=1)))
            k, i, c_, sg = self._src_arrays
            self.src.n_pts = k.size
            self.src.kind = k.ctypes.data_as(C.POINTER(C.c_int32))
            self.src.idx = i.ctypes.data_as(C.POINTER(C.c_int64))
            self.src.col = c_.ctypes.data_as(C.POINTER(C.c_int32))
            self.src.signal = _dp(sg)
            self.src.n_cols = sg.shape[1]
            self.src.n_rows = sg.shape[0]
            self.n_signal_rows = sg.shape[0]
        else:
            self.src.n_pts = 0
            self.n_signal_rows = None
        self.rec = Record()
        self.trace = None
        if prob.sensors is not None:
            sn = prob.sensors
            li, keep = self._localise(sn.idx)
            self._rec_arrays = (li, np.ascontiguousarray(np.asarray(sn.group, np.int32)[keep]))
            self.trace = np.zeros((max(prob.n_steps, 1), sn.n_groups))
            self.rec.n_pts = li.size
            self.rec.idx = self._rec_arrays[0].ctypes.data_as(C.POINTER(C.c_int64))
            self.rec.group = self._rec_arrays[1].ctypes.data_as(C.POINTER(C.c_int32))
            self.rec.n_groups = sn.n_groups
            self.rec.trace = _dp(self.trace)
            self.rec.n_rows = self.trace.shape[0]
        else:
            self.rec.n_pts = 0

    def _localise(self, idx):
        """Global flat cell indices -> window-local ones (and the kept mask)."""
        idx = np.asarray(idx, np.int64)
        full = list(self.prob.shape) + [1] * (3 - self.prob.ndim)
        i = idx % full[0]
        j = (idx // full[0]) % full[1]
        k = idx // (full[0] * full[1])
        win = self.window + [(0, 1)] * (3 - len(self.window))
        keep = ((i >= win[0][0]) & (i < win[0][1]) & (j >= win[1][0]) & (j < win[1][1])
                & (k >= win[2][0]) & (k < win[2][1]))
        ws = [w[1] - w[0] for w in win]
        li = (i - win[0][0]) + ws[0] * ((j - win[1][0]) + ws[1] * (k - win[2][0]))
        return np.ascontiguousarray(li[keep].astype(np.int64)), keep

    def _crop(self, a):
        g = self.prob.grid_shape
        a = np.asarray(a)
        lead = a.shape[:-len(g)] if a.ndim > len(g) else ()
        a = a.reshape(lead + g)
        sl = tuple(slice(w[0], w[1]) for w in reversed(self.window))
        return a[(Ellipsis,) + sl]

    def _bind_state(self):
        self.S.p = _dp(self.p)
        for q in range(len(self.v)):
            self.S.v[q] = _dp(self.v[q])
            self.S.psi1[q] = _dp(self.psi1[q])
            self.S.psi2[q] = _dp(self.psi2[q])

    def set_state(self, st: Dict[str, np.ndarray], step: Optional[int] = None):
        """Load a state (as from synth.random_state) into the FP64 fields.
        Arrays shaped like the whole grid are cut to the window; arrays
        already shaped like the window are taken as they are.  `step` sets
        the index of the next time step (source and trace row)."""
        names = "xyz"
        N = self.prob.nrelax
        wg = tuple(reversed(self.wshape))

        def cut(a, lead=()):
            a = np.asarray(a)
            if a.shape == lead + wg and self.wshape != tuple(self.prob.shape):
                return a
            return self._crop(a.reshape(lead + self.prob.grid_shape))
        self.p[:] = cut(st["p"]).astype(np.float64).ravel()
        for q in range(len(self.v)):
            self.v[q][:] = cut(st["v" + names[q]]).astype(np.float64).ravel()
            if N and ("psi1" + names[q]) in st:
                self.psi1[q][:] = cut(st["psi1" + names[q]], (N,)).reshape(N, -1)
                self.psi2[q][:] = cut(st["psi2" + names[q]], (N,)).reshape(N, -1)
        if step is not None:
            self.step_index = int(step)

    def run(self, n_steps: int):
        lib().orc_run(C.byref(self.G), C.byref(self.C), C.byref(self.S),
                      C.byref(self.src) if self.src.n_pts else None,
                      C.byref(self.rec) if self.rec.n_pts else None,
                      C.c_int64(self.step_index), C.c_int64(n_steps))
        self.step_index += n_steps
        return self

    def field(self, name: str) -> np.ndarray:
        """A state array reshaped to the (window) grid, numpy order."""
        g = tuple(reversed(self.wshape))
        names = {"p": self.p}
        for q, ch in enumerate("xyz"[: len(self.v)]):
            names["v" + ch] = self.v[q]
            names["psi1" + ch] = self.psi1[q]
            names["psi2" + ch] = self.psi2[q]
        a = names[name].copy()
        if a.ndim == 2:
            return a.reshape((a.shape[0],) + g)
        return a.reshape(g)


def derivative(field: np.ndarray, h: float, axis_q: int, at: str, bc=("zero",) * 3, taps=None) -> np.ndarray:
    """The oracle's raw staggered derivative of one field (for the operator pins)."""
    g = field.shape
    shape = tuple(reversed(g))
    if taps is None:
        t = [float(x) for x in coef.taylor_staggered_taps(4)]
        taps = (t[0], t[1], t[2], t[3], 0.0)
    G = make_grid(shape, bc, 1.0, h, taps, 0)
    f = np.ascontiguousarray(field, np.float64).ravel()
    out = np.zeros_like(f)
    fn = lib().orc_derivative_face if at == "face" else lib().orc_derivative_centre
    fn(C.byref(G), _dp(f), C.c_int(axis_q), _dp(out))
    return out.reshape(g)
