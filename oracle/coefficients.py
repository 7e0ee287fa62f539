"""FP64 coefficient construction for the oracle (test infrastructure only).

Builds, from a ``synth.Problem``, every per-point and per-axis coefficient the
time step uses, straight from the paper's closed forms:

* b = exp(-(d/kappa + alpha) dt), a = d (b - 1) / (kappa (d + kappa alpha))
  -- Eqs. (relaxation_a), (relaxation_b), Sec. 3.2;
* the two-stage C-PML with transition layer -- Sec. 3.3, Table 1 and the
  polynomial / linear / cosine transition functions with
  X(x) = (X_target - X_0) g(x) + X_0;
* K = rho c^2, the nonlinear coefficient chi -- Eq. (general6);
* dt = CFL h / c_max with c_max the high-frequency speed c / sqrt(kappa1 kappa2)
  implied by Eq. (dispersion_relations) -- Sec. 3.4 (CFL 0.4).

Readings where the paper is silent (placement on the staggered grid):
rho at a face is the mean of the two adjacent cells (the cell itself at a
non-periodic outer edge); the relaxation parameters of a face are those of
its lower-index cell; the PML profile is evaluated at the exact staggered
coordinate of each point.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np


def time_space_taps(r: float, M: int = 4, D: int = 2):
    """Taps g_1..g_M and the cross tap g_11 of the D-dimensional staggered
    operator optimised for the leapfrog step at Courant number r = c dt / h
    (Sec. 3.1 cites a time-space-domain optimised set without printing it;
    this is our derivation from that principle), D = 2 or 3.

    With b_m = (2m-1)/2 and a_q = k_q h, the scheme's dispersion relation is
    sin^2(r |a| / 2) / r^2 = sum_q G_q^2, where
    G_q = sum_m g_m sin(b_m a_q) + 2 g_11 sin(a_q / 2) sum_{t != q} cos(a_t).
    Expanding, sum_q G_q^2 = A^2 |a|^2 - A g_11 |a|^4 + (A g_11 - 2 A B) sum_q a_q^4
    + O(a^6), with A the a_q coefficient and B the a_q^3 one of G_q along an
    axis.  The taps make the relation hold
      - to order a^4 in every direction: A = 1/2; the |a|^4 term is the time
        error r^2 |a|^4 / 48, which asks g_11 = r^2 / 24 in any D; the
        direction-dependent sum_q a_q^4 term vanishes, g_11 = 2 B;
      - along the axes to order a^(2M): the odd powers a^p, p = 1, 3, ...,
        2M-1, of G_q along an axis (where it has D - 1 cross pairs) equal
        those of sin(r a / 2) / r, i.e.
        sum_m g_m b_m^p + 2 g_11 (D - 1) (1/2)^p = r^(p-1) / 2^p
      (the p = 3 condition is g_11 = 2 B again).  At r = 0 this is the Taylor
    set with g_11 = 0.  Returns [g_1..g_M, g_11].
    """
    if D not in (2, 3):
        raise ValueError("D must be 2 or 3")
    r = float(r)
    b = np.array([(2 * m - 1) / 2.0 for m in range(1, M + 1)])
    g11 = r * r / 24.0
    ps = [2 * n + 1 for n in range(M)]
    A = np.array([[bm ** p for bm in b] for p in ps])
    rhs = np.array([r ** (p - 1) / 2.0 ** p - 2.0 * g11 * (D - 1) * 0.5 ** p for p in ps])
    g = np.linalg.solve(A, rhs)
    return [float(x) for x in g] + [g11]


def taylor_staggered_taps(M: int = 4):
    """Taylor coefficients g_1..g_M of the 2M-th order staggered first derivative.

    Solves sum_i g_i (2i-1)^(2m-1) = delta_{m,1}, m = 1..M, in exact rational
    arithmetic (Gauss-Jordan on fractions).  For M = 4 this gives
    1225/1024, -245/3072, 49/5120, -5/7168.
    """
    from fractions import Fraction
    A = [[Fraction((2 * i - 1) ** (2 * m - 1)) for i in range(1, M + 1)] for m in range(1, M + 1)]
    b = [Fraction(1 if m == 1 else 0) for m in range(1, M + 1)]
    n = M
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        inv = 1 / A[col][col]
        A[col] = [x * inv for x in A[col]]
        b[col] *= inv
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
                b[r] -= f * b[col]
    return b  # list of Fractions, g_1..g_M (the system is scaled so h = 1, D = sum g_i * diff / h)


def relaxation_ab(d, alpha, kappa, dt):
    """Recursion coefficients of Eqs. (relaxation_a), (relaxation_b), FP64.

    b = exp(-(d/kappa + alpha) dt);  a = d / (kappa (d + kappa alpha)) (b - 1).
    a is 0 where d = 0 (no memory contribution).
    """
    d = np.asarray(d, np.float64)
    alpha = np.asarray(alpha, np.float64)
    kappa = np.asarray(kappa, np.float64)
    b = np.exp(-(d / kappa + alpha) * dt)
    denom = kappa * (d + kappa * alpha)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(d == 0.0, 0.0, d / np.where(denom == 0.0, 1.0, denom) * (b - 1.0))
    return a, b


def high_frequency_speed(c, kappa1, kappa2):
    """c / sqrt(kappa1 kappa2): the omega -> infinity phase speed of Eq. (dispersion_relations)."""
    c = np.asarray(c, np.float64)
    if kappa1 is None:
        return c
    return c / np.sqrt(np.asarray(kappa1, np.float64) * np.asarray(kappa2, np.float64))


def cfl_time_step(prob, cfl: float = 0.4) -> float:
    """dt = CFL h / c_max (Sec. 3.4), c_max over the medium at high frequency."""
    return float(cfl * prob.h / high_frequency_speed(prob.c, prob.kappa1, prob.kappa2).max())


def boundary_depth(n: int, L: int, staggered: bool) -> np.ndarray:
    """Depth into the boundary region (in cells, 0..L) of each point on one
    axis: the coordinate of the C-PML profiles of Sec. 3.3 and Table 1.

    Cell centres sit at x = i, faces at x = i + 1/2.  The region occupies the
    outer L cells of each side: on the low side its inner edge is x = L - 1/2
    and its outer edge x = -1/2; on the high side x = n - L - 1/2 and n - 1/2.
    """
    x = np.arange(n, dtype=np.float64) + (0.5 if staggered else 0.0)
    depth = np.zeros(n, np.float64)
    if L <= 0:
        return depth
    lo_in = L - 0.5
    hi_in = n - L - 0.5
    depth = np.where(x < lo_in, lo_in - x, depth)
    depth = np.where(x > hi_in, x - hi_in, depth)
    return np.minimum(depth, float(L))


def boundary_profile(X0: np.ndarray, depth: np.ndarray, nu: int, which: str,
                     LT: int, LB: int, npow: float, d_target: float, reading: str) -> np.ndarray:
    """Relaxation parameter inside the two-stage C-PML (Sec. 3.3, Table 1).

    X(x) = (X_target - X0) g(x) + X0 with
      nu = 1, d    : polynomial g = (x/L)^npow toward d_target
      nu = 1, alpha: linear     g = x/L      toward 0
      nu >= 2      : cosine     g = (1 - cos(pi x / L_T)) / 2 toward 0 over
                     the transition layer, 0 beyond it.
    Reading A: the nu = 1 ramps span the whole boundary L_T + L_B.
    Reading K: as C for nu = 1, but the nu >= 2 parameters keep their
    interior values (no transition layer: the unstable configuration of
    Sec. 3.3).
    Reading C: as A for d^{nu=1}; alpha^{nu=1} is blended by the cosine
    transition over L_T from the tissue's value into the C-PML profile
    d_target (1 - x/L), which is linear to 0 at the outer edge (d_target
    plays the role of the maximum frequency shift of a C-PML), so the
    transition layer turns the tissue's first mechanism into the single
    C-PML mechanism.
    `nu` is 1-based as in the paper; `which` is "d" or "alpha".
    """
    if reading.upper() not in ("A", "C", "K"):
        raise ValueError(f"C-PML reading {reading!r}: A, C or K")
    if reading.upper() == "K":
        if nu >= 2:
            return np.asarray(X0, np.float64).copy()
        reading = "C"
    X0 = np.asarray(X0, np.float64)
    L = LT + LB
    out = X0.copy()
    inside = depth > 0
    if not np.any(inside) or L == 0:
        return out
    if nu == 1 and which == "alpha" and reading.upper() == "C":
        # the tissue's alpha is blended (cosine over the transition layer)
        # into the C-PML profile alpha_cfs = d_target (1 - x/L), which falls
        # linearly to 0 at the outer edge
        gT = np.where(depth < LT, 0.5 * (1.0 - np.cos(np.pi * depth / max(LT, 1))), 1.0) if LT > 0 \
            else np.ones_like(depth)
        a_cfs = d_target * (1.0 - depth / L)
        return np.where(inside, (1.0 - gT) * X0 + gT * a_cfs, X0)
    if nu == 1:
        s = depth / L
        active = inside
        if which == "d":
            g = s ** npow
            tgt = d_target
        else:
            g = s
            tgt = 0.0
        out = np.where(active, (tgt - X0) * g + X0, X0)
    else:
        if LT > 0:
            g = np.where(depth < LT, 0.5 * (1.0 - np.cos(np.pi * depth / LT)), 1.0)
        else:
            g = np.ones_like(depth)
        out = np.where(inside, (0.0 - X0) * g + X0, X0)
    return out


def to_bf16(x) -> np.ndarray:
    """Round FP64 values to float32, then to bfloat16 (round to nearest even),
    returned as FP64: the storage rounding of bf16 coefficient maps."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    finite = np.isfinite(f)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    r = np.where(finite, r, u.astype(np.uint32))
    return r.view(np.float32).astype(np.float64)


def f16_scale(values) -> float:
    """Power-of-two scale of an FP16 coefficient map: the largest magnitude of
    the map (as float32) divided by the scale lies in [2^14, 2^15)."""
    m = float(np.max(np.abs(np.asarray(values, np.float64)).astype(np.float32))) if np.size(values) else 0.0
    if not (m > 0.0) or not math.isfinite(m):
        return 1.0
    _, ex = math.frexp(m)                      # m in [2^(ex-1), 2^ex)
    return math.ldexp(1.0, ex - 15)


def to_f16(x, scale: float) -> np.ndarray:
    """Storage rounding of an FP16 map: x / scale (exact) rounded to float32,
    then to half (round to nearest even), times the scale, as FP64."""
    q = (np.asarray(x, np.float64) / scale).astype(np.float32).astype(np.float16)
    return q.astype(np.float64) * scale


def build(prob, round_to: Optional[str] = None, window=None) -> Dict[str, object]:
    """All coefficient arrays of the oracle step, FP64 (flat, x fastest):
    Eqs. (relaxation_a), (relaxation_b) per mechanism and axis, the C-PML
    profiles of Sec. 3.3 / Table 1, K = rho c^2 and the nonlinear factor of
    Eq. (general6) (with Eq. (general5)'s kappa0 at the faces in the literal
    mode).

    Keys: K, chi (or None), buoy[q], ik1[q], a1[q] (N, n), b1[q], ik2[q],
    a2[q], b2[q], dt, taps (g1..g4, g11).
    `round_to` = "f32" rounds every stored coefficient map to float32 first
    (models coefficient maps kept in single precision); "bf16" rounds them to
    bfloat16, with b stored as 1 - b (b = 1 - bf16(1 - b)) and the cell
    density rounded before the face average (models bf16 maps); "f16" rounds
    them to half precision after dividing each map by its power-of-two scale
    (f16_scale of the map's values over the whole grid; the relaxation
    coefficients of a mechanism share one scale over the tissue values of
    every cell and the C-PML values of every axis), b as 1 - b (models FP16
    maps; whole grids only).
    `window` = ((x0, x1), (y0, y1)[, (z0, z1)]) builds the coefficients of that
    sub-box of the grid only, with the boundary profiles and face densities of
    its global position.
    """
    nd = prob.ndim
    shape = list(prob.shape) + [1] * (3 - nd)
    gshape = tuple(reversed(shape))           # (nz, ny, nx)
    if window is None:
        window = [(0, s) for s in prob.shape]
    win = [tuple(w) for w in window] + [(0, 1)] * (3 - nd)
    wshape = [w[1] - w[0] for w in win]
    wg = tuple(reversed(wshape))
    n = int(np.prod(wshape))
    # numpy slices of the window in the global arrays
    sl = tuple(slice(win[q][0], win[q][1]) for q in (2, 1, 0))
    def crop(a):
        return np.asarray(a).reshape(gshape)[sl].astype(np.float64)
    rho_src = np.asarray(prob.rho).reshape(gshape)
    c = crop(prob.c)
    rho = crop(prob.rho)
    # the face densities use the stored (possibly bf16) cell density; K and
    # chi are built from the input density and rounded as maps afterwards
    if round_to == "f16" and any(tuple(w) != (0, sz) for w, sz in zip(window, prob.shape)):
        raise ValueError("FP16 map rounding needs the whole grid (the map scales come from every cell)")
    s_rho = f16_scale(rho) if round_to == "f16" else 1.0
    rho_face_src = to_bf16(rho) if round_to == "bf16" else to_f16(rho, s_rho) if round_to == "f16" else rho
    N = prob.nrelax
    dt = float(prob.dt) if prob.dt and prob.dt > 0 else cfl_time_step(prob)
    K = rho * c * c
    chi = None
    if prob.nl_mode != "off":
        beta = crop(prob.beta)
        kappa0 = 1.0 / K
        if prob.nl_mode in ("pressure", "literal"):
            chi = kappa0 * (1.0 - 2.0 * beta)        # Eq. (general6) factor
        elif prob.nl_mode == "westervelt":
            chi = -2.0 * beta * kappa0
        else:
            raise ValueError(prob.nl_mode)
    taps = prob.taps
    if taps is None:
        g = [float(x) for x in taylor_staggered_taps(4)]
        taps = (g[0], g[1], g[2], g[3], 0.0)
    out: Dict[str, object] = {"dt": dt, "taps": tuple(float(t) for t in taps), "K": K.ravel(),
                              "chi": None if chi is None else chi.ravel()}
    periodic = [prob.bc[q] == "periodic" for q in range(3)]
    axis_of = {0: 2, 1: 1, 2: 0}  # problem axis q -> numpy axis
    k1 = crop(prob.kappa1) if N else np.ones(wg)
    k2 = crop(prob.kappa2) if N else np.ones(wg)
    LT, LB = int(prob.pml_transition), int(prob.pml_bound)
    L = LT + LB
    cp = float(prob.pml_cp) if prob.pml_cp and prob.pml_cp > 0 else float(np.asarray(prob.c).max())
    d_target = -(prob.pml_npow + 1.0) * cp * math.log(prob.pml_rc) / (2.0 * L * prob.h) if L > 0 else 0.0
    for q in range(nd):
        ax = axis_of[q]
        # rho at the +1/2 face: mean of the cell and its +1 neighbour (global)
        idx_hi = np.arange(win[q][0], win[q][1]) + 1
        if periodic[q]:
            idx_hi = idx_hi % shape[q]
        else:
            idx_hi = np.minimum(idx_hi, shape[q] - 1)
        others = tuple(slice(None) if i == ax else s_ for i, s_ in enumerate(sl))
        nb = np.take(rho_src[others], idx_hi, axis=ax).astype(np.float64)
        if round_to == "bf16":
            nb = to_bf16(nb)
        elif round_to == "f16":
            nb = to_f16(nb, s_rho)
        out[f"buoy{q}"] = (1.0 / (0.5 * (rho_face_src + nb))).ravel()
        if prob.nl_mode == "literal":
            # kappa_0 at the face of the momentum factor rho_0 (1 + kappa_0 p)
            # (Eq. general5): mean of the two cells' 1/K, from K as stored
            # (same neighbour rule as the density)
            s_K = f16_scale(K) if round_to == "f16" else 1.0
            Kw = (to_bf16(K) if round_to == "bf16" else to_f16(K, s_K) if round_to == "f16" else
                  K.astype(np.float32).astype(np.float64) if round_to == "f32" else K)
            c_src, r_src = np.asarray(prob.c).reshape(gshape), rho_src
            K_src = r_src.astype(np.float64) * c_src.astype(np.float64) ** 2
            Knb = np.take(K_src[others], idx_hi, axis=ax)
            Knb = (to_bf16(Knb) if round_to == "bf16" else to_f16(Knb, s_K) if round_to == "f16" else
                   Knb.astype(np.float32).astype(np.float64) if round_to == "f32" else Knb)
            out[f"k0f{q}"] = (0.5 * (1.0 / Kw + 1.0 / Knb)).ravel()
        out[f"ik1{q}"] = (1.0 / k1).ravel()
        out[f"ik2{q}"] = (1.0 / k2).ravel()
        a1 = np.zeros((N, n)); b1 = np.zeros((N, n)); a2 = np.zeros((N, n)); b2 = np.zeros((N, n))
        for stag, (dname, aname, kap, A, B) in ((True, ("d1", "alpha1", k1, a1, b1)),
                                                  (False, ("d2", "alpha2", k2, a2, b2))):
            depth1 = boundary_depth(shape[q], L, staggered=stag)[win[q][0]:win[q][1]]
            bshape = [1, 1, 1]; bshape[ax] = wshape[q]
            depth = np.broadcast_to(depth1.reshape(bshape), wg)
            for nu in range(N):
                d0 = crop(getattr(prob, dname)[nu])
                al0 = crop(getattr(prob, aname)[nu])
                d = boundary_profile(d0, depth, nu + 1, "d", LT, LB, prob.pml_npow, d_target, prob.pml_reading)
                al = boundary_profile(al0, depth, nu + 1, "alpha", LT, LB, prob.pml_npow, d_target, prob.pml_reading)
                a, b = relaxation_ab(d, al, kap, dt)
                A[nu] = a.ravel(); B[nu] = b.ravel()
        out[f"a1{q}"], out[f"b1{q}"], out[f"a2{q}"], out[f"b2{q}"] = a1, b1, a2, b2
    if round_to == "f32":
        for k, v in list(out.items()):
            if isinstance(v, np.ndarray) and not k.startswith("k0f"):
                out[k] = v.astype(np.float32).astype(np.float64)
    elif round_to == "bf16":
        for k, v in list(out.items()):
            if not isinstance(v, np.ndarray):
                continue
            if k.startswith("buoy") or k.startswith("k0f"):
                continue                       # computed from the rounded cell values
            if k.startswith("b1") or k.startswith("b2"):
                out[k] = 1.0 - to_bf16(1.0 - v)
            else:
                out[k] = to_bf16(v)
    elif round_to == "f16":
        # the tissue (unstretched) coefficients of every cell take part in
        # each mechanism's scale with the C-PML values of every axis
        tissue_ab = {}
        for nu in range(N):
            for key, dname, aname, kap in (("1", "d1", "alpha1", k1), ("2", "d2", "alpha2", k2)):
                a, b = relaxation_ab(crop(getattr(prob, dname)[nu]), crop(getattr(prob, aname)[nu]), kap, dt)
                tissue_ab[(key, nu)] = (a.ravel(), b.ravel())
        scale = {"K": f16_scale(out["K"])}
        if out["chi"] is not None:
            scale["chi"] = f16_scale(out["chi"])
        scale["ik1"] = f16_scale(1.0 / k1)
        scale["ik2"] = f16_scale(1.0 / k2)
        for key in ("1", "2"):
            for nu in range(N):
                a_all = [tissue_ab[(key, nu)][0]] + [out[f"a{key}{q}"][nu] for q in range(nd)]
                b_all = [1.0 - tissue_ab[(key, nu)][1]] + [1.0 - out[f"b{key}{q}"][nu] for q in range(nd)]
                scale[f"a{key}", nu] = f16_scale(np.concatenate(a_all))
                scale[f"b{key}", nu] = f16_scale(np.concatenate(b_all))
        out["K"] = to_f16(out["K"], scale["K"])
        if out["chi"] is not None:
            out["chi"] = to_f16(out["chi"], scale["chi"])
        for q in range(nd):
            out[f"ik1{q}"] = to_f16(out[f"ik1{q}"], scale["ik1"])
            out[f"ik2{q}"] = to_f16(out[f"ik2{q}"], scale["ik2"])
            for key in ("1", "2"):
                A, B = out[f"a{key}{q}"], out[f"b{key}{q}"]
                for nu in range(N):
                    A[nu] = to_f16(A[nu], scale[f"a{key}", nu])
                    B[nu] = 1.0 - to_f16(1.0 - B[nu], scale[f"b{key}", nu])
    elif round_to is not None:
        raise ValueError(round_to)
    return out
