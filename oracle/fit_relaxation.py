"""Fit relaxation parameter sets to power-law attenuation (host tool, FP64).

Minimises the paper's cost J = w NMSE(alpha_model, alpha_target)
+ (1 - w) NMSE(c_model, c_target), w = 0.1 (Sec. 4.1,
Eq. relaxation_parameter_optimization), over 1-20 MHz, with alpha_model and
c_model from Eq. (dispersion_relations) and the Kramers-Kronig phase velocity
as c_target.  The search runs in log space for d and alpha and linearly for
kappa inside the Table 2 bounds; it is a multi-start bounded quasi-Newton
search (`fit`), or the paper's coarse-to-fine grid search (`fit_grid`: 5 values
per dimension over the bounds, then finer grids around the best point, each
30 % narrower in every dimension, Sec. 4.1).

Writes synth/relaxation_sets.json, the parameter sets the synthetic
workloads use as inputs.  Run:  python -m oracle.fit_relaxation
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
from scipy.optimize import minimize

from . import analytic as an

W_ALPHA = 0.1
BOUNDS_KAPPA = (0.8, 1.2)
BOUNDS_LOG_D = (2.0, 10.0)
BOUNDS_LOG_ALPHA = (5.0, 12.0)


def nmse(x, y):
    """NMSE of Sec. 4.1: mean squared error over the variance of the target."""
    return float(np.mean((x - y) ** 2) / np.var(y))


def unpack(theta, N):
    k1, k2 = theta[0], theta[1]
    ld1 = theta[2:2 + N]; ld2 = theta[2 + N:2 + 2 * N]
    la1 = theta[2 + 2 * N:2 + 3 * N]; la2 = theta[2 + 3 * N:2 + 4 * N]
    return {"kappa1": float(k1), "kappa2": float(k2),
            "d1": [float(10 ** v) for v in ld1], "d2": [float(10 ** v) for v in ld2],
            "alpha1": [float(10 ** v) for v in la1], "alpha2": [float(10 ** v) for v in la2]}


def cost(theta, N, f, c0, att_t, c_t):
    """J of Eq. (relaxation_parameter_optimization), w_alpha = 0.1 (Sec. 4.1)."""
    p = unpack(theta, N)
    att, cph = an.model_curves(f, c0, p)
    if not np.all(np.isfinite(att)) or not np.all(np.isfinite(cph)):
        return 1e6
    return W_ALPHA * nmse(att, att_t) + (1 - W_ALPHA) * nmse(cph, c_t)


def fit(alpha0, y, N, c0=1540.0, f_ref=3e6, n_starts=24, seed=0):
    """Minimise J (Sec. 4.1) over N mechanisms inside the Table 2 bounds by a
    multi-start bounded quasi-Newton search polished by Nelder-Mead; returns
    the parameter dict with its cost and the attenuation / phase errors."""
    f = np.linspace(1e6, 20e6, 77)
    att_t = an.power_law_db_cm(f, alpha0, y)
    c_t = an.kk_phase_velocity(f, alpha0, y, c0, f_ref)
    rng = np.random.default_rng(seed)
    bounds = [BOUNDS_KAPPA, BOUNDS_KAPPA] + [BOUNDS_LOG_D] * (2 * N) + [BOUNDS_LOG_ALPHA] * (2 * N)
    best = None
    for s in range(n_starts):
        x0 = np.array([rng.uniform(*b) for b in bounds])
        # spread initial relaxation frequencies over the band
        x0[2 + 2 * N:2 + 3 * N] = np.sort(rng.uniform(6.5, 10.5, N))
        x0[2 + 3 * N:] = np.sort(rng.uniform(6.0, 9.5, N))
        r = minimize(cost, x0, args=(N, f, c0, att_t, c_t), method="L-BFGS-B", bounds=bounds,
                     options={"maxiter": 3000})
        r = minimize(cost, r.x, args=(N, f, c0, att_t, c_t), method="Nelder-Mead",
                     options={"maxiter": 20000, "xatol": 1e-6, "fatol": 1e-12})
        r.x = np.clip(r.x, [b[0] for b in bounds], [b[1] for b in bounds])
        val = cost(r.x, N, f, c0, att_t, c_t)
        if best is None or val < best[0]:
            best = (val, r.x)
    p = unpack(best[1], N)
    att, cph = an.model_curves(f, c0, p)
    p.update({"alpha0": alpha0, "y": y, "c0": c0, "f_ref": f_ref, "J": best[0],
              "max_att_rel_err_2_20MHz": float(np.max(np.abs(att / att_t - 1)[f >= 2e6])),
              "max_phase_rel_err": float(np.max(np.abs(cph / c_t - 1)))})
    return p


# bounds of the paper's search (Sec. 4.1): kappa linear, d and alpha in log10
PAPER_BOUNDS = {"kappa": (0.8, 1.2), "log_d": (2.0, 10.0), "log_alpha": (5.0, 12.0)}


def curves_batch(freqs_hz, c0, k1, k2, d1, a1, d2, a2):
    """Attenuation (dB/cm) and phase velocity of B parameter sets at once:
    Eq. (gamma1) and Eq. (dispersion_relations) with broadcasting; k1, k2 of
    shape (B,), d1, a1, d2, a2 of shape (N, B).  Returns arrays (B, F)."""
    w = 2 * math.pi * np.asarray(freqs_hz, np.float64)[None, :]
    k1 = k1[:, None]
    k2 = k2[:, None]

    def gam(d, a, kap):
        g = np.zeros((d.shape[1], w.shape[1]), np.complex128)
        for n in range(d.shape[0]):
            dn, an_ = d[n][:, None], a[n][:, None]
            g += (dn / kap ** 2) / (dn / kap + an_ + 1j * w)
        return g

    g1 = gam(d1, a1, k1)
    g2 = gam(d2, a2, k2)
    inner = 1.0 / (k1 * k2) - g1 / k2 - g2 / k1 + g1 * g2
    k = (w / c0) * inner ** (-0.5)
    return an.attenuation_db_cm(k), an.phase_velocity(w, k)


def grid_cost(theta, N, f, c0, att_t, c_t):
    """Cost J (Eq. relaxation_parameter_optimization) of B parameter vectors
    theta (B, 2 + 4N) in the layout of unpack."""
    k1, k2 = theta[:, 0], theta[:, 1]
    d1 = 10.0 ** theta[:, 2:2 + N].T
    d2 = 10.0 ** theta[:, 2 + N:2 + 2 * N].T
    a1 = 10.0 ** theta[:, 2 + 2 * N:2 + 3 * N].T
    a2 = 10.0 ** theta[:, 2 + 3 * N:2 + 4 * N].T
    with np.errstate(all="ignore"):
        att, cph = curves_batch(f, c0, k1, k2, d1, a1, d2, a2)
        j = (W_ALPHA * np.mean((att - att_t) ** 2, axis=1) / np.var(att_t)
             + (1 - W_ALPHA) * np.mean((cph - c_t) ** 2, axis=1) / np.var(c_t))
    j[~np.isfinite(j)] = np.inf
    return j


def _level_best(args):
    """Best point of one slice [start, end) of a level's grid (pool worker)."""
    start, end, axes, N, f, c0, att_t, c_t, chunk = args
    D, points = len(axes), len(axes[0])
    best = (np.inf, None)
    for s0 in range(start, end, chunk):
        idx = np.unravel_index(np.arange(s0, min(s0 + chunk, end)), (points,) * D)
        theta = np.stack([axes[i][idx[i]] for i in range(D)], axis=1)
        j = grid_cost(theta, N, f, c0, att_t, c_t)
        m = int(np.argmin(j))
        if j[m] < best[0]:
            best = (float(j[m]), theta[m].copy())
    return best


def fit_grid(alpha0, y, N, c0=1540.0, f_ref=3e6, points=5, refinements=4, shrink=0.3, chunk=20000,
             target=None, workers=1):
    """The paper's coarse-to-fine grid search (Sec. 4.1): `points` values per
    dimension spanning the current range (first the bounds), the best of the
    whole grid becomes the centre of the next search, whose range in every
    dimension is (1 - shrink) of the previous one; grid values beyond the
    bounds are moved onto them, so with an odd `points` the previous best is
    a point of every finer grid and the best cost never rises.
    1 + refinements searches in all.  target: optional (att, c) curves to fit
    instead of the power law; workers > 1 splits each grid over a process
    pool.  Returns the parameter dict, each level's best cost in `J_levels`."""
    f = np.linspace(1e6, 20e6, 77)
    if target is None:
        att_t = an.power_law_db_cm(f, alpha0, y)
        c_t = an.kk_phase_velocity(f, alpha0, y, c0, f_ref)
    else:
        att_t, c_t = target
    b = PAPER_BOUNDS
    lo = np.array([b["kappa"][0]] * 2 + [b["log_d"][0]] * (2 * N) + [b["log_alpha"][0]] * (2 * N))
    hi = np.array([b["kappa"][1]] * 2 + [b["log_d"][1]] * (2 * N) + [b["log_alpha"][1]] * (2 * N))
    blo, bhi = lo.copy(), hi.copy()
    D = lo.size
    total = points ** D
    pool = None
    if workers > 1:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(workers)
    best_theta, best_j, levels = None, np.inf, []
    centre, width = (lo + hi) / 2.0, hi - lo
    try:
        for level in range(refinements + 1):
            axes = [np.clip(np.linspace(centre[i] - width[i] / 2, centre[i] + width[i] / 2, points), blo[i], bhi[i])
                    for i in range(D)]
            cuts = np.linspace(0, total, (workers if pool else 1) + 1).astype(np.int64)
            jobs = [(int(cuts[i]), int(cuts[i + 1]), axes, N, f, c0, att_t, c_t, chunk)
                    for i in range(len(cuts) - 1)]
            results = pool.map(_level_best, jobs) if pool else [_level_best(jobs[0])]
            level_best = min(results, key=lambda r: r[0])
            levels.append(level_best[0])
            if level_best[0] < best_j:
                best_j, best_theta = level_best
            centre, width = best_theta, width * (1.0 - shrink)
    finally:
        if pool:
            pool.close()
            pool.join()
    p = unpack(best_theta, N)
    att, cph = an.model_curves(f, c0, p)
    p.update({"alpha0": alpha0, "y": y, "c0": c0, "f_ref": f_ref, "J": best_j, "J_levels": levels,
              "max_att_rel_err_2_20MHz": float(np.max(np.abs(att / att_t - 1)[f >= 2e6])),
              "max_phase_rel_err": float(np.max(np.abs(cph / c_t - 1)))})
    return p


TARGETS = {
    "N4_y1.1_a0.5": (0.5, 1.1, 4, 1540.0, 3e6),
    "N4_y1.1_fat": (0.48, 1.1, 4, 1478.0, 3e6),
    "N4_y1.1_muscle": (1.09, 1.1, 4, 1547.0, 3e6),
    "N4_y1.1_connective": (1.57, 1.1, 4, 1613.0, 3e6),
    "N3_y1.2_brain": (0.6, 1.2, 3, 1560.0, 1e6),
    "N3_y1.2_skull": (6.0, 1.2, 3, 2700.0, 1e6),
    "N2_y1.0_a0.5": (0.5, 1.0, 2, 1540.0, 3e6),
}


def main():
    out = {}
    for key, (a0, y, N, c0, fr) in TARGETS.items():
        p = fit(a0, y, N, c0=c0, f_ref=fr)
        out[key] = p
        print(key, "J=%.3e att_err=%.4f phase_err=%.5f" % (p["J"], p["max_att_rel_err_2_20MHz"], p["max_phase_rel_err"]))
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "synth", "relaxation_sets.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print("wrote", path)


if __name__ == "__main__":
    main()
