"""Fit relaxation parameter sets to power-law attenuation (host tool, FP64).

Minimises the paper's cost J = w NMSE(alpha_model, alpha_target)
+ (1 - w) NMSE(c_model, c_target), w = 0.1 (Sec. 4.1,
Eq. relaxation_parameter_optimization), over 1-20 MHz, with alpha_model and
c_model from Eq. (dispersion_relations) and the Kramers-Kronig phase velocity
as c_target.  The search runs in log space for d and alpha and linearly for
kappa inside the Table 2 bounds; it is a multi-start bounded quasi-Newton
search rather than the paper's coarse-to-fine grid (same cost, same bounds).

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
    return float(np.mean((x - y) ** 2) / np.var(y))


def unpack(theta, N):
    k1, k2 = theta[0], theta[1]
    ld1 = theta[2:2 + N]; ld2 = theta[2 + N:2 + 2 * N]
    la1 = theta[2 + 2 * N:2 + 3 * N]; la2 = theta[2 + 3 * N:2 + 4 * N]
    return {"kappa1": float(k1), "kappa2": float(k2),
            "d1": [float(10 ** v) for v in ld1], "d2": [float(10 ** v) for v in ld2],
            "alpha1": [float(10 ** v) for v in la1], "alpha2": [float(10 ** v) for v in la2]}


def cost(theta, N, f, c0, att_t, c_t):
    p = unpack(theta, N)
    att, cph = an.model_curves(f, c0, p)
    if not np.all(np.isfinite(att)) or not np.all(np.isfinite(cph)):
        return 1e6
    return W_ALPHA * nmse(att, att_t) + (1 - W_ALPHA) * nmse(cph, c_t)


def fit(alpha0, y, N, c0=1540.0, f_ref=3e6, n_starts=24, seed=0):
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
