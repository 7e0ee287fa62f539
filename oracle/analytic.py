"""Analytic relations of the paper (test infrastructure only).

* continuous dispersion relation of the multiple-relaxation model,
  Eq. (dispersion_relations) with Eq. (gamma1), Sec. 3.2 / appendix A;
* power-law attenuation target and its Kramers-Kronig phase velocity
  (Sec. 4.1; nearly-local form 1/c = 1/c0 + alpha0' tan(pi y / 2)
  (omega^(y-1) - omega_ref^(y-1)), and its y = 1 limit);
* the closed-form numerical dispersion relation of the lossless staggered
  leapfrog scheme of Sec. 3.1;
* the pre-shock (Poisson) solution of the inviscid Burgers equation and a
  Rusanov finite-volume solution of it, the nonlinear references of Sec. 4.5.
"""
from __future__ import annotations

import math

import numpy as np

NP_PER_DB = math.log(10.0) / 20.0


def gamma(omega, d, alpha, kappa):
    """gamma = sum_nu (d^nu / kappa^2) / (d^nu / kappa + alpha^nu + i omega), Eq. (gamma1)."""
    omega = np.asarray(omega, np.float64)
    g = np.zeros(omega.shape, np.complex128)
    for dn, an in zip(np.atleast_1d(d), np.atleast_1d(alpha)):
        g = g + (dn / kappa ** 2) / (dn / kappa + an + 1j * omega)
    return g


def wavenumber(omega, c, kappa1, kappa2, d1, alpha1, d2, alpha2):
    """Complex wavenumber k(omega) of Eq. (dispersion_relations), waves e^{i(omega t - k x)}."""
    omega = np.asarray(omega, np.float64)
    g1 = gamma(omega, d1, alpha1, kappa1)
    g2 = gamma(omega, d2, alpha2, kappa2)
    inner = 1.0 / (kappa1 * kappa2) - g1 / kappa2 - g2 / kappa1 + g1 * g2
    return (omega / c) * inner ** (-0.5)


def attenuation_db_cm(k):
    """Amplitude attenuation -Im(k) in dB/cm (k in 1/m), the attenuation of
    Eq. (dispersion_relations) in the units of Sec. 4.1."""
    return -np.imag(k) / NP_PER_DB / 100.0


def phase_velocity(omega, k):
    """Phase velocity omega / Re(k) of Eq. (dispersion_relations) (Sec. 4.1)."""
    return np.asarray(omega) / np.real(k)


def model_curves(freqs_hz, c, p):
    """(attenuation dB/cm, phase velocity m/s) of a parameter set dict at
    freqs: alpha_model and c_model of Eq. (relaxation_parameter_optimization),
    from Eq. (dispersion_relations)."""
    w = 2 * math.pi * np.asarray(freqs_hz, np.float64)
    k = wavenumber(w, c, p["kappa1"], p["kappa2"], np.asarray(p["d1"]), np.asarray(p["alpha1"]),
                   np.asarray(p["d2"]), np.asarray(p["alpha2"]))
    return attenuation_db_cm(k), phase_velocity(w, k)


def power_law_db_cm(freqs_hz, alpha0, y):
    """alpha(f) = alpha0 f^y, f in MHz, result in dB/cm: the target attenuation
    law of Sec. 4.1."""
    return alpha0 * (np.asarray(freqs_hz) / 1e6) ** y


def kk_phase_velocity(freqs_hz, alpha0, y, c0, f_ref):
    """Kramers-Kronig phase velocity of a power law (nearly-local form), the
    target phase velocity of Sec. 4.1 (its form is not printed there).

    alpha(omega) = a0 |omega|^y in Np/m with a0 from alpha0 [dB/cm/MHz^y];
    y != 1: 1/c = 1/c0 + a0 tan(pi y / 2) (omega^(y-1) - omega_ref^(y-1))
    y == 1: 1/c = 1/c0 - (2/pi) a0 ln(omega / omega_ref)
    """
    w = 2 * math.pi * np.asarray(freqs_hz, np.float64)
    wr = 2 * math.pi * f_ref
    a0 = alpha0 * NP_PER_DB * 100.0 / (2 * math.pi * 1e6) ** y
    if abs(y - 1.0) < 1e-12:
        inv = 1.0 / c0 - (2.0 / math.pi) * a0 * np.log(w / wr)
    else:
        inv = 1.0 / c0 + a0 * math.tan(math.pi * y / 2.0) * (w ** (y - 1.0) - wr ** (y - 1.0))
    return 1.0 / inv


def staggered_symbol(kh, taps):
    """sum_i g_i sin((2i-1) k h / 2): h/2 times the symbol of the staggered
    derivative D^{2M,4} of Sec. 3.1 without its cross tap."""
    kh = np.asarray(kh, np.float64)
    return sum(taps[i] * np.sin((2 * i + 1) * kh / 2.0) for i in range(4))


def discrete_omega(kvec_h, c, dt, h, taps):
    """omega of a plane wave exp(i(k.x - omega t)) under the lossless leapfrog
    scheme of Sec. 3.1 (the staggered updates with the operator D^{2M,4}).

    sin(omega dt / 2) = (c dt / h) sqrt(sum_q G_q^2),
    G_q = sum_i g_i sin((2i-1) k_q h / 2) + 2 g11 sin(k_q h / 2) sum_{t != q} cos(k_t h).
    """
    kvec_h = [np.asarray(k, np.float64) for k in kvec_h]
    s = 0.0
    for q, kq in enumerate(kvec_h):
        G = staggered_symbol(kq, taps)
        if taps[4] != 0.0:
            G = G + 2 * taps[4] * np.sin(kq / 2.0) * sum(np.cos(kt) for t, kt in enumerate(kvec_h) if t != q)
        s = s + G ** 2
    arg = c * dt / h * np.sqrt(s)
    return 2.0 / dt * np.arcsin(arg)


def burgers_poisson(p_in, t, x, beta_eff, rho0, c0, iters: int = 200):
    """Pre-shock solution of the inviscid Burgers equation for a progressive
    wave, the reference of the nonlinearity evaluation of Sec. 4.5.

    p(x, tau) = p_in(tau + beta_eff x p / (rho0 c0^3)), tau = t - x/c0 the
    retarded time (the implicit Poisson / Earnshaw form, valid before shock
    formation, sigma < 1).  `p_in` is a callable of time; solved by fixed
    point iteration.
    """
    tau = np.asarray(t, np.float64) - x / c0
    p = p_in(tau)
    coef = beta_eff * x / (rho0 * c0 ** 3)
    for _ in range(iters):
        p = p_in(tau + coef * p)
    return p


def burgers_rusanov(p_in, dtau, x, beta_eff, rho0, c0, cfl: float = 0.4):
    """The inviscid Burgers equation of a progressive wave, solved numerically
    with a Rusanov (local Lax-Friedrichs) finite-volume scheme, the reference
    solver of Sec. 4.5.

    In retarded time tau = t - x/c0 the wave obeys dp/dx = b p dp/dtau with
    b = beta_eff / (rho0 c0^3), a conservation law in the marching variable x:
    dp/dx + dF(p)/dtau = 0, F(p) = -b p^2 / 2.  `p_in` holds p at x = 0 on a
    uniform tau grid of spacing `dtau` (the pulse well inside it; p = 0 held at
    both ends).  Cell interfaces take piecewise-linear states with minmod
    slopes (second order away from extrema) and the Rusanov flux
    F* = (F(pL) + F(pR))/2 - a (pR - pL)/2, a = |b| max(|pL|, |pR|); the march
    in x is the two-stage strong-stability-preserving Runge-Kutta scheme with
    steps dx = cfl dtau / (|b| max |p|).  Returns p at distance x on the same
    tau grid.
    """
    u = np.array(p_in, np.float64)
    b = beta_eff / (rho0 * c0 ** 3)

    def rhs(v):
        w = np.concatenate([[0.0, 0.0], v, [0.0, 0.0]])
        d1, d2 = w[1:-1] - w[:-2], w[2:] - w[1:-1]
        slope = np.where(d1 * d2 > 0, np.sign(d1) * np.minimum(np.abs(d1), np.abs(d2)), 0.0)
        c = w[1:-1]
        pl = c[:-1] + 0.5 * slope[:-1]   # left state at interface i+1/2
        pr = c[1:] - 0.5 * slope[1:]     # right state
        a = abs(b) * np.maximum(np.abs(pl), np.abs(pr))
        flux = 0.5 * (-0.5 * b * pl ** 2 - 0.5 * b * pr ** 2) - 0.5 * a * (pr - pl)
        return -(flux[1:] - flux[:-1]) / dtau

    done = 0.0
    while done < x:
        amax = abs(b) * max(float(np.max(np.abs(u))), 1e-300)
        dx = min(cfl * dtau / amax, x - done)
        u1 = u + dx * rhs(u)
        u = 0.5 * (u + u1 + dx * rhs(u1))
        done += dx
    return u


def discrete_wavenumber_1d(freqs_hz, c, h, dt, p, taps, centred=True):
    """Complex k of the fully discrete 1D scheme with memory variables
    (Sec. 3.1 updates; recursion of Eqs. relaxation_a, relaxation_b,
    relaxation_psi).

    For a mode exp(i(omega t - k x)) the stored recursion
    chi^n = b chi^{n-1} + a D^n gives chi = a D / (1 - b e^{-i omega dt}); the
    stretched derivative is D (1/kappa + sum_nu a w / (1 - b e^{-i omega dt}))
    with w = (1 + e^{-i omega dt}) / 2 (centred) or 1 (endpoint).  Leapfrog in
    time and the staggered operator in space then give
    (h/dt) sin(omega dt / 2) = c sqrt(F1 F2) G(k h),
    G(z) = sum_i g_i sin((2i-1) z / 2), solved for complex k by Newton's method
    from the continuous estimate.
    """
    from .coefficients import relaxation_ab
    out = []
    for f in np.atleast_1d(np.asarray(freqs_hz, np.float64)):
        w = 2 * math.pi * f
        z1 = np.exp(-1j * w * dt)
        wgt = 0.5 * (1 + z1) if centred else 1.0
        def F(kap, d, al):
            a, b = relaxation_ab(np.asarray(d, np.float64), np.asarray(al, np.float64), kap, dt)
            return 1.0 / kap + np.sum(a * wgt / (1 - b * z1))
        F12 = F(p["kappa1"], p["d1"], p["alpha1"]) * F(p["kappa2"], p["d2"], p["alpha2"])
        rhs = (h / dt) * math.sin(w * dt / 2) / (c * np.sqrt(F12))
        z = w / c / np.sqrt(F12) * h
        for _ in range(100):
            g = sum(taps[i] * np.sin((2 * i + 1) * z / 2) for i in range(4)) - rhs
            dg = sum(taps[i] * (2 * i + 1) / 2 * np.cos((2 * i + 1) * z / 2) for i in range(4))
            step = g / dg
            z = z - step
            if abs(step) < 1e-15 * max(1.0, abs(z)):
                break
        out.append(z / h)
    return np.asarray(out)
