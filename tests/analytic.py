"""Closed-form solutions printed in the paper, used to pin the FP64 oracle.

Each function restates a formula of the paper in numpy; none of them shares
code with the oracle or the GPU path.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq
from scipy.special import erf, erfc


# ---------------------------------------------------------------------------------------------
# Three-phase Stefan problem, Sec. 4.2: front s(t) = 2 kappa sqrt(alpha_s t)
# ---------------------------------------------------------------------------------------------

def neumann_kappa(ste: float, T0: float = 0.0, Tm: float = 0.0, Tw: float = -1.0,
                  lam_s: float = 1.0, lam_l: float = 1.0, alpha_r: float = 1.0,
                  rho_r: float = 1.0) -> float:
    """Root of the transcendental equation of Sec. 4.2,
        Ste / (exp(k^2) erf k)
          - lam_l (T0 - Tm) sqrt(alpha_r) Ste / (lam_s (Tm - Tw) exp((sqrt(alpha_r) k rho_r)^2)
                                                  erfc(sqrt(alpha_r) k rho_r)) = k sqrt(pi),
    with the printed "exp(...)^2" read as exp((...)^2); alpha_r = alpha_s/alpha_l,
    rho_r = rho_s/rho_l.  For T0 = Tm the second term vanishes."""
    def fun(k):
        a = ste / (math.exp(k * k) * math.erf(k))
        if T0 != Tm:
            z = math.sqrt(alpha_r) * k * rho_r
            a -= (lam_l * (T0 - Tm) * math.sqrt(alpha_r) * ste /
                  (lam_s * (Tm - Tw) * math.exp(z * z) * math.erfc(z)))
        return a - k * math.sqrt(math.pi)
    return brentq(fun, 1e-9, 5.0, xtol=1e-15, rtol=1e-15)


def neumann_front(t, kappa: float, alpha_s: float):
    return 2.0 * kappa * np.sqrt(alpha_s * np.asarray(t, dtype=np.float64))


# ---------------------------------------------------------------------------------------------
# Binary solidification, Sec. 4.3 (semi-infinite, x >= 0, liquid at T0, C0)
# ---------------------------------------------------------------------------------------------

def binary_stefan_k(cp_s, cp_l, L, Tm, Tb, T0, alpha_s, alpha_l) -> float:
    """Root of Cp_s (Tm - Tb) / (L exp(k^2) erf k)
               - Cp_l (T0 - Tm) sqrt(alpha_l/alpha_s) / (L exp(k^2 alpha_s/alpha_l) erfc(k sqrt(alpha_s/alpha_l)))
               = k sqrt(pi)."""
    def fun(k):
        a = cp_s * (Tm - Tb) / (L * math.exp(k * k) * math.erf(k))
        if T0 != Tm:
            r = alpha_s / alpha_l
            a -= cp_l * (T0 - Tm) * math.sqrt(1.0 / r) / (L * math.exp(k * k * r) * math.erfc(k * math.sqrt(r)))
        return a - k * math.sqrt(math.pi)
    return brentq(fun, 1e-9, 5.0, xtol=1e-15, rtol=1e-15)


def binary_stefan_fields(x, t, k, Tb, Tm, T0, C0, kp, alpha_s, alpha_l, D_l):
    """T(x, t) and C(x, t) of Sec. 4.3; the front is at s = 2 k sqrt(alpha_s t)."""
    x = np.asarray(x, dtype=np.float64)
    s = 2.0 * k * math.sqrt(alpha_s * t)
    Ts = Tb - (Tb - Tm) / math.erf(k) * erf(x / (2.0 * math.sqrt(alpha_s * t)))
    Tl = T0 + (Tm - T0) / math.erfc(k * math.sqrt(alpha_s / alpha_l)) * erfc(x / (2.0 * math.sqrt(alpha_l * t)))
    a = k * k * alpha_s / D_l
    den = math.exp(-a) - (1.0 - kp) * k * math.sqrt(math.pi * alpha_s / D_l) * math.erfc(k * math.sqrt(alpha_s / D_l))
    Cs = kp * C0 * math.exp(-a) / den
    Cl = C0 + (1.0 - kp) * C0 * k * math.sqrt(math.pi * alpha_s / D_l) / den * erfc(x / (2.0 * math.sqrt(D_l * t)))
    T = np.where(x < s, Ts, Tl)
    C = np.where(x < s, Cs, Cl)
    return T, C, s


# ---------------------------------------------------------------------------------------------
# Appendix A: Marangoni convection in a vertically stratified system
# ---------------------------------------------------------------------------------------------

def stratified_marangoni(x, y, L, h, H, Th, Tc, T0, sigma_T, mu_h, lam_r=1.0, mu_r=1.0):
    """Temperature and velocity of Appendix A.  y = 0 at the interface, the lower
    (heavy, superscript H) fluid in -h < y < 0, the upper (light, superscript L)
    fluid in 0 < y < H; lam_r = lambda_upper / lambda_lower, mu_r likewise.
    Returns T, ux, uy on the broadcast of x and y."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = 2.0 * math.pi / L
    Ht, ht = H * w, h * w
    f = 1.0 / (lam_r * math.sinh(ht) * math.cosh(Ht) + math.sinh(Ht) * math.cosh(ht))
    g = math.sinh(Ht) * f
    dH = math.sinh(Ht) ** 2 - Ht ** 2
    dh = math.sinh(ht) ** 2 - ht ** 2
    hh = dH * dh / (mu_r * dh * (math.sinh(2 * Ht) - 2 * Ht) + dH * (math.sinh(2 * ht) - 2 * ht))
    Umax = -(T0 * sigma_T / mu_h) * g * hh
    C1H, C2H, C3H = math.sinh(Ht) ** 2 / dH, -H * Ht / dH, (2 * Ht - math.sinh(2 * Ht)) / (2 * dH)
    C1h, C2h, C3h = math.sinh(ht) ** 2 / dh, -h * ht / dh, (math.sinh(2 * ht) - 2 * ht) / (2 * dh)
    den = H + lam_r * h
    TL = ((Tc - Th) * y + lam_r * Tc * h + Th * H) / den + T0 * f * np.sinh(Ht - w * y) * np.cos(w * x)
    TH = ((lam_r * (Tc - Th) * y + lam_r * Tc * h + Th * H) / den
          + T0 * f * (math.sinh(Ht) * np.cosh(w * y) - lam_r * np.sinh(w * y) * math.cosh(Ht)) * np.cos(w * x))
    uxL = Umax * ((C1H + w * (C2H + C3H * y)) * np.cosh(w * y) + (C3H + w * C1H * y) * np.sinh(w * y)) * np.sin(w * x)
    uyL = -w * Umax * (C1H * y * np.cosh(w * y) + (C2H + C3H * y) * np.sinh(w * y)) * np.cos(w * x)
    uxH = Umax * ((C1h + w * (C2h + C3h * y)) * np.cosh(w * y) + (C3h + w * C1h * y) * np.sinh(w * y)) * np.sin(w * x)
    uyH = -w * Umax * (C1h * y * np.cosh(w * y) + (C2h + C3h * y) * np.sinh(w * y)) * np.cos(w * x)
    up = y >= 0
    return np.where(up, TL, TH), np.where(up, uxL, uxH), np.where(up, uyL, uyH), Umax


# ---------------------------------------------------------------------------------------------
# Single-phase references
# ---------------------------------------------------------------------------------------------

def poiseuille(yc, ny, g, nu):
    """Force-driven channel flow between walls at y = -1/2 and y = ny - 1/2."""
    s = np.asarray(yc, dtype=np.float64) + 0.5
    return g / (2.0 * nu) * s * (ny - s)


def ygb_velocity(sigma_T, gradT, R, mu_h, mu_l, alpha_l, alpha_h):
    """Young-Goldstein-Block migration speed (Sec. 4.1)."""
    U = -sigma_T * gradT * R / mu_h
    return 2.0 * U / ((2.0 + 3.0 * mu_l / mu_h) * (2.0 + alpha_l / alpha_h))


def contact_angle_bottom(phi):
    """Contact angle (degrees, inside the phi > 0 phase) of a droplet sitting on
    the bottom wall (at y = -1/2), from a least-squares circle through the
    phi = 0 contour: for a circular cap of radius R centred at height y_c,
    cos(theta) = (-1/2 - y_c) / R.  Contour points are the linear-interpolation
    crossings along rows (both sides) and along columns (top side)."""
    import numpy as _np
    ny, nx = phi.shape
    pts = []
    for y in range(ny):
        row = phi[y]
        for x in range(nx - 1):
            a, b = row[x], row[x + 1]
            if (a > 0) != (b > 0):
                pts.append((x + a / (a - b), y))
    for x in range(nx):
        col = phi[:, x]
        for y in range(ny - 1):
            a, b = col[y], col[y + 1]
            if (a > 0) != (b > 0):
                pts.append((x, y + a / (a - b)))
    P = _np.array(pts, dtype=_np.float64)
    A = _np.column_stack([P[:, 0], P[:, 1], _np.ones(len(P))])
    rhs = -(P[:, 0] ** 2 + P[:, 1] ** 2)
    (D, E, F), *_ = _np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = -D / 2.0, -E / 2.0
    R = math.sqrt(xc * xc + yc * yc - F)
    return math.degrees(math.acos(max(-1.0, min(1.0, (-0.5 - yc) / R)))), R, (xc, yc)
