"""Seeded synthetic inputs: grids, model parameters and initial fields.

This module only builds inputs.  It holds none of the LB method's arithmetic,
so both the GPU path and the FP64 oracle can be fed from it.  Every workload
is a dict ``{"grid": ..., "params": ..., "fields": ..., "steps": ..., "name": ...}``:

* ``grid``   -- lattice size and wall conditions (x is always periodic; walls
  sit half-way between rows, at y = -1/2 and y = ny - 1/2);
* ``params`` -- per-phase properties (liquid ``_l``, solid ``_s``, the
  surrounding phase phi = -1 ``_g``), enthalpy, solute, interface and
  surface-tension constants;
* ``fields`` -- initial phi, T, C, ux, uy as float64 arrays of shape (ny, nx).

The order parameter starts from the equilibrium profile phi = tanh(2 d / W)
with d the signed distance to the interface (positive inside the
phase-change material) and W = 4 cells, i.e. epsilon = W / (2 sqrt 2)
(Eq. 3 with phi_1 = 1, phi_2 = -1).

Lattice-unit values that the paper does not fix are chosen here and stated
beside each workload.
"""
from __future__ import annotations

import math

import numpy as np

WALL_DIRICHLET_T = 0
WALL_ADIABATIC = 1

INTERFACE_WIDTH = 4.0
EPS = INTERFACE_WIDTH / (2.0 * math.sqrt(2.0))


def base_params(**kw) -> dict:
    """Liquid-like defaults in lattice units: rho_l = Cp = 1, nu = 0.1 in every
    phase, lambda = 0.3, mobility 0.1, eps = sqrt(2) (W = 4).

    div u in the phase-field and enthalpy sources (Sec. 3.1, 3.3): with phase
    change the default is the lagged velocity divergence (divu_mode = 1), the
    reading that reproduces the final heights of Table 1 and the final droplet
    volume of Sec. 4.4; without phase change it is the model value mdot = 0 of
    Eq. NS1 (divu_mode = 0), which conserves sum phi exactly.  An explicit
    ``divu_mode`` overrides either."""
    p = dict(rho_l=1.0, rho_s=1.0, rho_g=1.0, mu_l=0.1, mu_s=0.1, mu_g=0.1,
             lam_l=0.3, lam_s=0.3, lam_g=0.3, cp_l=1.0, cp_s=1.0, cp_g=1.0,
             latent=10.0, T_sol=0.0, T_liq=0.0, k_p=1.0, D_l=0.1, D_s=0.1,
             eps=EPS, mobility=0.1, sigma0=1e-3, sigma_T=0.0, sigma_c=0.0, T_ref=0.0,
             c_ref=0.0, gx=0.0, gy=0.0, fs_modulated_st=1, phase_change_on=1)
    p.update(kw)
    p.setdefault("divu_mode", 1 if p["phase_change_on"] else 0)
    return p


def gas_properties(p: dict, rho_g: float, nu: float = 0.1, lam_ratio: float = 0.1) -> dict:
    """Surrounding phase with density rho_g, the liquid's volumetric heat
    capacity (rho Cp)_g = (rho Cp)_l, conductivity lam_ratio * lam_l and the
    common kinematic viscosity nu."""
    p = dict(p)
    p["rho_g"] = rho_g
    p["cp_g"] = p["rho_l"] * p["cp_l"] / rho_g
    p["lam_g"] = lam_ratio * p["lam_l"]
    p["mu_l"] = nu * p["rho_l"]
    p["mu_s"] = nu * p["rho_s"]
    p["mu_g"] = nu * rho_g
    return p


def grid(nx, ny, bc_bottom=WALL_DIRICHLET_T, bc_top=WALL_ADIABATIC, T_bottom=0.0, T_top=0.0,
         T_bottom_amp=0.0, T_bottom_modes=1, theta_bottom=90.0, theta_top=90.0) -> dict:
    """Lattice and walls; theta_* are the contact angles in degrees (inside the
    phi = 1 phase), passed on as their cosines (exactly 0 at 90 degrees)."""
    def cosd(t):
        return 0.0 if float(t) == 90.0 else math.cos(math.radians(float(t)))
    return dict(nx=int(nx), ny=int(ny), bc_bottom=int(bc_bottom), bc_top=int(bc_top),
                T_bottom=float(T_bottom), T_top=float(T_top), T_bottom_amp=float(T_bottom_amp),
                T_bottom_modes=int(T_bottom_modes), cos_theta_bottom=cosd(theta_bottom),
                cos_theta_top=cosd(theta_top))


def tanh_profile(d: np.ndarray, width: float = INTERFACE_WIDTH) -> np.ndarray:
    return np.tanh(2.0 * d / width)


def _coords(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def _fields(phi, T, C, ux=None, uy=None) -> dict:
    z = np.zeros_like(phi)
    return dict(phi=phi, T=T, C=C, ux=z.copy() if ux is None else ux, uy=z.copy() if uy is None else uy)


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------

def stefan_layer(nx=64, ny=256, h0=128, ste=0.1, rho_ratio=0.9, rho_g=0.1, T_wall=-1.0,
                 T_melt=0.0, lam=0.3, steps=2000) -> dict:
    """Film freezing on a cold wall with a gas layer on top (three-phase Stefan
    problem, Sec. 4.2): liquid for y < h0, gas above; bottom wall Dirichlet
    T_wall, top adiabatic; T_0 = T_m everywhere; L = Cp_s (T_m - T_w) / Ste;
    rho_s / rho_l = rho_ratio; no solute, no Marangoni stress."""
    x, y = _coords(nx, ny)
    d = (h0 - 0.5) - y
    phi = tanh_profile(d)
    T = np.full_like(phi, T_melt)
    C = np.zeros_like(phi)
    p = base_params(rho_s=rho_ratio, lam_l=lam, lam_s=lam, T_sol=T_melt, T_liq=T_melt,
                    latent=1.0 * (T_melt - T_wall) / ste)
    p = gas_properties(p, rho_g)
    g = grid(nx, ny, WALL_DIRICHLET_T, WALL_ADIABATIC, T_bottom=T_wall)
    return dict(name="stefan_layer_%dx%d" % (nx, ny), grid=g, params=p,
                fields=_fields(phi, T, C), steps=steps,
                meta=dict(h0=h0, ste=ste, rho_ratio=rho_ratio, T_wall=T_wall, T_melt=T_melt))


def thermocapillary_channel(nx=512, ny=256, h=None, T_h=20.0, T_c=10.0, T_0=4.0, T_ref=10.0,
                            sigma_ref=2.5e-2, mu=0.2, lam=0.2, ma=0.1, steps=20000,
                            width=INTERFACE_WIDTH, sigma_T=None) -> dict:
    """Marangoni convection of two superposed fluids (Sec. 4.1, second test and
    Appendix A): lower fluid (phi = 1) for y < h, upper fluid above, equal
    rho = Cp = 1, mu and lambda; bottom wall T_h + T_0 cos(2 pi x / L), top T_c;
    sigma(T) = sigma_ref + sigma_T (T - T_ref) with sigma_T < 0 fixed by
    Ma = rho Cp |sigma_T| T_0 h / (mu lambda) unless ``sigma_T`` is given (the
    paper's own Appendix-A runs use sigma_T = -5e-4); no phase change, no solute.
    The temperature starts from the conduction profile between the walls."""
    if h is None:
        h = ny // 2
    x, y = _coords(nx, ny)
    d = (h - 0.5) - y
    phi = tanh_profile(d, width)
    Htot = float(ny)
    T = T_h + (T_c - T_h) * (y + 0.5) / Htot
    C = np.zeros_like(phi)
    if sigma_T is None:
        sigma_T = -ma * mu * lam / (1.0 * 1.0 * T_0 * h)
    p = base_params(rho_l=1.0, rho_s=1.0, rho_g=1.0, mu_l=mu, mu_s=mu, mu_g=mu, lam_l=lam,
                    lam_s=lam, lam_g=lam, cp_l=1.0, cp_s=1.0, cp_g=1.0, latent=0.0,
                    sigma0=sigma_ref, sigma_T=sigma_T, T_ref=T_ref, phase_change_on=0,
                    fs_modulated_st=1, eps=width / (2.0 * math.sqrt(2.0)))
    g = grid(nx, ny, WALL_DIRICHLET_T, WALL_DIRICHLET_T, T_bottom=T_h, T_top=T_c,
             T_bottom_amp=T_0, T_bottom_modes=1)
    return dict(name="thermocapillary_channel_%dx%d" % (nx, ny), grid=g, params=p,
                fields=_fields(phi, T, C), steps=steps,
                meta=dict(h=h, H=ny - h, T_h=T_h, T_c=T_c, T_0=T_0, sigma_T=sigma_T, mu=mu, lam=lam))


def sessile_droplet(nx=512, ny=512, radius=100.0, rho_ratio=0.9, rho_g=0.001, ste=0.1, c0=0.05,
                    ma_T=10.0, ma_C=10.0, k_p=0.5, D_l=0.05, D_s=0.005, sigma0=0.01,
                    T_wall=-1.0, lam=0.3, nu=0.1, steps=None, perturb=0.0, seed=0, theta=90.0) -> dict:
    """Binary droplet freezing on a cold substrate (Sec. 4.4): a circular cap of
    radius R on the bottom wall with contact angle theta (degrees; 90 is the
    half-disc centred on the wall, the only angle of the paper's Sec. 4.4 case),
    solute C0 in the droplet, T_0 = T_m = 0, bottom wall Dirichlet T_wall with
    that wettability, top adiabatic.
    Thermal Marangoni: |sigma_T| from Ma_T = |sigma_T| (T_m - T_w) R / (mu_l alpha_l);
    solutal: |sigma_c| from Ma_C = |sigma_c| C0 R / (mu_l D_l); sigma falls with T
    and with C (Sec. 4.4).  ``perturb`` adds seeded uniform noise of that
    amplitude to T everywhere (upwards, so that no cell starts below T_m) and
    to C inside the droplet."""
    x, y = _coords(nx, ny)
    # the wall is at y = -1/2; the centre of a cap with contact angle theta lies
    # R cos(theta) below it
    xc, yc = nx / 2.0, -0.5 - (0.0 if theta == 90.0 else radius * math.cos(math.radians(theta)))
    d = radius - np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    phi = tanh_profile(d)
    T = np.zeros_like(phi)
    chi = np.clip(0.5 * (1.0 + phi), 0.0, 1.0)
    C = c0 * chi
    if perturb:
        rng = np.random.default_rng(seed)
        T = T + perturb * rng.uniform(0.0, 1.0, size=T.shape)
        C = C + perturb * chi * rng.uniform(-1.0, 1.0, size=C.shape)
    p = base_params(rho_s=rho_ratio, lam_l=lam, lam_s=lam, k_p=k_p, D_l=D_l, D_s=D_s,
                    sigma0=sigma0, latent=1.0 * (0.0 - T_wall) / ste, T_ref=0.0, c_ref=c0)
    p = gas_properties(p, rho_g, nu=nu)
    alpha_l = p["lam_l"] / (p["rho_l"] * p["cp_l"])
    p["sigma_T"] = -ma_T * p["mu_l"] * alpha_l / ((0.0 - T_wall) * radius) if ma_T else 0.0
    p["sigma_c"] = -ma_C * p["mu_l"] * D_l / (c0 * radius) if (ma_C and c0) else 0.0
    g = grid(nx, ny, WALL_DIRICHLET_T, WALL_ADIABATIC, T_bottom=T_wall, theta_bottom=theta)
    return dict(name="sessile_droplet_%dx%d" % (nx, ny), grid=g, params=p,
                fields=_fields(phi, T, C), steps=steps,
                meta=dict(radius=radius, ste=ste, c0=c0, ma_T=ma_T, ma_C=ma_C, theta=theta))


def parity_droplet(nx=128, ny=128, rho_g=0.1, seed=0, steps=100) -> dict:
    """Parity case: a 128x128 version of the sessile droplet with R = 0.3 nx,
    Marangoni stresses on, solute on, seeded +-1e-3 noise on T and on C in the
    droplet so that every term of the step is exercised within 100 steps."""
    w = sessile_droplet(nx=nx, ny=ny, radius=0.3 * nx, rho_g=rho_g, perturb=1e-3, seed=seed)
    w["name"] = "parity_droplet_%dx%d" % (nx, ny)
    w["steps"] = steps
    return w


def impurity_front(nx=4096, ny=4096, radius=200.0, rho_ratio_impurity=2.0, c0=0.05, ma=10.0,
                   ste=0.1, rho_ratio=0.9, T_wall=-1.0, lam=0.3, k_p=0.5, D_l=0.05, D_s=0.005,
                   sigma0=0.01, center=None, steps=1000) -> dict:
    """Planar freezing front from the cold bottom wall into a binary liquid
    (C0) that holds an insoluble circular impurity (the phi = -1 phase) of
    radius ``radius`` with rho_i / rho_l = 2 and lambda_i = lambda_l, centred
    at (nx/2, ny/4); Marangoni stresses at the impurity interface with
    Ma_T = Ma_C = ``ma`` as in ``sessile_droplet``; top wall adiabatic."""
    x, y = _coords(nx, ny)
    if center is None:
        center = (nx / 2.0, ny / 4.0)
    d = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2) - radius
    phi = tanh_profile(d)
    T = np.zeros_like(phi)
    chi = np.clip(0.5 * (1.0 + phi), 0.0, 1.0)
    C = c0 * chi
    p = base_params(rho_s=rho_ratio, lam_l=lam, lam_s=lam, k_p=k_p, D_l=D_l, D_s=D_s,
                    sigma0=sigma0, latent=1.0 * (0.0 - T_wall) / ste, T_ref=0.0, c_ref=c0)
    rho_i = rho_ratio_impurity * p["rho_l"]
    p = gas_properties(p, rho_i, lam_ratio=1.0)
    alpha_l = p["lam_l"] / (p["rho_l"] * p["cp_l"])
    p["sigma_T"] = -ma * p["mu_l"] * alpha_l / ((0.0 - T_wall) * radius)
    p["sigma_c"] = -ma * p["mu_l"] * D_l / (c0 * radius)
    g = grid(nx, ny, WALL_DIRICHLET_T, WALL_ADIABATIC, T_bottom=T_wall)
    return dict(name="impurity_front_%dx%d" % (nx, ny), grid=g, params=p,
                fields=_fields(phi, T, C), steps=steps,
                meta=dict(radius=radius, c0=c0, ma=ma, center=center))


def static_droplet(nx=96, ny=96, radius=20.0, sigma=0.01, rho_g=1.0, steps=4000) -> dict:
    """Static droplet in the middle of the box, no phase change, no solute,
    uniform temperature, constant surface tension (Laplace test)."""
    x, y = _coords(nx, ny)
    d = radius - np.sqrt((x - (nx - 1) / 2.0) ** 2 + (y - (ny - 1) / 2.0) ** 2)
    phi = tanh_profile(d)
    T = np.zeros_like(phi)
    C = np.zeros_like(phi)
    p = base_params(sigma0=sigma, phase_change_on=0, latent=0.0)
    p = gas_properties(p, rho_g, lam_ratio=1.0)
    g = grid(nx, ny, WALL_ADIABATIC, WALL_ADIABATIC)
    return dict(name="static_droplet_%dx%d" % (nx, ny), grid=g, params=p,
                fields=_fields(phi, T, C), steps=steps, meta=dict(radius=radius, sigma=sigma))


def wetting_droplet(nx=80, ny=40, radius=16.0, theta_wall=60.0, theta0=90.0, sigma=0.01, steps=6000) -> dict:
    """A droplet relaxing on a wall of contact angle theta_wall from a circular
    cap of angle theta0: equal densities, no phase change, no solute, uniform
    temperature, adiabatic walls; its equilibrium is a circular cap of angle
    theta_wall (no gravity)."""
    x, y = _coords(nx, ny)
    yc = -0.5 - (0.0 if theta0 == 90.0 else radius * math.cos(math.radians(theta0)))
    d = radius - np.sqrt((x - nx / 2.0) ** 2 + (y - yc) ** 2)
    phi = tanh_profile(d)
    z = np.zeros_like(phi)
    p = base_params(sigma0=sigma, phase_change_on=0, latent=0.0)
    p = gas_properties(p, 1.0, lam_ratio=1.0)
    g = grid(nx, ny, WALL_ADIABATIC, WALL_ADIABATIC, theta_bottom=theta_wall)
    return dict(name="wetting_droplet_%dx%d_%g" % (nx, ny, theta_wall), grid=g, params=p, fields=_fields(phi, z, z),
                steps=steps, meta=dict(radius=radius, theta_wall=theta_wall, theta0=theta0))


def liquid_bridge(nx=72, ny=48, half_width=14.0, theta_bottom=60.0, theta_top=45.0, c0=0.05, rho_g=0.1,
                  T_wall=-1.0, T_top=0.5, ste=0.1, perturb=1e-3, seed=7, steps=100) -> dict:
    """A binary liquid column spanning the channel from wall to wall (|x - x_c|
    < half_width, x_c the middle of the lattice), so that its interface meets
    both walls: bottom wall Dirichlet T_wall (freezing) with contact angle
    theta_bottom, top wall Dirichlet T_top with theta_top; the sessile
    droplet's properties (rho_s / rho_l 0.9, k_p 0.5, D_l 0.05, D_s 0.005,
    sigma0 0.01) with fixed sigma_T = -1e-3 and sigma_c = -2e-2; seeded
    uniform noise of amplitude ``perturb`` on T (upwards) and, relative, on C."""
    x, y = _coords(nx, ny)
    d = half_width - np.abs(x - (nx - 1) / 2.0)
    phi = tanh_profile(d)
    rng = np.random.default_rng(seed)
    T = perturb * rng.uniform(0.0, 1.0, size=phi.shape)
    C = np.where(phi > 0, c0, 0.0) * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=phi.shape))
    p = base_params(rho_s=0.9, T_sol=0.0, T_liq=0.0, latent=1.0 * (0.0 - T_wall) / ste, k_p=0.5, D_l=0.05,
                    D_s=0.005, sigma0=0.01, sigma_T=-1e-3, sigma_c=-2e-2, T_ref=0.0, c_ref=c0)
    p = gas_properties(p, rho_g)
    g = grid(nx, ny, WALL_DIRICHLET_T, WALL_DIRICHLET_T, T_bottom=T_wall, T_top=T_top,
             theta_bottom=theta_bottom, theta_top=theta_top)
    return dict(name="liquid_bridge_%dx%d" % (nx, ny), grid=g, params=p, fields=_fields(phi, T, C), steps=steps,
                meta=dict(half_width=half_width, theta_bottom=theta_bottom, theta_top=theta_top, c0=c0))


def droplet_sweep(n=256, seed=20251109, side_min=128, side_max=512, rho_g=0.1, steps=1000,
                  theta_range=(60.0, 120.0)) -> list:
    """A parameter sweep of independent freezing sessile droplets (the batched
    workload): square lattices with side uniform in [side_min, side_max],
    radius uniform in [0.2, 0.35] of the side, Stefan number uniform in
    [0.05, 0.5], Ma_T = Ma_C uniform in [0, 50], initial solute uniform in
    [0, 0.1], contact angle uniform in theta_range (degrees; None keeps 90),
    all drawn from numpy's default_rng(seed); gas density ratio 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.integers(side_min, side_max + 1))
        radius = float(rng.uniform(0.2, 0.35)) * side
        ste = float(rng.uniform(0.05, 0.5))
        ma = float(rng.uniform(0.0, 50.0))
        c0 = float(rng.uniform(0.0, 0.1))
        theta = 90.0 if theta_range is None else float(rng.uniform(*theta_range))
        w = sessile_droplet(nx=side, ny=side, radius=radius, rho_g=rho_g, ste=ste, c0=c0, ma_T=ma, ma_C=ma,
                            theta=theta)
        w["name"] = "sweep_%03d_%d" % (i, side)
        w["steps"] = steps
        w["meta"].update(side=side)
        out.append(w)
    return out


def thermocapillary_migration(radius=20.0, T_c=0.0, T_h=32.0, sigma0=2.5e-3, sigma_T=-1e-4, mu=0.2, lam=0.2,
                              steps=None) -> dict:
    """Droplet migration driven by a surface-tension gradient (Sec. 4.1, first
    benchmark): a droplet of radius R at the centre of an 8R x 16R box, equal
    density, heat capacity, viscosity and conductivity in both phases, walls at
    T_c (bottom) and T_h (top) with the linear profile between them,
    sigma = sigma0 + sigma_T (T - T_c), no phase change and no solute.  The
    steady migration velocity of Young, Goldstein and Block for these values is
    U_YGB = 2 U / ((2 + 3 mu_l/mu_h)(2 + alpha_l/alpha_h)) with
    U = -sigma_T grad T R / mu_h (R = 20: 1.333e-4)."""
    nx, ny = int(round(8 * radius)), int(round(16 * radius))
    x, y = _coords(nx, ny)
    d = radius - np.sqrt((x - (nx - 1) / 2.0) ** 2 + (y - (ny - 1) / 2.0) ** 2)
    phi = tanh_profile(d)
    # linear profile between the walls at y = -1/2 (T_c) and y = ny - 1/2 (T_h)
    T = T_c + (T_h - T_c) * (y + 0.5) / ny
    C = np.zeros_like(phi)
    p = base_params(mu_l=mu, mu_s=mu, mu_g=mu, lam_l=lam, lam_s=lam, lam_g=lam, sigma0=sigma0, sigma_T=sigma_T,
                    T_ref=T_c, phase_change_on=0, latent=0.0)
    g = grid(nx, ny, WALL_DIRICHLET_T, WALL_DIRICHLET_T, T_bottom=T_c, T_top=T_h)
    grad_T = (T_h - T_c) / ny
    U = -sigma_T * grad_T * radius / mu
    u_ygb = 2.0 * U / ((2.0 + 3.0) * (2.0 + 1.0))
    return dict(name="thermocapillary_migration_%dx%d" % (nx, ny), grid=g, params=p, fields=_fields(phi, T, C),
                steps=steps, meta=dict(radius=radius, grad_T=grad_T, U=U, U_YGB=u_ygb))


WORKLOADS = {
    "thermocapillary_migration": thermocapillary_migration,
    "wetting_droplet": wetting_droplet,
    "liquid_bridge": liquid_bridge,
    "stefan_layer": stefan_layer,
    "thermocapillary_channel": thermocapillary_channel,
    "sessile_droplet": sessile_droplet,
    "parity_droplet": parity_droplet,
    "impurity_front": impurity_front,
    "static_droplet": static_droplet,
}


def make(name: str, **kw) -> dict:
    return WORKLOADS[name](**kw)
