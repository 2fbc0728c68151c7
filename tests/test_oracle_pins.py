"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form
printed in the paper, a moment identity the LB equilibria and sources must
satisfy to recover the paper's macroscopic equations, an exact property of
the difference schemes, a conservation law of the model, or a value printed
in the paper (tests/golden).  A plausible mistake in any part of the oracle
(dropped term, wrong sign or index, transposed operand) fails at least one.
"""
import math
import os

import numpy as np
import pytest

import analytic as A
from paper_2511_09422_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
CS2 = 1.0 / 3.0


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line)
    return rows


# ------------------------------------------------------------------------------------------
# Difference schemes (end of Sec. 3.4)
# ------------------------------------------------------------------------------------------

def test_stencil_exact_on_quadratics(oracle_mod):
    nx, ny = 12, 10
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    a, b, c, d, e, f = 0.3, -1.2, 0.7, 0.11, -0.05, 0.09
    v = a + b * x + c * y + d * x * x + e * x * y + f * y * y
    g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    gx, gy, lap = oracle_mod.stencil_field(g, v, 0)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    np.testing.assert_allclose(gx[inner], (b + 2 * d * x + e * y)[inner], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gy[inner], (c + e * x + 2 * f * y)[inner], rtol=0, atol=1e-12)
    np.testing.assert_allclose(lap[inner], 2 * d + 2 * f, rtol=0, atol=1e-12)


def test_stencil_wall_ghosts(oracle_mod):
    nx, ny = 8, 6
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    # a field even about the wall y = -1/2: the mirror ghost is its exact extension
    v = (y + 0.5) ** 2
    g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    _, gy, lap = oracle_mod.stencil_field(g, v, 0)
    np.testing.assert_allclose(gy[0], 2 * 0.5, atol=1e-12)
    np.testing.assert_allclose(lap[0], 2.0, atol=1e-12)
    # a temperature linear in y with T = T_w(x) on the bottom wall: the Dirichlet
    # ghost 2 T_w - T is exact; the x-derivative of the cosine is the central difference
    Tb, amp, k = 2.0, 0.5, 2
    g = W.grid(nx, ny, W.WALL_DIRICHLET_T, W.WALL_DIRICHLET_T, T_bottom=Tb, T_top=Tb + 0.3 * ny,
               T_bottom_amp=amp, T_bottom_modes=k)
    wall = Tb + amp * np.cos(2 * np.pi * k * x / nx)
    T = wall + 0.3 * (y + 0.5)
    gx, gy, _ = oracle_mod.stencil_field(g, T, 1)  # bottom row only: the top wall is not consistent
    np.testing.assert_allclose(gy[0], 0.3, atol=1e-12)
    kk = 2 * np.pi * k / nx
    np.testing.assert_allclose(gx[0], -amp * np.sin(kk * x[0]) * np.sin(kk), atol=1e-12)


# ------------------------------------------------------------------------------------------
# Equilibria and sources: the moments that recover the model equations
# ------------------------------------------------------------------------------------------

def _moments(v):
    return v.sum(), (CX * v).sum(), (CY * v).sum(), (CX * CX * v).sum(), (CX * CY * v).sum(), (CY * CY * v).sum()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    p = W.base_params(rho_s=0.9, cp_s=0.8, cp_l=1.3)
    phi, C, rhoH, T, pr = rng.uniform(-1, 1), rng.uniform(0, 0.2), rng.uniform(-2, 12), rng.uniform(-1, 1), rng.uniform(-1e-2, 1e-2)
    ux, uy, rho, rhocp = rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.05), rng.uniform(0.1, 1), rng.uniform(0.5, 2)
    f, g, h, l = oracle_mod.equilibria(p, phi, C, rhoH, T, pr, ux, uy, rho, rhocp)
    rr = p["rho_l"] * 2 * p["cp_s"] * p["cp_l"] / (p["cp_s"] + p["cp_l"])
    # phase field: zeroth phi, first phi u (advective flux of Eq. ACE)
    m = _moments(f)
    np.testing.assert_allclose(m[:3], [phi, phi * ux, phi * uy], atol=1e-14)
    np.testing.assert_allclose(m[3:], [CS2 * phi, 0, CS2 * phi], atol=1e-14)
    # flow: zeroth 0 (pressure-based), first rho u, second p I + rho u u (Eq. NS2)
    m = _moments(g)
    np.testing.assert_allclose(m, [0, rho * ux, rho * uy, pr + rho * ux * ux, rho * ux * uy, pr + rho * uy * uy], atol=1e-14)
    # enthalpy: zeroth rho H, first rho Cp T u (Eq. Tem), second rho_ref Cp_ref T cs2 I + rho Cp T u u
    m = _moments(h)
    np.testing.assert_allclose(m, [rhoH, rhocp * T * ux, rhocp * T * uy, rr * T * CS2 + rhocp * T * ux * ux,
                                   rhocp * T * ux * uy, rr * T * CS2 + rhocp * T * uy * uy], atol=1e-13)
    # solute: zeroth C, first C u (Eq. c)
    m = _moments(l)
    np.testing.assert_allclose(m[:3], [C, C * ux, C * uy], atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_source_moments(oracle_mod, seed):
    rng = np.random.default_rng(10 + seed)
    kw = {k: rng.uniform(-0.1, 0.1) for k in ("dphiux", "dphiuy", "mdot", "S", "Fx", "Fy", "rfx", "rfy", "Ftx",
                                             "Fty", "ux", "uy", "Q", "dCux", "dCuy", "Rx", "Ry")}
    th = rng.uniform(0, 2 * np.pi)
    kw.update(nx=math.cos(th), ny=math.sin(th), phi=rng.uniform(-1, 1), eps=math.sqrt(2.0))
    F, G, H, L = oracle_mod.sources(**kw)
    divu = kw["mdot"]
    kf = (1 - kw["phi"] ** 2) / (math.sqrt(2) * kw["eps"])
    m = _moments(F)
    np.testing.assert_allclose(m[:3], [kw["phi"] * divu, kw["dphiux"] + CS2 * kf * kw["nx"],
                                       kw["dphiuy"] + CS2 * kf * kw["ny"]], atol=1e-14)
    m = _moments(G)
    uFx, uFy = kw["ux"] * kw["Ftx"], kw["uy"] * kw["Fty"]
    np.testing.assert_allclose(m, [kw["S"], kw["Fx"] + kw["rfx"], kw["Fy"] + kw["rfy"],
                                   kw["S"] * CS2 + 2 * uFx, kw["ux"] * kw["Fty"] + kw["uy"] * kw["Ftx"],
                                   kw["S"] * CS2 + 2 * uFy], atol=1e-14)
    m = _moments(H)
    np.testing.assert_allclose(m[:3], [kw["Q"], 0, 0], atol=1e-15)
    m = _moments(L)
    np.testing.assert_allclose(m[:3], [0, kw["dCux"] + CS2 * kw["Rx"], kw["dCuy"] + CS2 * kw["Ry"]], atol=1e-14)


# ------------------------------------------------------------------------------------------
# Enthalpy relation (Eq. Hfl)
# ------------------------------------------------------------------------------------------

def _tf99(oracle_mod, w, params, chunk=50):
    o = oracle_mod.Oracle(w["grid"], params, w["fields"])
    prev = 0.0
    for k in range(1, 400):
        o.step(chunk)
        r = o.reduce()
        frac = r[3] / r[4]
        if frac >= 0.99:
            o.close()
            return chunk * (k - 1) + chunk * (0.99 - prev) / (frac - prev), r
        prev = frac
    raise AssertionError("the droplet did not freeze")


def test_heat_capacity_readings(oracle_mod):
    """The property rule of Sec. 2 lists the heat capacity; the oracle applies
    it to the volumetric rho C_p of each phase (reading R17), not to rho and
    C_p apart.  (1) With C_p = 1 in every phase the two readings are the same
    function, so the runs agree bit for bit: the option changes nothing else
    (a gas density of 0.5 there; with C_p = 1 the gas's rho C_p is that
    density).  (2) On the freezing droplet with (rho C_p)_g = (rho C_p)_l at a
    gas density ratio of 0.1, where the literal product peaks threefold inside
    the liquid-gas interface, the literal reading moves the freezing time by
    5.0e-3 (1404.1 against 1397.1 steps) and the final V*_sl by 1e-6."""
    wu = W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.5, ste=0.15)
    uniform = dict(wu["params"], divu_mode=1, cp_l=1.0, cp_s=1.0, cp_g=1.0)
    runs = []
    for rule in (0, 1):
        o = oracle_mod.Oracle(wu["grid"], dict(uniform, rhocp_rule=rule), wu["fields"])
        o.step(300)
        runs.append(o.fields())
        o.close()
    for k in runs[0]:
        assert np.all(np.isfinite(runs[0][k])), k
        assert np.array_equal(runs[0][k], runs[1][k]), k
    w = W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.1, ste=0.15)
    t0, _ = _tf99(oracle_mod, w, dict(w["params"], divu_mode=1, rhocp_rule=0))
    t1, _ = _tf99(oracle_mod, w, dict(w["params"], divu_mode=1, rhocp_rule=1))
    assert 2e-3 < (t1 - t0) / t0 < 1e-2, (t0, t1)


def test_enthalpy_relation(oracle_mod):
    # a binary alloy with a mushy range, solid and liquid properties different
    p = W.base_params(rho_s=0.9, cp_s=0.7, cp_l=1.2, latent=4.0, T_sol=-0.3, T_liq=0.2)
    p = W.gas_properties(p, 0.1)
    rng = np.random.default_rng(3)
    for _ in range(300):
        T, chi = rng.uniform(-2, 2), rng.uniform(0, 1)
        e = oracle_mod.enthalpy_forward(p, T, chi)
        T2, fs = oracle_mod.enthalpy_invert(p, e, chi)
        assert abs(T2 - T) < 1e-12 and -1e-15 <= fs <= chi + 1e-15
    # Eq. Hfl at chi = 1, written out for the pure phase-change material
    rsHs = p["rho_s"] * p["cp_s"] * p["T_sol"]
    rlHl = p["rho_l"] * (p["cp_l"] * p["T_liq"] + p["latent"])
    for rH in np.linspace(rsHs - 1.5, rlHl + 1.5, 41):
        if rH < rsHs:
            fl, T = 0.0, rH / (p["rho_s"] * p["cp_s"])
        elif rH <= rlHl:
            fl = (rH - rsHs) / (rlHl - rsHs)
            T = p["T_sol"] + fl * (p["T_liq"] - p["T_sol"])
        else:
            fl, T = 1.0, p["T_liq"] + (rH - rlHl) / (p["rho_l"] * p["cp_l"])
        T2, fs = oracle_mod.enthalpy_invert(p, rH, 1.0)
        assert abs(T2 - T) < 1e-12 and abs(fs - (1 - fl)) < 1e-12
    # continuity at the solidus and liquidus enthalpies, for any chi
    for chi in (0.0, 0.3, 1.0):
        for T in (p["T_sol"], p["T_liq"]):
            e = oracle_mod.enthalpy_forward(p, T, chi)
            lo, hi = oracle_mod.enthalpy_invert(p, e - 1e-9, chi), oracle_mod.enthalpy_invert(p, e + 1e-9, chi)
            assert abs(lo[0] - hi[0]) < 1e-7 and abs(lo[1] - hi[1]) < 1e-7
    # the gas never holds solid
    assert oracle_mod.enthalpy_invert(p, -5.0, 0.0)[1] == 0.0


def test_property_rule(oracle_mod):
    # zeta(phi, f_s): liquid (1, 0), solid (1, 1), gas (-1, 0) -- end of Sec. 2
    for (phi, fs, want) in ((1, 0, 2.0), (1, 1, 5.0), (-1, 0, 7.0), (0, 0, 4.5)):
        assert abs(oracle_mod.zeta(phi, fs, 2.0, 5.0, 7.0) - want) < 1e-15


# ------------------------------------------------------------------------------------------
# Conservation laws
# ------------------------------------------------------------------------------------------

def test_phase_field_conservation(oracle_mod):
    """Without phase change sum(phi) is conserved to round-off (Sec. 2, 'strictly
    preserve mass conservation'), in a flow driven by surface tension."""
    w = W.static_droplet(nx=40, ny=36, radius=10, rho_g=0.1)
    # off-centre, so that the walls and the periodic seam see the flow
    w["fields"]["phi"] = W.tanh_profile(10 - np.hypot(np.arange(40)[None, :] - 7.3, np.arange(36)[:, None] - 12.1))
    o = oracle_mod.Oracle(w["grid"], w["params"], w["fields"])
    s0 = o.reduce()[0]
    o.step(300)
    s1 = o.reduce()[0]
    f = o.fields()
    assert np.abs(f["ux"]).max() > 1e-6  # a real flow
    assert abs(s1 - s0) <= 1e-12 * np.abs(f["phi"]).sum()


def test_solute_conservation(oracle_mod):
    """Eq. c is conservative and every wall is no-flux: sum(C) is constant, here
    through freezing, Marangoni flow and volume change."""
    w = W.parity_droplet(nx=48, ny=40)
    o = oracle_mod.Oracle(w["grid"], w["params"], w["fields"])
    c0 = o.reduce()[2]
    o.step(200)
    r = o.reduce()
    assert r[3] > 1.0  # something froze
    assert abs(r[2] - c0) <= 1e-11 * abs(c0)


# ------------------------------------------------------------------------------------------
# Analytic solutions printed in the paper
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ste", [0.1, 0.2])
def test_neumann_front(oracle_mod, ste):
    """Sec. 4.2: s(t) = 2 kappa sqrt(alpha_s t), here without volume change
    (rho_s = rho_l) and T_0 = T_m, kappa from the transcendental equation."""
    w = W.stefan_layer(nx=2, ny=160, h0=128, ste=ste, rho_ratio=1.0, rho_g=0.1)
    o = oracle_mod.Oracle(w["grid"], w["params"], w["fields"])
    kappa = A.neumann_kappa(ste)
    alpha_s = w["params"]["lam_s"] / (w["params"]["rho_s"] * w["params"]["cp_s"])
    for t in (1000, 2500):
        o.step(t - o.steps)
        s = o.reduce()[5]
        assert abs(s / A.neumann_front(t, kappa, alpha_s) - 1) < 4e-3, (t, s)


def test_neumann_superheated(oracle_mod):
    """Same problem with a superheated liquid (T_0 > T_m): the second term of the
    transcendental equation is active (alpha_r = 1, rho_r = 1)."""
    ny = 400
    w = W.stefan_layer(nx=2, ny=ny, h0=380, ste=0.2, rho_ratio=1.0, rho_g=0.1)
    w["fields"]["T"][:] = 0.3
    o = oracle_mod.Oracle(w["grid"], w["params"], w["fields"])
    p = w["params"]
    kappa = A.neumann_kappa(0.2, T0=0.3, Tm=0.0, Tw=-1.0, lam_s=p["lam_s"], lam_l=p["lam_l"])
    assert kappa < A.neumann_kappa(0.2)
    o.step(4000)
    s = o.reduce()[5]
    assert abs(s / A.neumann_front(4000, kappa, p["lam_s"]) - 1) < 1e-2, s



def test_solute_diffuses_at_the_solid_diffusivity(oracle_mod):
    """Inside the solid (f_s = 1) the effective diffusivity D_e / k_eff of
    Sec. 3.4 is k_p D_s / k_p = D_s: a Gaussian pulse spreads with variance
    s0^2 + 2 D_s t per direction, as in the liquid pin, not with k_p D_s."""
    nx = ny = 64
    s0, Ds, steps = 4.0, 0.02, 400
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    C = 0.05 * np.exp(-((x - nx / 2) ** 2 + (y - ny / 2) ** 2) / (2 * s0 * s0))
    p = W.base_params(D_l=0.05, D_s=Ds, k_p=0.5, sigma0=0.0, latent=10.0, T_sol=0.0, T_liq=0.0)
    g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    z = np.zeros_like(C)
    o = oracle_mod.Oracle(g, p, dict(phi=np.ones_like(C), T=np.full_like(C, -1.0), C=C, ux=z, uy=z.copy()))
    o.step(steps)
    f = o.fields()
    assert f["fs"].min() == 1.0
    m = f["C"].sum()
    xc = (f["C"] * x).sum() / m
    var_x = (f["C"] * (x - xc) ** 2).sum() / m
    want = s0 * s0 + 2 * Ds * steps
    assert abs(var_x / want - 1) < 0.01, (var_x, want)


def test_solute_partition_at_a_stationary_front(oracle_mod):
    """A column frozen below its middle and liquid above (walls at T = -1 and
    +1, linear steady temperature, so the front stays put): the solute
    relaxes until the pseudo-potential C / k_eff is uniform, i.e. C_solid /
    C_liquid = k_p, through the flux correction of R in Sec. 3.4.  The
    one-cell front leaves a discretisation error of 7 % (0.467 for k_p = 0.5);
    without the correction the ratio is 1, with its sign flipped 2.1."""
    nx, ny, kp = 4, 64, 0.5
    y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))[1]
    p = W.base_params(D_l=0.05, D_s=0.05, k_p=kp, sigma0=0.0, latent=10.0, T_sol=0.0, T_liq=0.0)
    g = W.grid(nx, ny, W.WALL_DIRICHLET_T, W.WALL_DIRICHLET_T, T_bottom=-1.0, T_top=1.0)
    z = np.zeros((ny, nx))
    o = oracle_mod.Oracle(g, p, dict(phi=np.ones((ny, nx)), T=-1.0 + 2.0 * (y + 0.5) / ny,
                                     C=np.full((ny, nx), 0.05), ux=z, uy=z.copy()))
    o.step(40000)
    f = o.fields()
    assert f["fs"][:, 0].sum() == 32.0                         # the front has not moved
    assert abs(f["C"].sum() / (0.05 * nx * ny) - 1) < 1e-10     # solute conserved
    ratio = f["C"][4:24].mean() / f["C"][40:60].mean()
    assert abs(ratio / kp - 1) < 0.1, ratio

def test_binary_solidification(oracle_mod):
    """Sec. 4.3 without gas (phi = 1 everywhere; the model reduces to the classical
    enthalpy method for a binary material): front, temperature and the solute
    rejected at the front against the closed forms."""
    ny, kp, C0, Dl, al = 300, 0.5, 0.1, 0.05, 0.3
    p = W.base_params(rho_s=1.0, lam_l=al, lam_s=al, k_p=kp, D_l=Dl, D_s=0.0, latent=10.0,
                      T_sol=0.0, T_liq=0.0, sigma0=0.0)
    g = W.grid(2, ny, W.WALL_DIRICHLET_T, W.WALL_ADIABATIC, T_bottom=-1.0)
    o = oracle_mod.Oracle(g, p, dict(phi=np.ones((ny, 2)), T=np.zeros((ny, 2)), C=np.full((ny, 2), C0)))
    k = A.binary_stefan_k(1.0, 1.0, 10.0, 0.0, -1.0, 0.0, al, al)
    t = 4000
    o.step(t)
    f, r = o.fields(), o.reduce()
    y = np.arange(ny) + 0.5
    Ta, Ca, s = A.binary_stefan_fields(y, t, k, -1.0, 0.0, 0.0, C0, kp, al, al, Dl)
    assert abs(r[5] / s - 1) < 3e-3
    assert np.abs(f["T"][:, 0] - Ta).max() < 0.03
    assert abs(r[2] / 2 - C0 * ny) < 1e-10 * C0 * ny
    # solute is rejected: depleted solid, enriched liquid ahead of the front,
    # far field at C0.  The enthalpy method resolves the front by one cell,
    # which smears the partition: the solid and the liquid peak are compared
    # with a tolerance of 30% of the closed-form depletion and enrichment.
    mid = int(s / 2)
    assert abs(f["C"][mid, 0] - Ca[mid]) < 0.3 * (C0 - Ca[mid])
    liq = y > s + 3
    assert np.abs(f["C"][liq, 0] - Ca[liq]).max() < 0.3 * (Ca.max() - C0)
    assert abs(f["C"][-1, 0] - C0) < 1e-6


def test_laplace_jump(oracle_mod):
    """Static droplet: the capillary force of Eq. Fs with delta = alpha |grad phi|^2,
    alpha = 3 sqrt(2) eps / 4, gives the 2-D Laplace jump sigma / R.  The
    isotropic gradient integrates |grad phi|^2 of the W = 4 profile to 0.939 of
    its exact value, so that is the jump to expect on this lattice."""
    N, R, sig = 48, 12.0, 0.01
    w = W.static_droplet(nx=N, ny=N, radius=R, rho_g=1.0, sigma=sig)
    o = oracle_mod.Oracle(w["grid"], w["params"], w["fields"])
    o.step(6000)
    f = o.fields()
    c = N // 2
    dp = f["p"][c - 2:c + 2, c - 2:c + 2].mean() - f["p"][:4, :4].mean()
    j = np.arange(-40, 40) + 0.5
    ph = np.tanh(j / 2.0)
    d = (np.roll(ph, -1) - np.roll(ph, 1)) / 2.0
    discrete = (3 * math.sqrt(2) * W.EPS / 4 * d[2:-2] ** 2).sum()
    assert 0.93 < discrete < 0.945
    assert abs(dp / (sig / R) / discrete - 1) < 0.03, dp / (sig / R)


def test_stratified_marangoni(oracle_mod):
    """Appendix A: layered thermocapillary flow, converged at L = 80, h = H = 20.
    The temperature matches the closed form closely; the velocity within the
    smearing of a 4-cell diffuse interface over a 20-cell layer."""
    L, h = 80, 20
    w = W.thermocapillary_channel(nx=L, ny=2 * h, h=h)
    m = w["meta"]
    o = oracle_mod.Oracle(w["grid"], w["params"], w["fields"])
    o.step(4000)
    f = o.fields()
    y = np.arange(2 * h) + 0.5 - h
    xq = L // 4
    T, ux, _, Um = A.stratified_marangoni(xq, y, L, h, h, m["T_h"], m["T_c"], m["T_0"], m["sigma_T"], m["mu"])
    assert np.abs(f["T"][:, xq] - T).max() < 1e-3
    err = f["ux"][:, xq] - ux
    assert np.sqrt((err ** 2).mean()) < 0.1 * Um
    lobe = h // 3
    assert 0.8 < f["ux"][lobe, xq] / ux[lobe] < 1.02
    T, _, uy, _ = A.stratified_marangoni(0, y, L, h, h, m["T_h"], m["T_c"], m["T_0"], m["sigma_T"], m["mu"])
    assert np.abs(f["uy"][:, 0] - uy).max() < 0.1 * Um
    # flow goes from the hot to the cold part of the interface
    assert f["ux"][h, L // 4] > 0 and f["ux"][h, 3 * L // 4] < 0


def test_heat_conduction_decay(oracle_mod):
    """Enthalpy set alone (no phase change, no flow): T(y, 0) = sin(pi (y+1/2)/ny)
    between two Dirichlet walls at T = 0 decays as exp(-alpha (pi/ny)^2 t); the
    two-relaxation-time collision with 1/tau_bar + 1/tau_tilde = 2 keeps the
    anti-bounce-back walls exactly half-way."""
    ny, lam = 40, 0.25
    p = W.base_params(lam_l=lam, lam_s=lam, lam_g=lam, phase_change_on=0, latent=0.0, sigma0=0.0)
    g = W.grid(2, ny, W.WALL_DIRICHLET_T, W.WALL_DIRICHLET_T)
    y = np.arange(ny) + 0.5
    T0 = np.repeat(np.sin(np.pi * y / ny)[:, None], 2, axis=1)
    o = oracle_mod.Oracle(g, p, dict(phi=np.ones((ny, 2)), T=T0, C=np.zeros((ny, 2))))
    t = 1500
    o.step(t)
    T = o.fields()["T"][:, 0]
    want = np.exp(-lam * (np.pi / ny) ** 2 * t) * np.sin(np.pi * y / ny)
    assert np.abs(T - want).max() < 2e-3 * want.max()


def test_poiseuille(oracle_mod):
    """Flow set alone: body force rho g between half-way bounce-back walls gives
    the parabola g (y+1/2)(ny-y-1/2) / (2 nu)."""
    ny, nu, gx = 24, 0.1, 1e-6
    p = W.base_params(phase_change_on=0, latent=0.0, sigma0=0.0, gx=gx)
    g = W.grid(2, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    o = oracle_mod.Oracle(g, p, dict(phi=np.ones((ny, 2)), T=np.zeros((ny, 2)), C=np.zeros((ny, 2))))
    o.step(6000)
    u = o.fields()["ux"][:, 0]
    want = A.poiseuille(np.arange(ny), ny, gx, nu)
    assert np.abs(u - want).max() < 5e-3 * want.max()



def test_transverse_gravity_leaves_the_shear_flow_unchanged(oracle_mod):
    """A body force across the channel (g_y) is balanced by the hydrostatic
    pressure it builds, so the Poiseuille flow along the channel must not
    change.  In the flow source of Sec. 3.2 the force enters through the
    effective force F~ = F - grad p + ..., whose cross terms with u would
    otherwise shear the flow: dropping grad p from F~ changes the profile by
    4 % at g_y = -3e-3; with it the change is 0.2 %."""
    nx, ny, gx = 4, 32, 1e-5
    def profile(gy):
        p = W.base_params(sigma0=0.0, gx=gx, gy=gy, phase_change_on=0, latent=0.0)
        g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
        z = np.zeros((ny, nx))
        o = oracle_mod.Oracle(g, p, dict(phi=np.ones((ny, nx)), T=z, C=z.copy(), ux=z.copy(), uy=z.copy()))
        o.step(20000)
        return o.fields()["ux"][:, 0]
    u0, u1 = profile(0.0), profile(-3e-3)
    assert np.abs(u0 / A.poiseuille(np.arange(ny), ny, gx, 0.1) - 1).max() < 0.01
    assert np.abs(u1 / u0 - 1).max() < 5e-3

def test_solid_drag(oracle_mod):
    """The solid-liquid interaction force f = f_s (0 - u*) holds a frozen region
    under the same body force that drives a Poiseuille flow.  In a uniform
    solid (f_s = 1) the printed rules rho u* = sum c_i g_i + F/2, u = u* + f/2
    and the first moment F + rho f of the source G_i have the steady state
    sum c_i g_i = F/2, so u* = F/rho and u = F/(2 rho) exactly: away from the
    walls the velocity is g_x / 2."""
    ny, gx = 24, 1e-6
    p = W.base_params(sigma0=0.0, gx=gx)
    g = W.grid(2, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    o = oracle_mod.Oracle(g, p, dict(phi=np.ones((ny, 2)), T=np.full((ny, 2), -0.5), C=np.zeros((ny, 2))))
    o.step(3000)
    f = o.fields()
    assert f["fs"].min() > 1 - 1e-9
    assert np.abs(f["ux"]).max() < 2 * gx
    assert np.abs(f["ux"][8:16] / gx - 0.5).max() < 1e-6


def test_no_solid_reduction(oracle_mod):
    """With every cell far above the melting point the phase-change model must
    reduce to the plain two-phase model (Sec. 2, reduction consistency): no
    solid, mdot = 0, and the same phase field, velocity and pressure.  (The
    temperature is not compared: the latent enthalpy that the liquid holds is
    not advected by Eq. Tem, whose flux is rho Cp T u, so where the interface
    moves T differs from a run without latent heat.)"""
    w = W.static_droplet(nx=32, ny=32, radius=9, rho_g=0.1)
    w["fields"]["T"][:] = 5.0
    w["grid"]["bc_bottom"] = W.WALL_ADIABATIC
    a = dict(w["params"], phase_change_on=1, latent=3.0, T_sol=-1.0, T_liq=-1.0)
    b = dict(w["params"], phase_change_on=0)
    oa = oracle_mod.Oracle(w["grid"], a, w["fields"])
    ob = oracle_mod.Oracle(w["grid"], b, w["fields"])
    oa.step(200)
    ob.step(200)
    fa, fb = oa.fields(), ob.fields()
    assert fa["fs"].max() == 0.0
    for k in ("phi", "ux", "uy", "p"):
        assert np.array_equal(fa[k], fb[k]), k



@pytest.mark.parametrize("rho_top", [1.0, 0.5, 0.1])
def test_hydrostatic_pressure_under_gravity(oracle_mod, rho_top):
    """Two layers at rest between adiabatic walls under the body force
    F_b = rho g (g is not printed; it is zero unless set): at steady state
    dp/dy = rho g in each layer, rho_l = 1 below and rho_top above, without
    surface tension.  A short, viscous column (32 rows, nu = 0.3) damps the
    start-up sound waves within the run."""
    nx, ny, h, gy = 8, 32, 16, -1e-5
    y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))[1]
    phi = W.tanh_profile((h - 0.5) - y)
    z = np.zeros_like(phi)
    p = W.gas_properties(W.base_params(phase_change_on=0, latent=0.0, gy=gy, sigma0=0.0), rho_top, nu=0.3,
                         lam_ratio=1.0)
    g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    o = oracle_mod.Oracle(g, p, dict(phi=phi, T=z, C=z.copy(), ux=z.copy(), uy=z.copy()))
    o.step(6000)
    f = o.fields()
    prof = f["p"].mean(axis=1)
    slope_low = np.polyfit(np.arange(3, 11), prof[3:11], 1)[0]
    slope_high = np.polyfit(np.arange(21, 29), prof[21:29], 1)[0]
    assert abs(slope_low / (p["rho_l"] * gy) - 1) < 0.01, slope_low
    assert abs(slope_high / (rho_top * gy) - 1) < 0.01, slope_high
    assert np.sqrt(f["ux"] ** 2 + f["uy"] ** 2).max() < 1e-5

def test_table1_final_height(oracle_mod):
    """Table 1 (tests/golden): a film freezes completely in a closed box and its
    final height is h_0 rho_l / rho_s by mass conservation.  In a closed box the
    expansion can only compress the gas; the phase field follows that only
    when its div u source is the velocity divergence (divu_mode = 1).  The
    paper's own errors reach 7e-3; this lattice (a 16-cell film, 4-cell
    interface, gas density 0.1) lands within 2.5%, with the right sign."""
    rows = [list(map(float, r.split())) for r in _golden("table1_final_height.txt")]
    for rr, analytic, *_ in rows:
        assert abs(analytic - 1.0 / rr) < 1e-3
    h0 = 16
    for rr in (0.8, 0.9, 1.2):
        w = W.stefan_layer(nx=2, ny=3 * h0, h0=h0, rho_ratio=rr, rho_g=0.1, ste=0.2)
        o = oracle_mod.Oracle(w["grid"], dict(w["params"], divu_mode=1), w["fields"])
        for _ in range(20):
            o.step(500)
            r = o.reduce()
            if r[3] >= 0.999 * r[4]:
                break
        hf = r[5] / h0
        analytic = [a for (x, a, *_) in rows if abs(x - rr) < 1e-9][0]
        assert abs(hf / analytic - 1) < 0.025, (rr, hf)
        assert (hf - 1) * (1 - rr) > 0



@pytest.mark.parametrize("mobility", [0.1, 0.05, 0.2])
def test_droplet_expansion_end_state(oracle_mod, mobility):
    """Sec. 4.4 (tests/golden): a freezing droplet with rho_s / rho_l = 0.9 ends
    at V*_sl = 1.1107, 3.7e-4 from the mass-conservation value 1 / 0.9.  The
    oracle with the velocity-divergence source (divu_mode = 1, as for Table 1)
    reaches 1 / 0.9 within 1e-3 on a 48 x 40 lattice (R = 12, Ste = 0.15,
    nu = 0.1 in every phase as in all workloads here) once the droplet is
    solid; with the model value mdot (divu_mode = 0) the closed box's gas takes
    up most of the expansion and V*_sl stays near 1.04.  The end state moves
    with the viscosity (1.120 at nu = 0.05, 1.100 at 0.2): part of the
    expansion goes into compressing the gas, by an amount the viscous damping
    of the start-up flow sets, so this pins the configuration at nu = 0.1.
    It fails when the pressure's G_0 term, whose relaxation time the paper
    leaves unnamed (taken as tau_g), takes tau = 1, 1/2, 2 tau_g or is dropped.
    The mobility M = 0.05 and 0.2 (tau_f = 0.65 and 1.1, tau_g = 0.8) tells
    tau_g from the phase field's tau_f there: with tau_f the end state misses
    1 / 0.9 by -7e-3 and +1.5e-2, with tau_g by 2e-4 at most."""
    kv = dict(r.split("=") for r in _golden("printed_numbers.txt"))
    kv = {k.strip(): float(v) for k, v in kv.items()}
    assert abs(kv["droplet_final_Vsl"] * 0.9 - 1) <= kv["droplet_final_Vsl_error"] + 1e-5
    w = W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.1, ste=0.15)
    o = oracle_mod.Oracle(w["grid"], dict(w["params"], divu_mode=1, mobility=mobility), w["fields"])
    for _ in range(20):
        o.step(250)
        r = o.reduce()
        if r[3] >= 0.999 * r[4]:
            break
    assert r[3] >= 0.999 * r[4]
    o.step(500)
    r = o.reduce()
    assert abs(r[7] * 0.9 - 1) < 1e-3, r[7]
    assert abs(r[6] - r[7]) < 1e-6  # all of the material is solid


def test_temperature_origin_invariance(oracle_mod):
    """With the same volumetric heat capacity in every phase, the enthalpy
    equation of Sec. 3.3, d(rho H)/dt + div(rho Cp T u) = div(lambda grad T)
    + rho Cp T div u, does not change when a constant is added to every
    temperature (melting point, wall, initial field): the extra terms
    c [d(rho Cp)/dt + div(rho Cp u) - rho Cp div u] vanish.  So a film that
    freezes while it expands (rho_s / rho_l = 0.8, Cp_s = 1.25) must reach the
    same solid height whatever the origin of T.  Discretely this holds with
    the velocity-divergence source (divu_mode = 1), whose div u is the one the
    advection sees: within 2e-3 for shifts of +5 and -3 (measured 9e-4).  It
    fails by 2-8 % when the source Q is dropped, when the rho H correction
    Q/2 is dropped, or when the source is weighted with the antisymmetric
    time; with mdot as div u (divu_mode = 0) the height moves by 3 %."""
    def height(shift):
        w = W.stefan_layer(nx=4, ny=96, h0=48, ste=0.2, rho_ratio=0.8)
        p = dict(w["params"], T_sol=shift, T_liq=shift, cp_s=1.0 / 0.8, divu_mode=1)
        g = dict(w["grid"], T_bottom=w["grid"]["T_bottom"] + shift)
        f = dict(w["fields"], T=w["fields"]["T"] + shift)
        o = oracle_mod.Oracle(g, p, f)
        o.step(2000)
        return o.reduce()[3] / 4
    h0 = height(0.0)
    assert h0 > 10
    for shift in (5.0, -3.0):
        assert abs(height(shift) / h0 - 1) < 2e-3, shift

def test_printed_ygb_velocity():
    """The migration speed printed in Sec. 4.1 follows from the YGB formula."""
    kv = dict(r.split("=") for r in _golden("printed_numbers.txt"))
    kv = {k.strip(): float(v) for k, v in kv.items()}
    u = A.ygb_velocity(-1e-4, 0.1, 20.0, 0.2, 0.2, 0.2, 0.2)
    assert abs(u / kv["ygb_velocity"] - 1) < 1e-3


@pytest.mark.parametrize("divu_mode,bound", [(0, 1e-6), (1, 5e-6)])
def test_parity_cases_are_well_conditioned(oracle_mod, divu_mode, bound):
    """The oracle moves by less than ``bound`` (relative, per field) after 100
    steps when the inputs of the droplet parity case are perturbed by 1e-7,
    i.e. FP32 round-off is not amplified past the 1e-5 parity bar.  This holds
    because the interface normal is regularised as
    grad phi / sqrt(|grad phi|^2 + 1e-6); with 1e-12 the same perturbation
    grows to 1e-3.  With the model value mdot as div u (divu_mode = 0) the
    response stays below 1e-6; with the lagged velocity divergence
    (divu_mode = 1) the velocity's own perturbation enters phi through the
    source w_i phi div u and the moment correction, and phi moves by 2.3e-6,
    still a quarter of the bar."""
    w = W.parity_droplet(nx=128, ny=128)
    p = dict(w["params"], divu_mode=divu_mode)
    f = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in w["fields"].items()}
    rng = np.random.default_rng(5)
    g = {k: v * (1 + 1e-7 * rng.uniform(-1, 1, size=v.shape)) for k, v in f.items()}
    a = oracle_mod.Oracle(w["grid"], p, f)
    b = oracle_mod.Oracle(w["grid"], p, g)
    a.step(100)
    b.step(100)
    fa, fb = a.fields(), b.fields()
    speed = np.sqrt(fa["ux"] ** 2 + fa["uy"] ** 2).max()
    for k in ("phi", "T", "fs", "C", "ux", "uy", "p"):
        scale = speed if k in ("ux", "uy") else np.abs(fa[k]).max()
        assert np.abs(fa[k] - fb[k]).max() / scale < bound, k


@pytest.mark.parametrize("divu_mode", [0, 1])
def test_end_of_run_observables_are_well_conditioned(oracle_mod, divu_mode):
    """The end-of-run quantities compared with the GPU are stable under a 1e-7
    perturbation of the initial temperature: the mean solid height of the
    film-freezing workload after 2000 steps and the solid volume of a frozen
    droplet move by < 1e-4 (relative).
    The solid height on the single centre column depends on the reading of
    div u.  With the lagged velocity divergence (divu_mode = 1) it is as well
    conditioned as the sums (measured 6e-8 and 3e-9).  With the model value
    mdot (divu_mode = 0) it is not: the expanding film pushes the liquid-gas
    interface while the phase field does not see the gas being compressed,
    the interface decelerates and x-perturbations grow (a Rayleigh-Taylor-type
    mode), so the column height moves by about 3e-3."""
    def pair(w, steps):
        w["params"] = dict(w["params"], divu_mode=divu_mode)
        f = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in w["fields"].items()}
        g = {k: v.copy() for k, v in f.items()}
        g["T"] = g["T"] + 1e-7 * np.random.default_rng(5).uniform(0.0, 1.0, size=g["T"].shape)
        a = oracle_mod.Oracle(w["grid"], w["params"], f)
        b = oracle_mod.Oracle(w["grid"], w["params"], g)
        a.step(steps)
        b.step(steps)
        return a.reduce(), b.reduce()

    ra, rb = pair(W.stefan_layer(nx=64, ny=256), 2000)
    assert abs(ra[3] - rb[3]) <= 1e-4 * ra[3], (ra[3], rb[3])
    if divu_mode == 1:
        assert abs(ra[5] - rb[5]) <= 1e-6 * ra[5], (ra[5], rb[5])
    else:
        assert abs(ra[5] - rb[5]) > 1e-4 * ra[5]  # the single-column height is the sensitive one
    ra, rb = pair(W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.1, ste=0.2), 1324)
    assert abs(ra[6] - rb[6]) <= 1e-4 * ra[6], (ra[6], rb[6])
    if divu_mode == 1:
        assert abs(ra[5] - rb[5]) <= 1e-6 * ra[5], (ra[5], rb[5])


def test_reported_fields_carry_the_enthalpy(oracle_mod):
    """With div u the lagged velocity divergence (divu_mode = 1), phi is known
    before the enthalpy relation, and the material fraction chi = clamp((1 +
    phi)/2) of Eq. Hfl (the chi-weighted reading) is that of the reported phi,
    as in the property rule.  So every cell's enthalpy rho H is the mixture
    rule of the reported fields, T (f_s (rho Cp)_s + (chi - f_s) (rho Cp)_l +
    (1 - chi) (rho Cp)_g) + rho_l L (chi - f_s), to round-off (each branch of
    Eq. Hfl with T_s = T_l satisfies it exactly).  Taking chi from sum f_i
    instead, while phi carries the div u correction, breaks it by about
    rho_l L phi div u / 4 in the interface."""
    w = W.parity_droplet(nx=64, ny=48)
    p = w["params"]
    assert p["divu_mode"] == 1 and p["T_sol"] == p["T_liq"]
    o = oracle_mod.Oracle(w["grid"], p, w["fields"])
    o.step(300)
    f = o.fields()
    chi = np.clip(0.5 * (1.0 + f["phi"]), 0.0, 1.0)
    rcp_l, rcp_s, rcp_g = p["rho_l"] * p["cp_l"], p["rho_s"] * p["cp_s"], p["rho_g"] * p["cp_g"]
    e = f["T"] * (f["fs"] * rcp_s + (chi - f["fs"]) * rcp_l + (1.0 - chi) * rcp_g) + p["rho_l"] * p["latent"] * (chi - f["fs"])
    interface = np.abs(f["phi"]) < 0.9
    assert interface.sum() > 50
    np.testing.assert_allclose(e, f["rhoH"], rtol=0, atol=1e-12 * np.abs(f["rhoH"]).max())


def test_phase_field_follows_an_accelerating_flow(oracle_mod):
    """The time-derivative term of F_i (Sec. 3.1), w_i c_i . d_t(phi u) / cs2,
    removes the error -(tau_f - 1/2) d_t(phi u) that the lattice's second-order
    expansion leaves in the phase-field flux.  A slab of the phi = 1 phase
    (interfaces normal to x, periodic x) in a fluid of equal density, at rest
    and accelerated from t = 0 by a uniform body force g along x, moves with
    the core flow: far from the walls u(t) = g t, and the interface position
    must follow X(t) - X(0) = integral u dt.  Without the term it lags by
    (tau_f - 1/2) u(t) (4.5e-2 cells here, tau_f = 1.4, u = 0.05); with it the
    offset stays within a fifth of that (measured 2.4e-3).  No surface tension,
    no phase change."""
    nx, ny, mob, g = 64, 64, 0.3, 2.5e-4
    x, y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    phi = W.tanh_profile(16.0 - np.abs(x - 31.5))
    z = np.zeros_like(phi)
    p = W.base_params(phase_change_on=0, latent=0.0, sigma0=0.0, mobility=mob, gx=g)
    o = oracle_mod.Oracle(W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC), p,
                          dict(phi=phi, T=z, C=z.copy(), ux=z.copy(), uy=z.copy()))
    rows = slice(ny // 2 - 2, ny // 2 + 2)

    def centre(f):  # phase of the first Fourier mode of phi along x, middle rows
        c = np.sum(f["phi"][rows].mean(axis=0) * np.exp(-2j * np.pi * np.arange(nx) / nx))
        return -np.angle(c) * nx / (2 * np.pi)

    f = o.fields()
    x0, u_prev, travel = centre(f), f["ux"][rows].mean(), 0.0
    for _ in range(200):
        o.step(1)
        f = o.fields()
        u = f["ux"][rows].mean()
        travel += 0.5 * (u + u_prev)  # trapezoid: exact for the linear u(t)
        u_prev = u
    assert abs(u - 200 * g) < 1e-2 * 200 * g  # the core accelerates freely
    moved = ((centre(f) - x0 + nx / 2) % nx) - nx / 2
    lag = (3 * mob) * u  # (tau_f - 1/2) u
    assert abs(moved - travel) < 0.2 * lag, (moved, travel, lag)


def test_dirichlet_wall_of_short_wavelength(oracle_mod):
    """Anti-bounce-back at a Dirichlet wall (Sec. 4.5) whose temperature varies
    along it, T_w = A cos(k x), with 16 cells per period: steady conduction in
    a resting liquid reaches the closed form A cos(k x) exp(-k (y + 1/2)) (wall
    at y = -1/2, adiabatic top far away), row by row, within 0.5 % (measured
    0.39 %, the O(k^2) error k^2/24).  T_w sampled at each link's own crossing
    point (x +- 1/2 for the diagonal links) instead of the foot of the cell
    lowers the effective wall amplitude by a further (1 - cos(k/2))/3 and
    misses by 1.03 %; a dropped factor 2 or a mirror ghost fails by far more."""
    period, ny, lam = 16, 48, 0.3
    nx, k = 2 * period, 2 * np.pi / period
    phi, z = np.ones((ny, nx)), np.zeros((ny, nx))
    p = W.base_params(phase_change_on=0, latent=0.0, sigma0=0.0, lam_l=lam, lam_s=lam, lam_g=lam)
    g = W.grid(nx, ny, W.WALL_DIRICHLET_T, W.WALL_ADIABATIC, T_bottom=0.0, T_bottom_amp=1.0, T_bottom_modes=2)
    o = oracle_mod.Oracle(g, p, dict(phi=phi, T=z.copy(), C=z.copy(), ux=z.copy(), uy=z.copy()))
    o.step(3000)
    T = o.fields()["T"]
    xs = np.arange(nx)
    for y in range(6):
        amp = 2.0 / nx * np.sum(T[y] * np.cos(k * xs))
        closed = np.exp(-k * (y + 0.5))
        assert abs(amp / closed - 1) < 5e-3, (y, amp, closed)
        assert abs(T[y].mean()) < 1e-9  # the mean stays at the wall's mean
