"""Pins of the oracle's D2Q5 option for the phase-field and solute sets
(lb_params.lattice_fl = 1) against closed forms: a Gaussian solute pulse in a
uniform liquid at rest spreads with variance s0^2 + 2 D t per direction (the
diffusivity D_e = c_s^2 (tau_l - 1/2) of Sec. 3.4, the same on both lattices);
sum phi and sum C are conserved exactly; and on a freezing droplet the two
lattices agree to the truncation error of the same equations."""
import numpy as np
import pytest

import oracle
from paper_2511_09422_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build_oracle()


def _gaussian_case(lattice, nx=64, ny=64, s0=4.0, D=0.05):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    r2 = (x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2
    C = 0.05 * np.exp(-r2 / (2 * s0 * s0))
    phi = np.ones_like(C)
    T = np.ones_like(C)
    p = W.base_params(D_l=D, D_s=D, phase_change_on=0, latent=0.0, sigma0=0.0)
    p["lattice_fl"] = lattice
    g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC)
    return g, p, dict(phi=phi, T=T, C=C, ux=np.zeros_like(C), uy=np.zeros_like(C)), x, y


@pytest.mark.parametrize("lattice", [0, 1])
def test_gaussian_solute_spreads_at_the_model_diffusivity(lattice):
    s0, D, steps = 4.0, 0.05, 400
    g, p, f, x, y = _gaussian_case(lattice, s0=s0, D=D)
    o = oracle.Oracle(g, p, f)
    o.step(steps)
    C = o.fields()["C"]
    m0 = C.sum()
    xc = (C * x).sum() / m0
    var_x = (C * (x - xc) ** 2).sum() / m0
    var_y = (C * (y - (C * y).sum() / m0) ** 2).sum() / m0
    want = s0 * s0 + 2 * D * steps
    assert abs(var_x - want) <= 0.01 * want, (lattice, var_x, want)
    assert abs(var_y - want) <= 0.01 * want, (lattice, var_y, want)
    assert abs(m0 - f["C"].sum()) <= 1e-12 * f["C"].sum()


def test_d2q5_conserves_phi_and_solute_on_a_droplet():
    """Without phase change and with div u the model value mdot = 0
    (divu_mode = 0), sum phi and sum C are conserved to round-off."""
    w = W.parity_droplet(nx=64, ny=48)
    p = dict(w["params"], phase_change_on=0, lattice_fl=1, divu_mode=0)
    o = oracle.Oracle(w["grid"], p, w["fields"])
    s0 = o.reduce()
    o.step(150)
    s1 = o.reduce()
    n = 64 * 48
    assert abs(s1[0] - s0[0]) <= 1e-10 * n   # sum phi
    assert abs(s1[2] - s0[2]) <= 1e-10 * n   # sum C


def test_d2q5_and_d2q9_agree_on_a_freezing_droplet():
    w = W.parity_droplet(nx=64, ny=48)
    a = oracle.Oracle(w["grid"], w["params"], w["fields"])
    b = oracle.Oracle(w["grid"], dict(w["params"], lattice_fl=1), w["fields"])
    a.step(200)
    b.step(200)
    fa, fb = a.fields(), b.fields()
    assert not np.array_equal(fa["phi"], fb["phi"])           # the option is in effect
    assert float(np.abs(fa["phi"] - fb["phi"]).max()) <= 2e-2
    assert float(np.abs(fa["C"] - fb["C"]).max()) <= 2e-2 * float(np.abs(fa["C"]).max())
    assert float(np.abs(fa["T"] - fb["T"]).max()) <= 1e-2
