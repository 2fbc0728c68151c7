"""Pins of the oracle's wetting condition (contact angle at a wall) against
geometry: a two-dimensional droplet without gravity relaxes to a circular cap,
and the cap's contact angle is fixed by the circle alone (cos theta = distance
from the wall to the centre over the radius).  Starting from the half-disc
(90 degrees), the oracle's droplet must settle at the wall's angle; a 90-degree
wall must leave the half-disc where it is; and the ghost rule's sign and
coefficient match the derivative of the tanh profile at the contact line."""
import math

import numpy as np
import pytest

import analytic
import oracle
from paper_2511_09422_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build_oracle()


@pytest.mark.parametrize("lattice_fl", [0, 1], ids=["D2Q9", "D2Q5"])
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_droplet_relaxes_to_the_wall_contact_angle(theta, lattice_fl):
    """The wall condition acts on the stencils of phi, so it holds with either
    lattice of the phase-field set."""
    w = W.wetting_droplet(theta_wall=theta)
    o = oracle.Oracle(w["grid"], dict(w["params"], lattice_fl=lattice_fl), w["fields"])
    o.step(9000)
    got, radius, _ = analytic.contact_angle_bottom(o.fields()["phi"])
    assert abs(got - theta) <= 2.0, (theta, got)
    # mass of the droplet is conserved while it spreads or beads up
    assert abs(o.reduce()[0] - float(np.sum(w["fields"]["phi"]))) <= 1e-9 * w["fields"]["phi"].size



def _bridge(theta_b, theta_t, nx=96, ny=40, half=18.0, sigma=0.01):
    """A liquid column |x - x_c| < half spanning the channel between two
    adiabatic walls of contact angles theta_b and theta_t: equal densities,
    no phase change, no solute, uniform temperature."""
    x, y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    phi = W.tanh_profile(half - np.abs(x - (nx - 1) / 2.0))
    z = np.zeros_like(phi)
    p = W.gas_properties(W.base_params(sigma0=sigma, phase_change_on=0, latent=0.0), 1.0, lam_ratio=1.0)
    g = W.grid(nx, ny, W.WALL_ADIABATIC, W.WALL_ADIABATIC, theta_bottom=theta_b, theta_top=theta_t)
    return g, p, dict(phi=phi, T=z, C=z.copy(), ux=z.copy(), uy=z.copy())


@pytest.mark.parametrize("theta_b,theta_t", [(60.0, 60.0), (120.0, 120.0), (45.0, 75.0)])
def test_liquid_bridge_laplace_pressure(theta_b, theta_t):
    """Between parallel walls a distance H apart, each free interface of a
    liquid bridge settles at a circular arc that meets the walls at their
    angles, so its curvature is (cos theta_b + cos theta_t) / H and the
    liquid's pressure differs from the gas's by -sigma (cos theta_b +
    cos theta_t) / H (below it for wetting walls, above it for non-wetting
    ones).  As in the static-droplet Laplace pin, the isotropic gradient
    integrates the capillary force of the W = 4 profile to 0.939 of its
    exact value, which is the jump to expect on the lattice."""
    nx, ny, sigma = 96, 40, 0.01
    g, p, f = _bridge(theta_b, theta_t, nx=nx, ny=ny, sigma=sigma)
    o = oracle.Oracle(g, p, f)
    o.step(8000)
    P = o.fields()["p"]
    xc = (nx - 1) // 2
    p_liquid = P[8:32, xc - 3:xc + 4].mean()
    p_gas = np.concatenate([P[8:32, :4], P[8:32, -4:]], axis=1).mean()
    j = np.arange(-40, 40) + 0.5
    d = np.gradient(np.tanh(j / 2.0))
    discrete = float((3 * math.sqrt(2) * W.EPS / 4 * d[2:-2] ** 2).sum())
    want = -sigma * (math.cos(math.radians(theta_b)) + math.cos(math.radians(theta_t))) / ny * discrete
    assert abs((p_liquid - p_gas) / want - 1.0) < 0.03, (p_liquid - p_gas, want)

def test_ninety_degree_wall_keeps_the_half_disc():
    w = W.wetting_droplet(theta_wall=90.0)
    assert w["grid"]["cos_theta_bottom"] == 0.0
    o = oracle.Oracle(w["grid"], w["params"], w["fields"])
    o.step(3000)
    got, _, _ = analytic.contact_angle_bottom(o.fields()["phi"])
    assert abs(got - 90.0) <= 0.2, got


def test_ghost_rule_matches_the_tanh_profile_at_the_wall():
    """phi = tanh(d / (sqrt 2 eps)) for a straight interface through the contact
    point at angle theta (inside phi > 0): its normal derivative at the wall
    equals -cos(theta) (1 - phi^2) / (sqrt 2 eps), the rule the ghost encodes."""
    eps = W.EPS
    for theta in (30.0, 60.0, 120.0, 150.0):
        th = math.radians(theta)
        m = (math.sin(th), -math.cos(th))  # unit normal into the phi > 0 wedge

        def phi(x, y):
            return math.tanh((x * m[0] + y * m[1]) / (math.sqrt(2.0) * eps))

        for x in (-2.0, -0.7, 0.0, 0.9, 2.5):
            h = 1e-5
            dn = (phi(x, h) - phi(x, -h)) / (2 * h)  # wall normal +y, wall at y = 0
            p = phi(x, 0.0)
            assert abs(dn - (-math.cos(th) * (1 - p * p) / (math.sqrt(2.0) * eps))) <= 1e-8
