"""Wetting and thermocapillary migration on the GPU: parity with the FP64
oracle at contact angles other than 90 degrees, the equilibrium contact angle
of a relaxing droplet (geometry fixes it), and the steady migration velocity
of a droplet in a temperature gradient against the Young-Goldstein-Block
value quoted in Sec. 4.1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import analytic  # noqa: E402
import test_parity_gpu as P  # noqa: E402
from paper_2511_09422_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09422_gb300 import _build, lbfreeze
    _build.build()
    lbfreeze.load()


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_parity_with_contact_angle(oracle_mod, theta):
    w = W.sessile_droplet(nx=96, ny=64, radius=20.0, rho_g=0.1, perturb=1e-3, theta=theta)
    w["grid"]["cos_theta_top"] = float(np.cos(np.radians(180.0 - theta)))
    got, red, want, wred = P._run_pair(oracle_mod, w, 100)
    P._assert_parity(got, want, label="theta %g" % theta)
    P._assert_reduce(red, wred)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_equilibrium_contact_angle(theta):
    from paper_2511_09422_gb300 import lbfreeze
    w = W.wetting_droplet(nx=256, ny=128, radius=40.0, theta_wall=theta)
    s = lbfreeze.Solver(w["grid"], w["params"], P._f32(w))
    s.step(40000)
    got, _, _ = analytic.contact_angle_bottom(s.fields()["phi"].astype(np.float64))
    s.close()
    assert abs(got - theta) <= 1.5, (theta, got)


def test_thermocapillary_migration_velocity():
    """Sec. 4.1: R = 20 in an 8R x 16R box, grad T = 0.1, U_YGB = 1.333e-4; the
    droplet velocity U_r = sum phi u_y / sum phi over phi > 0 settles at U_YGB."""
    from paper_2511_09422_gb300 import lbfreeze
    w = W.thermocapillary_migration()
    u_ygb = w["meta"]["U_YGB"]
    s = lbfreeze.Solver(w["grid"], w["params"], P._f32(w))
    hist = []
    t_ref = w["meta"]["radius"] / w["meta"]["U"]  # R / U
    for k in range(30):
        s.step(4000)
        f = s.fields()
        m = f["phi"] > 0
        hist.append(float((f["phi"][m] * f["uy"][m]).sum() / f["phi"][m].sum()))
    s.close()
    late = np.array(hist[-5:])
    ratio = late / u_ygb
    assert np.all(ratio > 0), hist                      # towards the hot wall (+y)
    assert abs(late[-1] - late[0]) <= 0.02 * u_ygb, hist  # settled
    assert abs(ratio[-1] - 1.0) <= 0.10, (ratio[-1], [h / u_ygb for h in hist], 30 * 4000 / t_ref)
