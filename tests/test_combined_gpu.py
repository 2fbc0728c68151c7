"""Options of the step combined on the GPU, each against the FP64 oracle run
with the same options: wetting walls with the D2Q5 phase-field and solute
sets and with half-precision storage, a liquid column whose interface meets
two Dirichlet walls of different contact angles while it freezes, and the
edge shapes of the row and strip layout under D2Q5 and half storage.  The
bars are those of the single options: 1e-5 per field for FP32 D2Q9 storage,
the same 1e-5 for D2Q5 f and l (test_d2q5_gpu), and the half-storage bar of
test_fp16_gpu.  Every case is well conditioned: the oracle itself moves by
less than 1e-6 when its inputs are perturbed by 1e-7."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_d2q5_gpu as Q  # noqa: E402
import test_fp16_gpu as H  # noqa: E402
import test_parity_gpu as P  # noqa: E402
from paper_2511_09422_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09422_gb300 import _build, lbfreeze
    _build.build()
    lbfreeze.load()


def _wet_droplet(theta):
    w = W.sessile_droplet(nx=96, ny=64, radius=20.0, rho_g=0.1, perturb=1e-3, theta=theta)
    w["grid"]["cos_theta_top"] = float(np.cos(np.radians(180.0 - theta)))
    return w


def _check(got, want, tol, label):
    errs = P._rel_errors(got, want)
    bad = {k: v for k, v in errs.items() if not v <= (tol[k] if isinstance(tol, dict) else tol)}
    assert not bad, (label, bad, errs)
    assert all(np.isfinite(got[k]).all() for k in P.FIELDS), label


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_d2q5_with_contact_angle(oracle_mod, theta):
    w = _wet_droplet(theta)
    got, red, want, wred = P._run_pair(oracle_mod, w, 100, params=dict(w["params"], lattice_fl=Q.Q5))
    _check(got, want, Q.TOL_Q5, "D2Q5, theta %g" % theta)
    P._assert_reduce(red, wred)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_half_storage_with_contact_angle(oracle_mod, theta):
    w = _wet_droplet(theta)
    got, red, want, wred = P._run_pair(oracle_mod, w, 100, params=dict(w["params"], pop_storage=H.F16))
    _check(got, want, H.FIELD_TOL, "FP16, theta %g" % theta)


@pytest.mark.parametrize("theta_b,theta_t", [(60.0, 45.0), (30.0, 150.0)])
def test_liquid_bridge_between_wetting_walls(oracle_mod, theta_b, theta_t):
    """The column freezes from the cold bottom wall while both walls impose
    their contact angles and the top wall its temperature."""
    w = W.liquid_bridge(theta_bottom=theta_b, theta_top=theta_t)
    got, red, want, wred = P._run_pair(oracle_mod, w, 100)
    P._assert_parity(got, want, label="bridge %g/%g" % (theta_b, theta_t))
    P._assert_reduce(red, wred)
    assert want["fs"].max() > 0.1  # solid has formed at the wetting wall


def test_liquid_bridge_d2q5(oracle_mod):
    w = W.liquid_bridge()
    got, red, want, wred = P._run_pair(oracle_mod, w, 100, params=dict(w["params"], lattice_fl=Q.Q5))
    _check(got, want, Q.TOL_Q5, "bridge D2Q5")
    P._assert_reduce(red, wred)


@pytest.mark.parametrize("shape", P.EDGE_SHAPES)
def test_d2q5_edge_shapes(oracle_mod, shape):
    w = P.edge_workload(*shape)
    got, red, want, wred = P._run_pair(oracle_mod, w, 30, params=dict(w["params"], lattice_fl=Q.Q5))
    _check(got, want, Q.TOL_Q5, "D2Q5 %s" % (shape,))


@pytest.mark.parametrize("form", H.HALF_FORMS)
@pytest.mark.parametrize("shape", P.EDGE_SHAPES)
def test_half_storage_edge_shapes(oracle_mod, shape, form):
    w = P.edge_workload(*shape)
    got, red, want, wred = P._run_pair(oracle_mod, w, 30, params=dict(w["params"], pop_storage=form))
    _check(got, want, H.FIELD_TOL, "half storage %d %s" % (form, shape))


def test_batch_of_wetting_bridges_equals_lone_lattices():
    """Instances with different contact angles (and shapes) step bit for bit
    like lone lattices, with either lattice of the phase-field and solute sets."""
    from paper_2511_09422_gb300 import lbfreeze
    for lattice in (0, Q.Q5):
        ws = [W.liquid_bridge(nx=72, ny=48, theta_bottom=60.0, theta_top=45.0),
              W.liquid_bridge(nx=95, ny=61, half_width=20.0, theta_bottom=120.0, theta_top=90.0),
              W.liquid_bridge(nx=40, ny=37, half_width=8.0, theta_bottom=30.0, theta_top=150.0)]
        for w in ws:
            w["params"] = dict(w["params"], lattice_fl=lattice)
            w["fields"] = P._f32(w)
        b = lbfreeze.Batch(ws)
        b.step(21)
        for i, w in enumerate(ws):
            s = lbfreeze.Solver(w["grid"], w["params"], w["fields"])
            s.step(21)
            want = s.fields()
            got = b.instance(i).fields()
            for k in P.FIELDS:
                assert np.array_equal(got[k], want[k]), (lattice, i, k)
            s.close()
        b.close()
