"""The learned surrogate's coupling with the LB solver on the GPU:
lb_set_fields, the packing / update / check kernels of libcno against numpy,
the interface-width check against the closed form of the tanh profile, and
the jump-with-fallback stepper (a rejected jump leaves the LB result bitwise
unchanged; an accepted one installs the prediction)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_09422_gb300 import workloads as W  # noqa: E402

FIELDS = ("phi", "T", "fs", "C", "ux", "uy", "p")


@pytest.fixture(scope="module", autouse=True)
def _libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09422_gb300 import _build, cno, lbfreeze
    _build.build()
    lbfreeze.load()
    cno.load()


def _f32(w):
    return {k: np.asarray(v, np.float32) for k, v in w["fields"].items()}


def test_set_fields_without_fs_and_p_equals_creation():
    from paper_2511_09422_gb300 import lbfreeze
    w = W.parity_droplet(nx=96, ny=80)
    f = _f32(w)
    a = lbfreeze.Solver(w["grid"], w["params"], f)
    b = lbfreeze.Solver(w["grid"], w["params"], f)
    b.step(7)
    b.set_fields({"phi": f["phi"], "T": f["T"], "C": f["C"], "ux": f["ux"], "uy": f["uy"]})
    a.step(20)
    b.step(20)
    fa, fb = a.fields(), b.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()


def test_set_fields_round_trip_after_a_run():
    """get_fields -> set_fields -> get_fields reproduces the conserved and
    thermal fields; velocity and pressure differ by the force half-terms."""
    from paper_2511_09422_gb300 import lbfreeze
    w = W.parity_droplet(nx=128, ny=96)
    s = lbfreeze.Solver(w["grid"], w["params"], _f32(w))
    s.step(300)
    f1 = s.fields()
    r1 = s.reduce()
    s.set_fields(f1)
    f2 = s.fields()
    r2 = s.reduce()
    for k in ("phi", "T", "fs", "C"):
        scale = max(float(np.abs(f1[k]).max()), 1e-30)
        assert float(np.abs(f2[k] - f1[k]).max()) <= 1e-4 * scale, (k, float(np.abs(f2[k] - f1[k]).max()))
    assert abs(r2[0] - r1[0]) <= 1e-6 * abs(r1[0])        # sum phi
    assert abs(r2[3] - r1[3]) <= 1e-5 * max(abs(r1[3]), 1.0)  # sum f_s
    s.step(50)
    assert np.all(np.isfinite(s.reduce()))
    s.close()


def test_pack_delta_update_kernels_match_numpy():
    from paper_2511_09422_gb300 import cno
    rng = np.random.default_rng(3)
    ny, nx = 24, 40
    cur = [torch.as_tensor(rng.standard_normal((ny, nx)).astype(np.float32)).cuda() for _ in FIELDS]
    nxt = [torch.as_tensor(rng.standard_normal((ny, nx)).astype(np.float32)).cuda() for _ in FIELDS]
    off = rng.standard_normal(7).astype(np.float32)
    isc = rng.uniform(0.5, 2.0, 7).astype(np.float32)
    x = cno.pack_fields(cur, off, isc)
    t = torch.empty((ny, nx, 7), dtype=torch.float32, device="cuda")
    cno.pack_delta(cur, nxt, isc, t)
    out = torch.as_tensor(rng.standard_normal((1, ny, nx, 7)).astype(np.float32)).cuda()
    dst = [torch.empty_like(c) for c in cur]
    cno.apply_update(cur, dst, out, isc)
    band = [torch.empty_like(c) for c in cur]
    cno.apply_update(cur, band, out, isc, phi_band=0.5)
    torch.cuda.synchronize()
    c = np.stack([a.cpu().numpy() for a in cur], -1)
    n = np.stack([a.cpu().numpy() for a in nxt], -1)
    want_x = ((c - off) * isc).astype(np.float32)
    got_x = x[0].float().cpu().numpy()
    assert np.array_equal(got_x[..., :7], torch.as_tensor(want_x).to(torch.bfloat16).float().numpy())
    assert np.all(got_x[..., 7:] == 0)
    assert np.array_equal(t.cpu().numpy(), ((n - c) * isc).astype(np.float32))
    want_u = c.astype(np.float64) + isc.astype(np.float64) * out[0].cpu().numpy().astype(np.float64)
    got_u = np.stack([a.cpu().numpy() for a in dst], -1)
    assert np.all(np.abs(got_u - want_u) <= 2.0 ** -23 * np.abs(want_u) + 1e-30)
    got_b = np.stack([a.cpu().numpy() for a in band], -1)
    outside = np.abs(c[..., 0]) >= 0.5
    assert outside.any() and (~outside).any()
    assert np.array_equal(got_b[..., 0][outside], c[..., 0][outside])
    assert np.array_equal(got_b[..., 0][~outside], got_u[..., 0][~outside])
    assert np.array_equal(got_b[..., 1:], got_u[..., 1:])
    zero = [torch.empty_like(c) for c in cur]
    sc0 = isc.copy()
    sc0[4:] = 0.0
    cno.apply_update(cur, zero, out, sc0)
    got_z = np.stack([a.cpu().numpy() for a in zero], -1)
    assert np.array_equal(got_z[..., 4:], c[..., 4:])          # scale 0: copied
    assert np.array_equal(got_z[..., :4], got_u[..., :4])
    clamped = [torch.empty_like(c) for c in cur]
    lo = [-0.5] * 7
    hi = [0.25] * 7
    cno.apply_update(cur, clamped, out, isc, lo=lo, hi=hi)
    got_c = np.stack([a.cpu().numpy() for a in clamped], -1)
    assert np.array_equal(got_c, np.clip(got_u, -0.5, 0.25).astype(np.float32))


def test_field_checks_match_numpy_and_the_tanh_width():
    from paper_2511_09422_gb300 import cno
    ny, nx = 96, 64
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    phi = np.tanh(2.0 * (40.3 - y) / W.INTERFACE_WIDTH).astype(np.float32)  # flat interface, W = 4
    fs = np.clip(0.5 * (1 + phi), 0, 1).astype(np.float32) * 0.25
    Tf = (np.arange(ny * nx, dtype=np.float32).reshape(ny, nx) * 1e-3 - 1.0).astype(np.float32)
    s = cno.field_checks(torch.as_tensor(phi).cuda(), torch.as_tensor(fs).cuda(), torch.as_tensor(Tf).cuda())
    assert s[5] == float(Tf.min()) and s[6] == float(Tf.max())
    s = s[:5]
    p = phi.astype(np.float64)
    gy = np.empty_like(p)
    gy[1:-1] = 0.5 * (p[2:] - p[:-2])
    gy[0] = p[1] - p[0]
    gy[-1] = p[-1] - p[-2]
    gx = 0.5 * (np.roll(p, -1, 1) - np.roll(p, 1, 1))
    want = (p.sum(), np.clip(0.5 * (1 + p), 0, 1).sum(), fs.astype(np.float64).sum(), (1 - p * p).sum(),
            np.sqrt(gx * gx + gy * gy).sum())
    assert np.allclose(s, want, rtol=1e-12, atol=1e-9)
    width = 2.0 * s[3] / s[4]
    assert abs(width - W.INTERFACE_WIDTH) <= 0.03 * W.INTERFACE_WIDTH, width


def test_enthalpy_sum_matches_the_lb_reduction():
    """sum rho H of the check kernel (mixture rule, latent part rho_l L (chi - f_s))
    on the fields of an LB state equals the LB's own sum of the enthalpy moment."""
    from paper_2511_09422_gb300 import cno, lbfreeze
    w = W.parity_droplet(nx=128, ny=96)
    p = w["params"]
    s = lbfreeze.Solver(w["grid"], p, _f32(w))
    s.step(400)
    F = s.fields(device=True)
    r = s.reduce()
    hc = (p["rho_l"] * p["cp_l"], p["rho_s"] * p["cp_s"], p["rho_g"] * p["cp_g"], p["rho_l"] * p["latent"])
    c = cno.field_checks(F["phi"], F["fs"], F["T"], hc)
    assert abs(c[7] - r[1]) <= 1e-5 * abs(r[1]), (c[7], r[1])
    s.close()


def _tiny_model(seed=0):
    from paper_2511_09422_gb300 import cno, surrogate
    net = cno.Net()
    net.set_params(surrogate.init_params(seed))
    norm = surrogate.Normaliser(np.zeros(7, np.float32), np.ones(7, np.float32), np.full(7, 1e-3, np.float32))
    return net, norm


def test_rejected_jumps_leave_the_lb_result_unchanged():
    from paper_2511_09422_gb300 import lbfreeze, surrogate
    w = W.parity_droplet(nx=128, ny=64)
    net, norm = _tiny_model()
    a = lbfreeze.Solver(w["grid"], w["params"], _f32(w))
    b = lbfreeze.Solver(w["grid"], w["params"], _f32(w))
    st = surrogate.SurrogateStepper(a, net, norm, w["params"], k=20, mass_tol=-1.0)  # every check fails
    st.advance(130)
    b.step(130)
    fa, fb = a.fields(), b.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
    s = st.stats()
    assert s["accepted"] == 0 and s["rejected"] >= 1 and s["chunks"] == 6 and s["lb_chunks"] == 6
    assert a.steps == 130
    net.close()


def test_accepted_jump_installs_the_prediction():
    from paper_2511_09422_gb300 import lbfreeze, surrogate
    w = W.parity_droplet(nx=128, ny=64)
    net, norm = _tiny_model(seed=1)
    s = lbfreeze.Solver(w["grid"], w["params"], _f32(w))
    st = surrogate.SurrogateStepper(s, net, norm, w["params"], k=20, mass_tol=1e9, width_tol=1e9, h_tol=1e30,
                                    slow_only=False)
    st._lb_chunk(measure=True)   # a fresh enthalpy rate, as before any attempt
    assert st.try_jump()
    got = s.fields(device=True)
    for k in ("phi", "C"):
        want = st.pred[k]
        assert float((got[k] - want).abs().max()) <= 1e-4 * max(float(want.abs().max()), 1e-30), k
    # T comes back through the enthalpy inversion, which makes (T, f_s) consistent
    # with the phase diagram: unchanged where the predicted pair already is (liquid,
    # f_s <= 0, above the liquidus T_liq = 0)
    liquid = (st.pred["fs"] <= 0) & (st.pred["T"] > 1e-6)
    assert int(liquid.sum()) > 100
    # on the temperature scale of the case (wall at -1, melting point 0); the
    # latent enthalpy rho_l L ~ 10 sets the FP32 resolution of T to ~1e-6
    dT = (got["T"] - st.pred["T"]).abs()[liquid]
    assert float(dT.max()) <= 1e-5
    s.step(10)
    assert np.all(np.isfinite(s.reduce()))
    net.close()
