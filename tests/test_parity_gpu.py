"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Bar (per field, after the stated number of steps): max |gpu - oracle|
divided by the field's scale <= 1e-5.  The scale is max |oracle| for phi,
f_s, C and p; for the temperature it is the temperature range of the problem
(oracle field and Dirichlet wall temperatures), since T has an arbitrary
origin; for u_x and u_y it is the largest speed the oracle reaches during the
compared run (after 1 step or at the end), since a decaying transient would
otherwise divide a fixed round-off by a vanishing speed.  The GPU computes in
FP32 (round-off 6e-8 per operation) and stores the populations as deviations
from lagged references.  Every case here is well conditioned: the oracle
itself moves by less than 1e-6 when its inputs are perturbed by 1e-7
(tests/test_oracle_pins.py checks this for the droplet case), so FP32
round-off is not amplified past the bar.  Both sides start from the same
float32 initial fields.
"""
import os

import numpy as np
import pytest

from paper_2511_09422_gb300 import lbfreeze
from paper_2511_09422_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("phi", "T", "fs", "C", "ux", "uy", "p")
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_09422_gb300 import _build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    lbfreeze.load()


def _f32(w):
    return {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}


def _speed(f):
    return float(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2).max())


def _wall_temperatures(grid):
    out = []
    if grid.get("bc_bottom") == W.WALL_DIRICHLET_T:
        a = abs(grid.get("T_bottom_amp", 0.0))
        out += [grid["T_bottom"] - a, grid["T_bottom"] + a]
    if grid.get("bc_top") == W.WALL_DIRICHLET_T:
        out.append(grid["T_top"])
    return out


def _run_pair(oracle_mod, w, steps, params=None):
    params = params or w["params"]
    f32 = _f32(w)
    s = lbfreeze.Solver(w["grid"], params, f32)
    s.step(steps)
    got = s.fields()
    red = s.reduce()
    s.close()
    o = oracle_mod.Oracle(w["grid"], params, {k: v.astype(np.float64) for k, v in f32.items()})
    peak = 0.0
    if steps > 1:
        o.step(1)
        peak = _speed(o.fields())
    o.step(steps - o.steps)
    want = o.fields()
    want["_peak_speed"] = max(peak, _speed(want))
    want["_walls"] = _wall_temperatures(w["grid"])
    return got, red, want, o.reduce()


def _rel_errors(got, want):
    """max |gpu - oracle| per field over the field's scale (see the module text)."""
    out = {}
    speed = want.get("_peak_speed", _speed(want))
    tvals = [float(want["T"].min()), float(want["T"].max())] + list(want.get("_walls", []))
    for k in FIELDS:
        if k in ("ux", "uy"):
            scale = speed
        elif k == "T":
            scale = max(tvals) - min(tvals)
        else:
            scale = float(np.abs(want[k]).max())
        diff = float(np.abs(got[k].astype(np.float64) - want[k]).max())
        out[k] = diff / scale if scale > 0 else diff
    return out


def _assert_parity(got, want, tol=TOL, label=""):
    errs = _rel_errors(got, want)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "%s: fields above %.0e: %s (all: %s)" % (label, tol, bad, errs)
    return errs


def _assert_reduce(red, wred):
    # phi, rho H, C, f_s, chi sums: FP32 cells summed in FP64
    for k in range(5):
        assert abs(red[k] - wred[k]) <= 1e-5 * max(abs(wred[k]), 1.0), (k, red, wred)
    assert abs(red[5] - wred[5]) <= 1e-4 * max(abs(wred[5]), 1.0)


CASES = [
    ("parity_droplet_128", lambda: W.parity_droplet(nx=128, ny=128), 100),
    ("ragged_droplet_37x29", lambda: W.parity_droplet(nx=37, ny=29), 100),
    ("ragged_droplet_97x71", lambda: W.parity_droplet(nx=97, ny=71, seed=3), 100),
    ("stefan_layer_64x256", lambda: W.stefan_layer(nx=64, ny=256), 100),
    ("channel_64x32", lambda: W.thermocapillary_channel(nx=64, ny=32, h=16, sigma_T=-5e-4), 100),
    ("impurity_front_160", lambda: W.impurity_front(nx=160, ny=128, radius=20.0), 100),
]


@pytest.mark.parametrize("divu_mode", [0, 1])
@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_parity_100_steps(oracle_mod, name, make, steps, divu_mode):
    """Each case with both readings of div u in the phase-field and enthalpy
    sources: the model value mdot (divu_mode = 0) and the lagged velocity
    divergence (divu_mode = 1, the default of the freezing workloads)."""
    w = make()
    p = dict(w["params"], divu_mode=divu_mode)
    got, red, want, wred = _run_pair(oracle_mod, w, steps, params=p)
    _assert_parity(got, want, label="%s divu_mode %d" % (name, divu_mode))
    _assert_reduce(red, wred)


EDGE_SHAPES = [(1, 40), (2, 17), (31, 1), (5, 3), (30, 30), (31, 31), (60, 61), (61, 5), (240, 36), (121, 37),
               (125, 97)]


def edge_workload(nx, ny):
    """The droplet parity case cut to nx x ny (centred in x), with equal solid
    and liquid density and viscosity."""
    w = W.parity_droplet(nx=max(nx, 8), ny=max(ny, 8))
    w["params"] = dict(w["params"], rho_s=w["params"]["rho_l"], mu_s=w["params"]["mu_l"])
    x0 = (max(nx, 8) - nx) // 2
    for k in w["fields"]:
        w["fields"][k] = np.ascontiguousarray(w["fields"][k][:ny, x0:x0 + nx])
    w["grid"] = dict(w["grid"], nx=nx, ny=ny)
    return w


@pytest.mark.parametrize("divu_mode", [0, 1])
@pytest.mark.parametrize("shape", EDGE_SHAPES)
def test_parity_edge_shapes(oracle_mod, shape, divu_mode):
    """A one-column lattice (x-periodic onto itself), a one-row lattice (both
    walls on the same row), shapes at and just past a 30-column warp strip and
    a 4-strip block, and row counts at the edges of the row layout (2-row
    wall bands, then inner segments, 8 rows long at these sizes): one inner
    row (ny = 5), whole segments only (ny = 36), and a last inner segment of
    1 row (ny = 37) or of 5 rows (ny = 97).
    Equal solid and liquid densities: in a one-row lattice the expansion
    source drives phi far above 1 and makes the case ill-conditioned."""
    w = edge_workload(*shape)
    p = dict(w["params"], divu_mode=divu_mode)
    got, red, want, wred = _run_pair(oracle_mod, w, 30, params=p)
    _assert_parity(got, want, label="%s divu_mode %d" % (shape, divu_mode))


def test_parity_initial_state(oracle_mod):
    """Right after lb_create the fields are those of the initial state.  The
    initial temperature spans only 1e-3 here while the liquid's enthalpy is
    about 10 (latent heat), so T is compared in units of the FP32 spacing of
    that enthalpy (9.5e-7), and the other fields relatively."""
    w = W.parity_droplet(nx=64, ny=48)
    got, red, want, wred = _run_pair(oracle_mod, w, 0)
    errs = _rel_errors(got, want)
    for k in ("phi", "fs", "C", "ux", "uy", "p"):
        assert errs[k] <= TOL, (k, errs)
    assert np.abs(got["T"] - want["T"]).max() <= 4 * 9.5e-7
    np.testing.assert_allclose(got["phi"], _f32(w)["phi"], atol=2e-7)


def test_parity_sinusoidal_wall_and_gravity(oracle_mod):
    w = W.thermocapillary_channel(nx=50, ny=40, h=20, sigma_T=-5e-4)
    p = dict(w["params"], gy=-1e-5)
    got, red, want, wred = _run_pair(oracle_mod, w, 100, params=p)
    _assert_parity(got, want, label="channel+gravity")


def test_parity_unmodulated_surface_force(oracle_mod):
    w = W.parity_droplet(nx=64, ny=64)
    p = dict(w["params"], fs_modulated_st=0)
    got, red, want, wred = _run_pair(oracle_mod, w, 100, params=p)
    _assert_parity(got, want, label="F_s without (1 - f_s)")


def test_parity_binary_mushy_range(oracle_mod):
    """A binary material with T_s < T_l (mushy cells) and different Cp."""
    w = W.parity_droplet(nx=64, ny=48)
    p = dict(w["params"], T_sol=-0.2, T_liq=0.05, cp_s=0.8, latent=5.0)
    got, red, want, wred = _run_pair(oracle_mod, w, 100, params=p)
    _assert_parity(got, want, label="mushy")


def test_parity_full_size_bench_workload(oracle_mod):
    """The benchmark's 4096 x 4096 planar-front / impurity lattice, in the
    launch configuration the benchmark times (div u the lagged velocity
    divergence, the workload's default), a few steps against the oracle on
    every cell."""
    w = W.impurity_front(nx=4096, ny=4096)
    got, red, want, wred = _run_pair(oracle_mod, w, 3)
    _assert_parity(got, want, label="4096^2")
    _assert_reduce(red, wred)


def test_torch_stream_and_device_io(oracle_mod):
    """Inputs and outputs in torch CUDA memory, work on a torch stream."""
    w = W.parity_droplet(nx=48, ny=40)
    f32 = _f32(w)
    dev = {k: torch.from_numpy(v).cuda().contiguous() for k, v in f32.items()}
    stream = torch.cuda.Stream()
    s = lbfreeze.Solver(w["grid"], w["params"], dev, stream=stream)
    with torch.cuda.stream(stream):
        s.step(50)
        out = s.fields(device=True)
    stream.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in f32.items()})
    o.step(1)
    peak = _speed(o.fields())
    o.step(49)
    want = o.fields()
    want["_peak_speed"] = max(peak, _speed(want))
    want["_walls"] = _wall_temperatures(w["grid"])
    _assert_parity(got, want, label="torch I/O")



def test_device_fields_ordered_across_streams():
    """A solver on a stream of its own hands device fields to work on torch's
    current stream, and takes them back, with no synchronisation by the
    caller: after a long queue of steps on the solver's stream, the fields
    read on the current stream, and the state set from tensors made there,
    equal those of a solver on the current stream bit for bit."""
    w = W.parity_droplet(nx=512, ny=512)
    f32 = _f32(w)
    side = torch.cuda.Stream()
    s = lbfreeze.Solver(w["grid"], w["params"], f32, stream=side)
    ref = lbfreeze.Solver(w["grid"], w["params"], f32)
    s.step(300)
    d = s.fields(device=True)
    got = {k: v.cpu().numpy() for k, v in d.items()}   # read on the current stream
    ref.step(300)
    want = ref.fields()
    for k in FIELDS:
        assert np.array_equal(got[k], want[k]), k
    back = {k: (v * 1.0) for k, v in d.items()}         # made on the current stream
    s.set_fields(back)
    del back, d
    ref.set_fields(want)
    s.step(20)
    ref.step(20)
    a, b = s.fields(), ref.fields()
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    s.close()
    ref.close()

def test_checkpoint_resume_bitwise(tmp_path):
    w = W.parity_droplet(nx=64, ny=48)
    f32 = _f32(w)
    a = lbfreeze.Solver(w["grid"], w["params"], f32)
    a.step(40)
    a.save(str(tmp_path / "ck.bin"))
    a.step(40)
    fa = a.fields()
    b = lbfreeze.Solver(w["grid"], w["params"], f32)
    b.load_state(str(tmp_path / "ck.bin"))
    assert b.steps == 40
    b.step(40)
    fb = b.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.reduce(), b.reduce())


def test_repeatable_bitwise():
    w = W.parity_droplet(nx=80, ny=64)
    f32 = _f32(w)
    r = []
    for _ in range(2):
        s = lbfreeze.Solver(w["grid"], w["params"], f32)
        s.step(30)
        r.append((s.fields(), s.reduce()))
        s.close()
    for k in FIELDS:
        assert np.array_equal(r[0][0][k], r[1][0][k])
    assert np.array_equal(r[0][1], r[1][1])


def test_non_finite_input_reported():
    """Fault injection on the host: a NaN in the initial temperature must come
    back as LB_ERR_UNSTABLE from lb_reduce, and the handle stays usable for
    destroy."""
    w = W.parity_droplet(nx=32, ny=32)
    f32 = _f32(w)
    f32["T"][10, 10] = np.nan
    s = lbfreeze.Solver(w["grid"], w["params"], f32)
    s.step(3)
    with pytest.raises(lbfreeze.LbError) as e:
        s.reduce()
    assert e.value.status == lbfreeze.LB_ERR_UNSTABLE
    with pytest.raises(lbfreeze.LbError):
        s.step(1)  # sticky
    s.close()


def test_reduce_matches_oracle_and_v0(oracle_mod):
    w = W.parity_droplet(nx=96, ny=80)
    got, red, want, wred = _run_pair(oracle_mod, w, 100)
    _assert_reduce(red, wred)
    assert abs(red[7] - wred[7]) < 1e-5 and abs(red[6] - wred[6]) < 1e-5


def _freezing_time(step, reduce, max_steps, frac=0.99):
    """First crossing of sum f_s = frac * sum chi, linearly interpolated between
    the two steps that bracket it; returns (t_f, diagnostics at the crossing)."""
    prev = None
    for n in range(1, max_steps + 1):
        step(1)
        r = reduce()
        g1 = r[3] - frac * r[4]
        if g1 >= 0.0:
            if prev is None:
                return float(n), r
            return (n - 1) + (-prev) / (g1 - prev), r
        prev = g1
    raise AssertionError("no full freezing within %d steps" % max_steps)


@pytest.mark.parametrize("divu_mode", [0, 1])
def test_freezing_time_and_final_solid_volume(oracle_mod, divu_mode):
    """A small sessile droplet (R = 12) run to full freezing: the freezing time
    and the solid volume V*_s at the end of the run (20 % past the oracle's
    freezing time) agree with the oracle within 1e-3.  With the lagged velocity
    divergence as div u (divu_mode = 1) the front position -- the solid height
    on the centre column -- is compared too; with mdot (divu_mode = 0) it is
    ill-conditioned in the oracle itself and is not (see
    test_end_of_run_observables_are_well_conditioned)."""
    w = W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.1, ste=0.2)
    w["params"] = dict(w["params"], divu_mode=divu_mode)
    f32 = _f32(w)
    s = lbfreeze.Solver(w["grid"], w["params"], f32)
    tf_gpu, _ = _freezing_time(s.step, s.reduce, 5000)
    o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in f32.items()})
    tf_ora, _ = _freezing_time(o.step, o.reduce, 5000)
    assert abs(tf_gpu - tf_ora) <= 1e-3 * tf_ora, (tf_gpu, tf_ora)
    n_end = int(1.2 * tf_ora) + 1
    s.step(n_end - s.steps)
    o.step(n_end - o.steps)
    red, wred = s.reduce(), o.reduce()
    s.close()
    assert abs(red[6] - wred[6]) <= 1e-3 * wred[6], (red[6], wred[6])
    if divu_mode == 1:
        assert abs(red[5] - wred[5]) <= 1e-3 * wred[5], (red[5], wred[5])


@pytest.mark.parametrize("divu_mode", [0, 1])
def test_front_position_stefan_layer_end_of_run(oracle_mod, divu_mode):
    """The film-freezing workload over its full 2000 steps: the front position,
    as the mean solid height sum f_s / nx, within 1e-3 of the oracle's; with
    divu_mode = 1 also the solid height on the centre column."""
    w = W.stefan_layer(nx=64, ny=256)
    w["params"] = dict(w["params"], divu_mode=divu_mode)
    f32 = _f32(w)
    s = lbfreeze.Solver(w["grid"], w["params"], f32)
    s.step(w["steps"])
    red = s.reduce()
    s.close()
    o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in f32.items()})
    o.step(w["steps"])
    wred = o.reduce()
    nx = w["grid"]["nx"]
    h_gpu, h_ora = red[3] / nx, wred[3] / nx
    assert h_ora > 5.0  # the front has advanced several cells
    assert abs(h_gpu - h_ora) <= 1e-3 * h_ora, (h_gpu, h_ora)
    if divu_mode == 1:
        assert abs(red[5] - wred[5]) <= 1e-3 * wred[5], (red[5], wred[5])
