"""Half-precision population storage: every set in FP16 (lb_params.pop_storage
= LB_STORAGE_F16), or f, g and l in FP16 with the enthalpy set h in FP32
(LB_STORAGE_F16_H32).

The populations are stored as scaled FP16 deviations and the arithmetic stays
FP32, so the results differ from the oracle by the rounding of every stored
population to 11 bits.  These tests state that difference: per field after 100
steps (same scales as the FP32 parity tests), and on the end-of-run quantities
-- the freezing time of a droplet and the mean front height of the film --
which must stay within 1e-3 of the oracle like the FP32 path."""
import numpy as np
import pytest

from paper_2511_09422_gb300 import lbfreeze
from paper_2511_09422_gb300 import workloads as W

import test_parity_gpu as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F16 = 1
F16_H32 = 2
HALF_FORMS = [F16, F16_H32]
# Six roundings of a stored deviation to 11 bits (6 x 2^-11 = 2.9e-3).  Measured
# after 100 steps over the seven cases below, both half forms: at most 2.3e-3
# (C, ragged 97 x 71 droplet), 2.1e-3 (u_y and p, heated channel), 1.0e-3
# (phi, impurity front), 5.2e-4 (f_s), 1.8e-4 (T).
FIELD_TOL = 6 * 2.0 ** -11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_09422_gb300 import _build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    lbfreeze.load()


def _half(w, form=F16):
    return dict(w, params=dict(w["params"], pop_storage=form))


@pytest.mark.parametrize("form", HALF_FORMS)
@pytest.mark.parametrize("name,make,steps", P.CASES, ids=[c[0] for c in P.CASES])
def test_fp16_fields_against_oracle(oracle_mod, name, make, steps, form):
    w = make()
    got, red, want, wred = P._run_pair(oracle_mod, w, steps, params=_half(w, form)["params"])
    errs = P._rel_errors(got, want)
    assert all(v <= FIELD_TOL for v in errs.values()), (name, errs)
    assert all(np.isfinite(got[k]).all() for k in P.FIELDS)



@pytest.mark.parametrize("form", HALF_FORMS)
def test_fp16_full_size_bench_workload(oracle_mod, form):
    """The 4096 x 4096 impurity front in half storage, as the benchmark's
    half-storage legs run it, a few steps against the oracle on every cell."""
    w = W.impurity_front(nx=4096, ny=4096)
    got, red, want, wred = P._run_pair(oracle_mod, w, 3, params=_half(w, form)["params"])
    errs = P._rel_errors(got, want)
    assert all(v <= FIELD_TOL for v in errs.values()), errs

@pytest.mark.parametrize("form", HALF_FORMS)
def test_fp16_freezing_time(oracle_mod, form):
    w = W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.1, ste=0.2)
    f32 = P._f32(w)
    s = lbfreeze.Solver(w["grid"], _half(w, form)["params"], f32)
    tf_gpu, _ = P._freezing_time(s.step, s.reduce, 5000)
    s.close()
    o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in f32.items()})
    tf_ora, _ = P._freezing_time(o.step, o.reduce, 5000)
    assert abs(tf_gpu - tf_ora) <= 1e-3 * tf_ora, (tf_gpu, tf_ora)


@pytest.mark.parametrize("form", HALF_FORMS)
def test_fp16_front_height_end_of_run(oracle_mod, form):
    w = W.stefan_layer(nx=64, ny=256)
    f32 = P._f32(w)
    s = lbfreeze.Solver(w["grid"], _half(w, form)["params"], f32)
    s.step(w["steps"])
    red = s.reduce()
    s.close()
    o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in f32.items()})
    o.step(w["steps"])
    wred = o.reduce()
    assert abs(red[3] - wred[3]) <= 1e-3 * wred[3], (red[3] / 64, wred[3] / 64)


@pytest.mark.parametrize("form", HALF_FORMS)
def test_fp16_checkpoint_resume_bitwise(tmp_path, form):
    w = _half(W.parity_droplet(nx=64, ny=48), form)
    f32 = P._f32(w)
    a = lbfreeze.Solver(w["grid"], w["params"], f32)
    a.step(30)
    a.save(str(tmp_path / "ck16.bin"))
    a.step(30)
    fa = a.fields()
    b = lbfreeze.Solver(w["grid"], w["params"], f32)
    b.load_state(str(tmp_path / "ck16.bin"))
    b.step(30)
    fb = b.fields()
    for k in P.FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
    c = lbfreeze.Solver(w["grid"], dict(w["params"], pop_storage=0), f32)
    with pytest.raises(lbfreeze.LbError):
        c.load_state(str(tmp_path / "ck16.bin"))  # written with the other storage


@pytest.mark.parametrize("form", HALF_FORMS)
def test_fp16_batch_matches_single_and_rejects_mixed_storage(form):
    ws = [_half(W.parity_droplet(nx=40, ny=33, seed=1), form), _half(W.impurity_front(nx=128, ny=100, radius=15.0), form),
          _half(W.sessile_droplet(nx=150, ny=130, radius=40.0, rho_g=0.1, ste=0.3, c0=0.07), form)]
    for w in ws:
        w["fields"] = P._f32(w)
    b = lbfreeze.Batch(ws)
    b.step(11)
    for i, w in enumerate(ws):
        s = lbfreeze.Solver(w["grid"], w["params"], w["fields"])
        s.step(11)
        want = s.fields()
        s.close()
        got = b.instance(i).fields()
        for k in P.FIELDS:
            assert np.array_equal(got[k], want[k]), (i, k)
    b.close()
    mixed = [ws[0], dict(ws[1], params=dict(ws[1]["params"], pop_storage=3 - form))]
    with pytest.raises(lbfreeze.LbError) as e:
        lbfreeze.Batch(mixed)
    assert "pop_storage" in str(e.value)


def test_half_forms_with_fp32_enthalpy_store_fewer_bytes():
    """Device bytes of the population buffers: FP32 144, FP16 72, FP16 with an
    FP32 enthalpy set 90 bytes per cell and buffer."""
    w = W.parity_droplet(nx=64, ny=48)
    f32 = P._f32(w)
    sizes = {}
    for form in (0, F16, F16_H32):
        s = lbfreeze.Solver(w["grid"], dict(w["params"], pop_storage=form), f32)
        sizes[form] = s.device_bytes
        s.close()
    plane = 64 * 48  # pitch 64
    assert sizes[0] - sizes[F16] == 2 * (144 - 72) * plane
    assert sizes[0] - sizes[F16_H32] == 2 * (144 - 90) * plane
