"""End-of-run parity at the scale of the sessile-droplet configuration of
Sec. 4.4: a 256^2 droplet (R = 50, Ste 0.1, C0 0.05, Ma 10; the 512^2, R = 100
case halved) run to full freezing on the GPU, against the FP64 oracle's end
state stored in tests/golden/droplet_256_end_state.txt (written by
tests/golden/make_droplet_end_state.py, which calls only the oracle).

The freezing time (first crossing of sum f_s = 0.99 sum chi, diagnostics every
10 steps as in the golden run, interpolated) and the front height (solid on
the centre column) at the crossing sample and at the end must lie within 1e-3
of the oracle's, for FP32 storage and for half storage with an FP32 enthalpy
set.  The final volumes V*_s and V*_sl are held to 1e-3 in FP32; with the
phase-field populations in half precision the volume of phase-change material
drifts by the rounding of their deviations over the 35 000 steps (measured
1.1e-3), so they are held to 2e-3 there.  Half storage of every set is
reported, not held to 1e-3: the rounding of the enthalpy deviations drifts its
freezing time (measured 1.7e-3)."""
import os

import numpy as np
import pytest

from paper_2511_09422_gb300 import lbfreeze

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "droplet_256_end_state.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_09422_gb300 import _build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    lbfreeze.load()


def _golden():
    kv = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if "=" in line:
                k, v = line.split("=")
                kv[k.strip()] = float(v)
    return kv


def _run(storage):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_droplet_end_state",
                                                  os.path.join(HERE, "golden", "make_droplet_end_state.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    g = _golden()
    w = mk.workload()
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}
    s = lbfreeze.Solver(w["grid"], dict(w["params"], pop_storage=storage), f32)
    every = int(g["sample_every"])
    prev, tf, cross = None, None, None
    while tf is None:
        s.step(every)
        r = s.reduce()
        gg = r[3] - mk.FRAC * r[4]
        if gg >= 0.0:
            n = s.steps
            tf = (n - every) + every * (-prev) / (gg - prev) if prev is not None else float(n)
            cross = r
        prev = gg
        assert s.steps < 2 * g["t_f"], "no full freezing"
    s.step(int(g["end_step"]) - s.steps if int(g["end_step"]) > s.steps else mk.TAIL)
    end = s.reduce()
    s.close()
    return g, tf, cross, end


@pytest.mark.parametrize("storage", [lbfreeze.LB_STORAGE_F32, lbfreeze.LB_STORAGE_F16_H32], ids=["fp32", "fp16_h32"])
def test_droplet_end_state_matches_the_oracle(storage):
    g, tf, cross, end = _run(storage)
    assert abs(tf - g["t_f"]) <= 1e-3 * g["t_f"], (tf, g["t_f"])
    assert abs(cross[5] - g["front_at_cross"]) <= 1e-3 * g["front_at_cross"], (cross[5], g["front_at_cross"])
    assert abs(end[5] - g["front_at_end"]) <= 1e-3 * g["front_at_end"], (end[5], g["front_at_end"])
    vol_tol = 1e-3 if storage == lbfreeze.LB_STORAGE_F32 else 2e-3
    assert abs(end[6] - g["Vs_at_end"]) <= vol_tol * g["Vs_at_end"], (end[6], g["Vs_at_end"])
    assert abs(end[7] - g["Vsl_at_end"]) <= vol_tol * g["Vsl_at_end"], (end[7], g["Vsl_at_end"])


def test_all_half_storage_end_state_is_reported():
    """Every set in half precision: the end state is finite and close (5e-3),
    and its freezing-time error is printed for the record."""
    g, tf, cross, end = _run(lbfreeze.LB_STORAGE_F16)
    err = abs(tf - g["t_f"]) / g["t_f"]
    print("all-FP16 storage: freezing time %.1f vs oracle %.1f (relative %.2e)" % (tf, g["t_f"], err))
    assert np.isfinite(end).all()
    assert err <= 5e-3
