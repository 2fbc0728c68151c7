"""What the trained surrogate gains over the LB step alone, measured on a
held-out droplet: a network is trained here (a short schedule on LB
trajectories) and the freezing time is run to 99 % solid with the LB alone,
with strict jumps, and with enthalpy-projected jumps; the gains and errors are
printed as a JSON report.

Checked invariants:
- a strict run in which no jump was accepted is the LB run, bit for bit, so
  its freezing time is the LB's;
- handing a state back to the LB (lb_set_fields at the equilibrium of its own
  fields) moves the freezing time by at most 1e-4 per hand-back: the floor
  that an accepted jump costs even when its prediction is exact.
The checks of a strict jump do not guarantee the 1e-3 freezing-time bar by
themselves: the bench records a network whose two accepted jumps (of 323)
moved it by 2e-3."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09422_gb300 import _build, cno, lbfreeze
    _build.build()
    lbfreeze.load()
    cno.load()


def _held_out():
    from paper_2511_09422_gb300 import surrogate as S
    # a droplet outside the 16-lattice training set below (which holds the first 8
    # droplets of the sweep): the 24th, the one the bench holds out
    return S.training_workloads(48, 256)[23]


def test_trained_surrogate_gain_and_accuracy(tmp_path):
    from paper_2511_09422_gb300 import surrogate as S
    net, norm, info = S.train_default(n_instances=16, steps=6000, iters=600)
    held = _held_out()
    tf_lb, dt_lb, _ = S.freezing_time(held)
    tf_s, dt_s, st_s = S.freezing_time(held, net, norm)
    tf_p, dt_p, st_p = S.freezing_time(held, net, norm, h_project=True)
    net.close()
    report = dict(training=info, lb=dict(t_f=tf_lb, s=dt_lb),
                  strict=dict(t_f=tf_s, s=dt_s, rel_error=abs(tf_s - tf_lb) / tf_lb, speedup=dt_lb / dt_s,
                              stepper=st_s),
                  projected=dict(t_f=tf_p, s=dt_p, rel_error=abs(tf_p - tf_lb) / tf_lb, speedup=dt_lb / dt_p,
                                 stepper=st_p))
    (tmp_path / "surrogate_gain.json").write_text(json.dumps(report, indent=1, default=float))
    print(json.dumps(report, default=float))
    assert np.isfinite(tf_lb) and tf_lb > 0 and np.isfinite(tf_s) and np.isfinite(tf_p)
    if st_s["accepted"] == 0:
        assert tf_s == tf_lb   # every chunk ran on the LB
    assert st_p["chunks"] > 0 and np.isfinite(report["projected"]["speedup"])


def test_hand_back_costs_at_most_1e4_of_the_freezing_time_per_jump():
    from paper_2511_09422_gb300 import lbfreeze
    w = _held_out()
    f32 = {k: np.asarray(v, np.float32) for k, v in w["fields"].items()}

    def run(hand_back_at):
        s = lbfreeze.Solver(w["grid"], w["params"], f32)
        n, prev, tf = 0, (0, 0.0), float("nan")
        while n < 60000:
            s.step(50)
            n += 50
            if n in hand_back_at:
                s.set_fields(s.fields(device=True))   # the state handed back unchanged
            r = s.reduce()
            f = r[3] / r[4]
            if f >= 0.99:
                tf = prev[0] + (0.99 - prev[1]) / (f - prev[1]) * (n - prev[0])
                break
            prev = (n, f)
        s.close()
        return tf

    t0 = run(set())
    pts = set(range(1000, 16000, 1000))
    t1 = run(pts)
    per = abs(t1 - t0) / t0 / len(pts)
    assert per <= 1e-4, (t0, t1, per)
