"""Host logic of the surrogate stepper, on the CPU with fakes for the solver,
the network and the library's check kernels: the cadence of LB chunks and
jumps, the enthalpy rate measured before an attempt, the doubling backoff
after a rejection, and the step accounting."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_09422_gb300 import cno, surrogate as S  # noqa: E402
from paper_2511_09422_gb300 import workloads as W  # noqa: E402


class FakeSolver:
    ny, nx = 8, 8

    def __init__(self):
        self.steps_run = 0
        self.calls = []
        self.installed = 0

    def step(self, n):
        self.steps_run += n
        self.calls.append(("step", n))

    def fields(self, out):
        for k, v in out.items():
            v.fill_(float(self.steps_run))
        return out

    def set_fields(self, f):
        self.installed += 1
        self.calls.append(("set", 0))


class FakeNet:
    def forward(self, x, out):
        out.zero_()
        return out


@pytest.fixture
def fakes(monkeypatch):
    state = {"accept": False}

    def field_checks(phi, fs=None, T=None, hcoef=None):
        # constant mass (1) and width (4); the enthalpy is the field's value, which the
        # fake solver sets to its step count: the LB loses one unit per step
        return (0.0, 1.0, 0.0, 2.0, 1.0, -1.0, 0.0, float(phi.reshape(-1)[0]))

    monkeypatch.setattr(cno, "field_checks", field_checks)
    monkeypatch.setattr(cno, "pack_fields", lambda *a, **k: None)

    def apply_update(src, dst, out, scale, phi_band=0.0, lo=None, hi=None):
        for a, b in zip(src, dst):
            # a prediction that matches the LB rate when accepted, far off otherwise
            b.copy_(a + (S.K_JUMP if state["accept"] else 1e6))

    monkeypatch.setattr(cno, "apply_update", apply_update)
    return state


def _stepper(fs, **kw):
    p = W.base_params()
    return S.SurrogateStepper(fs, FakeNet(), S.Normaliser(np.zeros(7, np.float32), np.ones(7, np.float32),
                                                         np.ones(7, np.float32)), p, device="cpu", **kw)


def test_rejections_back_off_and_every_step_is_run_by_the_lb(fakes):
    fakes["accept"] = False
    fs = FakeSolver()
    st = _stepper(fs, max_backoff=4)
    st.advance(20 * S.K_JUMP + 7)
    s = st.stats()
    assert fs.steps_run == 20 * S.K_JUMP + 7          # nothing skipped: the LB ran every step
    assert fs.installed == 0 and s["accepted"] == 0
    # attempts after a measured chunk, then backoffs of 1, 2, 4, 4, ... LB chunks
    assert s["rejected"] == 5, s
    assert s["lb_chunks"] == 20
    assert fs.calls[-1] == ("step", 7)


def test_accepted_jumps_alternate_with_measured_lb_chunks(fakes):
    fakes["accept"] = True
    fs = FakeSolver()
    st = _stepper(fs, jumps_per_lb=2)
    st.advance(9 * S.K_JUMP)
    s = st.stats()
    # chunk pattern: LB (measures the rate), jump, jump, LB, jump, jump, LB, jump, jump
    assert s["accepted"] == 6 and s["lb_chunks"] == 3 and s["rejected"] == 0, s
    assert fs.installed == 6
    assert fs.steps_run == 3 * S.K_JUMP          # the LB ran only its own chunks
    assert st.last["accepted"] and st.last["enthalpy_mismatch"] <= 1e-9


def test_no_jump_without_a_fresh_rate(fakes):
    fakes["accept"] = True
    fs = FakeSolver()
    st = _stepper(fs)
    assert not st.try_jump()          # the rate has not been measured yet
    assert fs.installed == 0
