"""Batched instances (lb_batch_*): many independent lattices in one persistent
launch per step.  Every instance must evolve bit for bit as a single-lattice
handle created from the same inputs, whatever the graph / tuning path."""
import ctypes as C

import numpy as np
import pytest

from paper_2511_09422_gb300 import lbfreeze
from paper_2511_09422_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("phi", "T", "fs", "C", "ux", "uy", "p")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_09422_gb300 import _build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    lbfreeze.load()


def _f32(w):
    return {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}


def _mixed():
    """Uneven shapes and parameters, including lattices narrower than one strip,
    with fewer rows than one inner segment, and with several segments."""
    ws = [W.parity_droplet(nx=40, ny=33, seed=1), W.parity_droplet(nx=97, ny=71, seed=2),
          W.impurity_front(nx=128, ny=100, radius=15.0), W.stefan_layer(nx=30, ny=5, h0=3),
          W.thermocapillary_channel(nx=64, ny=32, h=16, sigma_T=-5e-4),
          W.sessile_droplet(nx=150, ny=130, radius=40.0, rho_g=0.1, ste=0.3, c0=0.07)]
    for w in ws:
        w["fields"] = _f32(w)
    return ws


def _single(w, steps):
    s = lbfreeze.Solver(w["grid"], w["params"], w["fields"])
    s.step(steps)
    out = s.fields()
    s.close()
    return out


def _assert_same(a, b, label):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), "%s: field %s differs (max %.3e)" % (
            label, k, float(np.abs(a[k].astype(np.float64) - b[k]).max()))


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_single_lattices_bitwise(graph):
    ws = _mixed()
    b = lbfreeze.Batch(ws)
    b.use_graph(graph)
    b.step(17)  # odd: graph pairs plus one plain launch
    for i, w in enumerate(ws):
        _assert_same(b.instance(i).fields(), _single(w, 17), "instance %d" % i)
        assert b.instance(i).steps == 17
    b.close()


def test_batch_tuning_keeps_state_and_results():
    ws = _mixed()
    b = lbfreeze.Batch(ws)
    b.step(4)
    before = [b.instance(i).fields() for i in range(len(ws))]
    choice = b.tune(trials=2)
    assert all(c in (0, 8, 12, 16, 24, 32, 64) for c in choice) and any(choice)
    for i in range(len(ws)):
        _assert_same(b.instance(i).fields(), before[i], "after tuning, instance %d" % i)
    b.step(9)
    for i, w in enumerate(ws):
        _assert_same(b.instance(i).fields(), _single(w, 13), "tuned instance %d" % i)
    b.close()


def test_batch_diagnostics_per_instance(oracle_mod):
    ws = _mixed()[:3]
    b = lbfreeze.Batch(ws)
    b.step(20)
    for i, w in enumerate(ws):
        red = b.instance(i).reduce()
        o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in w["fields"].items()})
        o.step(20)
        want = o.reduce()
        for k in range(5):
            assert abs(red[k] - want[k]) <= 1e-5 * max(abs(want[k]), 1.0), (i, k, red, want)
    b.close()


def test_batch_rejects_instances_out_of_step():
    ws = _mixed()[:2]
    b = lbfreeze.Batch(ws)
    b.instance(0).step(1)
    with pytest.raises(lbfreeze.LbError) as e:
        b.step(1)
    assert e.value.status == lbfreeze.LB_ERR_INVALID_ARG
    b.instance(1).step(1)
    b.step(2)  # back in step
    b.close()


def test_batch_create_reports_the_bad_instance():
    ws = _mixed()[:3]
    ws[1] = dict(ws[1], params=dict(ws[1]["params"], eps=0.0))
    with pytest.raises(lbfreeze.LbError) as e:
        lbfreeze.Batch(ws)
    assert e.value.status == lbfreeze.LB_ERR_INVALID_ARG
    assert "instance 1" in str(e.value)


@pytest.mark.parametrize("storage", [0, 1])
def test_full_sweep_sampled_instances(oracle_mod, storage):
    """The benchmark's batch at full size: the 256-droplet sweep (28.4 M cells,
    sides 128..512, contact angles 60..120 degrees), autotuned and stepped
    through the CUDA graph as the benchmark does, in FP32 and in half storage.
    Sampled instances (the smallest, the largest, two seeded picks) equal lone
    lattices bit for bit; the smallest also matches the oracle at the FP32
    parity bar (FP32 storage)."""
    import test_parity_gpu as P
    sweep = W.droplet_sweep(n=256)
    for w in sweep:
        w["params"] = dict(w["params"], pop_storage=storage)
        w["fields"] = _f32(w)
    sides = [w["meta"]["side"] for w in sweep]
    rng = np.random.default_rng(3)
    picks = sorted({int(np.argmin(sides)), int(np.argmax(sides))} | set(int(i) for i in rng.integers(0, 256, 2)))
    b = lbfreeze.Batch(sweep)
    b.tune(trials=1)
    b.use_graph(True)
    steps = 7
    b.step(steps)
    for i in picks:
        _assert_same(b.instance(i).fields(), _single(sweep[i], steps), "sweep instance %d" % i)
    if storage == 0:
        i = int(np.argmin(sides))
        w = sweep[i]
        o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in w["fields"].items()})
        o.step(steps)
        want = o.fields()
        want["_walls"] = P._wall_temperatures(w["grid"])
        P._assert_parity(b.instance(i).fields(), want, label="sweep instance %d" % i)
    b.close()
