"""The D2Q5 option for the phase-field and solute sets on the GPU
(lb_params.lattice_fl = LB_LATTICE_D2Q5): parity with the FP64 oracle's D2Q5
option at 1e-5 after 100 steps, end-of-run freezing time within 1e-3,
batches bitwise equal to single lattices, checkpoints, and the reductions."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_parity_gpu as P  # noqa: E402
from paper_2511_09422_gb300 import workloads as W  # noqa: E402

Q5 = 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09422_gb300 import _build, lbfreeze
    _build.build()
    lbfreeze.load()


def _q5(w):
    return dict(w, params=dict(w["params"], lattice_fl=Q5))


# Every field keeps the 1e-5 bar of the D2Q9 path.
TOL_Q5 = {"phi": 1e-5, "T": 1e-5, "fs": 1e-5, "C": 1e-5, "ux": 1e-5, "uy": 1e-5, "p": 1e-5}

# The ragged 97 x 71 droplet with div u = mdot (divu_mode = 0) passes through a
# short ill-conditioned transient at the top wall: between steps 99 and 105 the
# expansion flow reaches the gas layer under the wall, where the D2Q5 phase field
# overshoots to phi = -1.014, and any perturbation there grows about 100-fold and
# decays again by step 107.  Two GPU runs whose inputs differ by 1e-7 differ by
# 1.2e-5 in u_y at step 100 and 2.3e-5 at step 102, as much as GPU and oracle do
# (test_d2q5_top_wall_transient_is_ill_conditioned), so that case is compared at
# step 150, after the transient (measured 4e-6).  All other cases, and this one
# with the lagged velocity divergence, are compared at step 100.
STEPS_Q5 = {("ragged_droplet_97x71", 0): 150}


@pytest.mark.parametrize("divu_mode", [0, 1])
@pytest.mark.parametrize("name,make,steps", P.CASES, ids=[c[0] for c in P.CASES])
def test_parity_d2q5(oracle_mod, name, make, steps, divu_mode):
    w = _q5(make())
    p = dict(w["params"], divu_mode=divu_mode)
    steps = STEPS_Q5.get((name, divu_mode), steps)
    got, red, want, wred = P._run_pair(oracle_mod, w, steps, params=p)
    errs = P._rel_errors(got, want)
    bad = {k: v for k, v in errs.items() if not v <= TOL_Q5[k]}
    assert not bad, (name, divu_mode, bad, errs)
    P._assert_reduce(red, wred)


def test_d2q5_top_wall_transient_is_ill_conditioned(oracle_mod):
    """The transient that makes the mdot-reading 97 x 71 droplet unfit for a
    comparison at step 100 is a property of the case, not a difference between
    GPU and oracle: a GPU run from inputs perturbed by 1e-7 (relative) moves
    away from the unperturbed GPU run by more than 1e-5 in u_y at step 102, and
    the GPU-oracle difference there is of the same size; by step 150 both are
    back below 1e-5."""
    from paper_2511_09422_gb300 import lbfreeze
    w = _q5(W.parity_droplet(nx=97, ny=71, seed=3))
    p = dict(w["params"], divu_mode=0)
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}
    rng = np.random.default_rng(5)
    g32 = {k: (v.astype(np.float64) * (1 + 1e-7 * rng.uniform(-1, 1, size=v.shape))).astype(np.float32)
           for k, v in f32.items()}
    a, b = lbfreeze.Solver(w["grid"], p, f32), lbfreeze.Solver(w["grid"], p, g32)
    o = oracle_mod.Oracle(w["grid"], p, {k: v.astype(np.float64) for k, v in f32.items()})
    out = {}
    for n in (102, 150):
        a.step(n - a.steps)
        b.step(n - b.steps)
        o.step(n - o.steps)
        fa, fb, fo = a.fields(), b.fields(), o.fields()
        speed = float(np.sqrt(fo["ux"] ** 2 + fo["uy"] ** 2).max())
        gg = float(np.abs(fa["uy"].astype(np.float64) - fb["uy"]).max()) / speed
        go = float(np.abs(fa["uy"].astype(np.float64) - fo["uy"]).max()) / speed
        out[n] = (gg, go)
    a.close()
    b.close()
    gg, go = out[102]
    assert gg > 1e-5, out
    assert go < 3.0 * gg, out
    assert max(out[150]) < 1e-5, out


def test_d2q5_full_size_bench_workload(oracle_mod):
    """The 4096 x 4096 impurity front with D2Q5 f and l, as the benchmark's
    D2Q5 leg runs it, a few steps against the oracle on every cell."""
    w = _q5(W.impurity_front(nx=4096, ny=4096))
    got, red, want, wred = P._run_pair(oracle_mod, w, 3, params=w["params"])
    errs = P._rel_errors(got, want)
    bad = {k: v for k, v in errs.items() if not v <= TOL_Q5[k]}
    assert not bad, (bad, errs)
    P._assert_reduce(red, wred)

def test_d2q5_freezing_time(oracle_mod):
    from paper_2511_09422_gb300 import lbfreeze
    w = _q5(W.sessile_droplet(nx=48, ny=40, radius=12.0, rho_g=0.1, ste=0.2))
    f32 = P._f32(w)
    s = lbfreeze.Solver(w["grid"], w["params"], f32)
    tf_gpu, _ = P._freezing_time(s.step, s.reduce, 5000)
    s.close()
    o = oracle_mod.Oracle(w["grid"], w["params"], {k: v.astype(np.float64) for k, v in f32.items()})
    tf_ora, _ = P._freezing_time(o.step, o.reduce, 5000)
    assert abs(tf_gpu - tf_ora) <= 1e-3 * tf_ora, (tf_gpu, tf_ora)


def test_d2q5_batch_checkpoint_and_reductions(tmp_path):
    from paper_2511_09422_gb300 import lbfreeze
    ws = [_q5(W.parity_droplet(nx=40, ny=33, seed=1)), _q5(W.impurity_front(nx=128, ny=100, radius=15.0))]
    for w in ws:
        w["fields"] = P._f32(w)
    b = lbfreeze.Batch(ws)
    b.step(9)
    for i, w in enumerate(ws):
        s = lbfreeze.Solver(w["grid"], w["params"], w["fields"])
        s.step(9)
        want = s.fields()
        got = b.instance(i).fields()
        for k in P.FIELDS:
            assert np.array_equal(got[k], want[k]), (i, k)
        r1 = s.reduce()
        L = lbfreeze.load()
        L.lb_reduce_noalloc.restype = C.c_int
        L.lb_reduce_noalloc.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
        out = (C.c_double * 8)()
        assert L.lb_reduce_noalloc(C.c_void_p(s.handle), out) == 0
        # the two reductions sum per lattice row or per warp: the last digits differ
        assert np.allclose(r1, np.array(out[:]), rtol=1e-11, atol=1e-12)
        s.save(str(tmp_path / ("q5_%d.bin" % i)))
        s.step(7)
        after = s.fields()
        t = lbfreeze.Solver(w["grid"], w["params"], w["fields"])
        t.load_state(str(tmp_path / ("q5_%d.bin" % i)))
        t.step(7)
        for k in P.FIELDS:
            assert np.array_equal(t.fields()[k], after[k]), (i, k)
        u = lbfreeze.Solver(w["grid"], dict(w["params"], lattice_fl=0), w["fields"])
        with pytest.raises(lbfreeze.LbError):
            u.load_state(str(tmp_path / ("q5_%d.bin" % i)))   # a D2Q9 handle rejects a D2Q5 state
        for h in (s, t, u):
            h.close()
    b.close()
    mixed = [ws[0], dict(ws[1], params=dict(ws[1]["params"], lattice_fl=0))]
    with pytest.raises(lbfreeze.LbError) as e:
        lbfreeze.Batch(mixed)
    assert "lattice_fl" in str(e.value)
