"""The y-slab decomposition on the GPU (lb_slab_create, lb_slab_pack,
lb_slab_unpack): a lattice cut into slabs that exchange their two boundary
rows after every step advances bit for bit like the whole lattice.

Slabs of one lattice are stepped here in one process on one GPU, the halo
messages copied between them by the calls (device buffers), and in two
processes sharing the GPU whose messages go through host memory and gloo
(paper_2511_09422_gb300.slab).  No kernel waits on another: every exchange
happens on the host between steps."""
import os
import socket

import numpy as np
import pytest

from paper_2511_09422_gb300 import lbfreeze
from paper_2511_09422_gb300 import slab as S
from paper_2511_09422_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = lbfreeze.FIELD_NAMES


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_09422_gb300 import _build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    lbfreeze.load()


def _f32(w):
    return {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}


def _slabs(w, cuts):
    """Slab handles of w's lattice for the row cuts [0, c1, c2, ..., ny]."""
    ny = w["grid"]["ny"]
    f = _f32(w)
    out = []
    for y0, y1 in zip(cuts[:-1], cuts[1:]):
        lo, hi = S.local_rows(ny, y0, y1)
        local = {k: np.ascontiguousarray(v[lo:hi]) for k, v in f.items()}
        out.append((lbfreeze.Solver(w["grid"], w["params"], local, slab=(y0, y1)), y0, y1, y0 - lo))
    return out


def _exchange(slabs, bufs):
    for (a, *_), (b, *_), (ab, ba) in zip(slabs, slabs[1:], bufs):
        a.pack_halo(1, ab)
        b.pack_halo(0, ba)
        b.unpack_halo(0, ab)
        a.unpack_halo(1, ba)


def _run_slabs(w, cuts, steps):
    slabs = _slabs(w, cuts)
    n = slabs[0][0].halo_bytes
    bufs = [(torch.empty(n, dtype=torch.uint8, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda"))
            for _ in slabs[1:]]
    _exchange(slabs, bufs)
    for _ in range(steps):
        for s, *_ in slabs:
            s.step(1)
        _exchange(slabs, bufs)
    fields = {k: [] for k in FIELDS}
    red = np.zeros(8)
    for s, y0, y1, lo in slabs:
        f = s.fields()
        for k in FIELDS:
            fields[k].append(f[k][lo:lo + y1 - y0])
        red[:6] += s.reduce()[:6]
        s.close()
    return {k: np.concatenate(v) for k, v in fields.items()}, red


CASES = [
    ("droplet_97x71_3slabs", lambda: W.parity_droplet(nx=97, ny=71, seed=3), [0, 20, 45, 71], {}),
    ("droplet_128x96_mdot", lambda: W.parity_droplet(nx=128, ny=96), [0, 48, 96], dict(divu_mode=0)),
    ("droplet_97x71_fp16", lambda: W.parity_droplet(nx=97, ny=71, seed=3), [0, 30, 71],
     dict(pop_storage=lbfreeze.LB_STORAGE_F16)),
    ("droplet_97x71_fp16_h32", lambda: W.parity_droplet(nx=97, ny=71, seed=3), [0, 37, 71],
     dict(pop_storage=lbfreeze.LB_STORAGE_F16_H32)),
    ("droplet_97x71_d2q5", lambda: W.parity_droplet(nx=97, ny=71, seed=3), [0, 4, 67, 71],
     dict(lattice_fl=lbfreeze.LB_LATTICE_D2Q5)),
    ("impurity_front_160x128_4slabs", lambda: W.impurity_front(nx=160, ny=128, radius=20.0), [0, 32, 64, 96, 128],
     {}),
    ("bridge_two_dirichlet_walls", lambda: W.liquid_bridge(), [0, 24, 48], {}),
]


@pytest.mark.parametrize("name,make,cuts,opts", CASES, ids=[c[0] for c in CASES])
def test_slabs_equal_the_whole_lattice_bitwise(name, make, cuts, opts):
    """Slabs of 4 rows at the walls, uneven cuts, half storage, D2Q5, both
    readings of div u and Dirichlet walls at both ends: after 60 steps the
    owned rows of the slabs equal the whole lattice's fields bit for bit, and
    the slabs' diagnostics add up to the lattice's (same cells, summed in
    another order)."""
    w = make()
    w["params"] = dict(w["params"], **opts)
    got, red = _run_slabs(w, cuts, 60)
    s = lbfreeze.Solver(w["grid"], w["params"], _f32(w))
    s.step(60)
    want, wred = s.fields(), s.reduce()
    s.close()
    for k in FIELDS:
        assert np.array_equal(got[k], want[k]), (name, k, float(np.abs(got[k] - want[k]).max()))
    for k in range(6):
        assert abs(red[k] - wred[k]) <= 1e-12 * max(abs(wred[k]), 1.0), (k, red[k], wred[k])


def test_slab_arguments_are_checked():
    w = W.parity_droplet(nx=32, ny=40)
    f = _f32(w)
    for y0, y1 in ((0, 3), (2, 20), (20, 38), (-1, 10), (30, 41)):
        lo, hi = max(y0 - 2, 0), min(y1 + 2, 40)
        local = {k: np.ascontiguousarray(v[lo:hi]) for k, v in f.items()}
        with pytest.raises((lbfreeze.LbError, ValueError)):
            lbfreeze.Solver(w["grid"], w["params"], local, slab=(y0, y1))
    s = lbfreeze.Solver(w["grid"], w["params"], {k: np.ascontiguousarray(v[:22]) for k, v in f.items()}, slab=(0, 20))
    assert s.halo_bytes == 2 * 32 * (36 * 4 + 9 * 4)
    buf = np.empty(s.halo_bytes, dtype=np.uint8)
    with pytest.raises(lbfreeze.LbError):
        s.pack_halo(0, buf)  # the bottom wall: no neighbour below
    s.pack_halo(1, buf)
    s.close()
    whole = lbfreeze.Solver(w["grid"], w["params"], f)
    assert whole.halo_bytes == 0
    whole.close()


def _free_port() -> int:
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    return port


def _rank_main(rank, world, port, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        w = W.impurity_front(nx=160, ny=128, radius=20.0)
        s = S.SlabSolver(w["grid"], w["params"], _f32(w), dist, rank, world)
        s.step(steps)
        red = s.reduce()
        q.put((rank, s.y0, s.y1, s.fields(), red))
        s.close()
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo_equal_the_whole_lattice_bitwise():
    """Two processes on the one GPU, each with a slab of the 160 x 128
    impurity front, exchanging their halos through host memory and gloo after
    every step (SlabSolver): after 100 steps the gathered fields equal the
    whole lattice bit for bit, and the all-reduced diagnostics, V*_s and V*_sl
    included, equal the lattice's."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, 100, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.impurity_front(nx=160, ny=128, radius=20.0)
    s = lbfreeze.Solver(w["grid"], w["params"], _f32(w))
    s.step(100)
    want, wred = s.fields(), s.reduce()
    s.close()
    for k in FIELDS:
        assert np.array_equal(np.concatenate([g[3][k] for g in got]), want[k]), k
    for rank, y0, y1, f, red in got:
        np.testing.assert_allclose(red, wred, rtol=1e-12, atol=1e-12)
