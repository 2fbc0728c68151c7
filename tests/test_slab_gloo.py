"""The y-slab decomposition's host logic on the CPU: the row partition, and
the per-step halo exchange of paper_2511_09422_gb300.slab over gloo ranks.

The exchange is driven here by a stand-in for the library's slab handle: a
toy lattice whose step, like the LB step, makes every owned row depend on the
rows up to two away (a nonlinear five-row stencil, periodic in x, mirrored at
the two walls), with the library's halo message layout (two owned rows per
face) and ghost rows.  Run as two and three gloo ranks, the slabs must
reproduce the whole toy lattice bit for bit: a wrong neighbour, face, row
offset or ordering of the exchange breaks that.  The CUDA slab itself is
checked against the whole lattice on the GPU (tests/test_slab_gpu.py)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_09422_gb300 import slab as S  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _toy_rows(a: np.ndarray, rows, ny_global: int, y_first: int) -> np.ndarray:
    """New values of ``rows`` (local indices) of the toy lattice ``a`` whose
    local row 0 is global row ``y_first``: a five-row, three-column nonlinear
    stencil; rows beyond the global walls are mirrored."""
    out = np.empty((len(rows), a.shape[1]))
    for k, y in enumerate(rows):
        acc = np.zeros(a.shape[1])
        for dy, w in ((-2, 0.05), (-1, 0.2), (0, 0.5), (1, 0.15), (2, 0.1)):
            g = y_first + y + dy
            if g < 0:
                g = -g - 1
            elif g >= ny_global:
                g = 2 * ny_global - g - 1
            row = a[g - y_first]
            acc += w * (0.25 * np.roll(row, 1) + 0.5 * row + 0.25 * np.roll(row, -1))
        out[k] = acc + 0.01 * np.sin(acc)
    return out


class ToySlab:
    """Stand-in for lbfreeze.Solver(slab=...): halo_bytes, pack_halo,
    unpack_halo and step, on a float64 toy lattice."""

    def __init__(self, full: np.ndarray, y0: int, y1: int):
        self.ny, self.nx = full.shape
        self.lo, self.hi = S.local_rows(self.ny, y0, y1)
        self.y0, self.y1 = y0, y1
        self.a = full[self.lo:self.hi].copy()
        self.glo, self.ghi = y0 - self.lo, self.hi - y1

    @property
    def halo_bytes(self):
        return 2 * self.nx * 8

    def step(self):
        own = list(range(self.glo, self.glo + self.y1 - self.y0))
        # a ghost row's mirror partner never lies outside the local rows: the
        # global walls are only at ends without ghost rows
        new = _toy_rows(self.a, own, self.ny, self.lo)
        self.a[self.glo:self.glo + len(own)] = new

    def pack_halo(self, face, buf):
        r = self.glo if face == 0 else self.a.shape[0] - self.ghi - 2
        buf[:] = np.frombuffer(np.ascontiguousarray(self.a[r:r + 2]).tobytes(), dtype=np.uint8)

    def unpack_halo(self, face, buf):
        r = 0 if face == 0 else self.a.shape[0] - 2
        self.a[r:r + 2] = np.frombuffer(np.asarray(buf).tobytes(), dtype=np.float64).reshape(2, self.nx)


def _whole(full, steps):
    a = full.copy()
    for _ in range(steps):
        a = _toy_rows(a, list(range(a.shape[0])), a.shape[0], 0)
    return a


def _rank_main(rank, world, port, ny, nx, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = np.random.default_rng(11).uniform(-1.0, 1.0, size=(ny, nx))
        y0, y1 = S.slab_rows(ny, world, rank)
        h = ToySlab(full, y0, y1)
        x = S.SlabExchange(h, dist, rank, world)
        x.exchange()
        for _ in range(steps):
            h.step()
            x.exchange()
        q.put((rank, y0, y1, h.a[h.glo:h.glo + y1 - y0].copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ny", [(2, 23), (3, 17)])
def test_slabs_reproduce_the_whole_toy_lattice(world, ny):
    import torch.multiprocessing as mp
    nx, steps = 12, 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ny, nx, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=180) for _ in procs), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = _whole(np.random.default_rng(11).uniform(-1.0, 1.0, size=(ny, nx)), steps)
    rows = np.concatenate([g[3] for g in got])
    assert [g[1] for g in got] == [S.slab_rows(ny, world, r)[0] for r in range(world)]
    assert rows.shape == want.shape
    assert np.array_equal(rows, want)


@pytest.mark.parametrize("ny,world", [(8, 2), (9, 2), (4096, 8), (4097, 3), (12, 3)])
def test_slab_rows_cover_the_lattice(ny, world):
    parts = [S.slab_rows(ny, world, r) for r in range(world)]
    assert parts[0][0] == 0 and parts[-1][1] == ny
    for (a0, a1), (b0, b1) in zip(parts, parts[1:]):
        assert a1 == b0
    heights = [y1 - y0 for y0, y1 in parts]
    assert min(heights) >= S.MIN_ROWS and max(heights) - min(heights) <= 1


def test_slab_rows_reject_too_thin_slabs():
    with pytest.raises(ValueError):
        S.slab_rows(15, 4, 0)
    with pytest.raises(ValueError):
        S.slab_rows(100, 2, 2)


def test_local_rows_add_ghosts_only_between_slabs():
    assert S.local_rows(40, 0, 20) == (0, 22)
    assert S.local_rows(40, 20, 40) == (18, 40)
    assert S.local_rows(40, 10, 30) == (8, 32)
    assert S.local_rows(40, 0, 40) == (0, 40)
