"""One lattice cut into y-slabs, one slab per rank (one rank per GPU).

The step of Sec. 3 reads, for every cell, its own populations and those of its
eight neighbours, and the isotropic stencils (end of Sec. 3.4) of the fields
computed from them reach one cell further.  So a slab advances exactly as its
rows of the whole lattice do when, before every step, it holds copies of the
two rows of state on either side that belong to its neighbours (ghost rows).
After each step every rank sends its two lowest owned rows to the rank below
and its two highest to the rank above, and receives theirs into its ghost
rows: one point-to-point exchange per face and step, through
torch.distributed (NCCL with device buffers, or gloo with host buffers).  The
diagnostics are sums over the slabs (an FP64 all-reduce).

The arithmetic stays in the CUDA library (lbfreeze.Solver with slab=); this
module only partitions the rows and moves the messages.
"""
from __future__ import annotations

import numpy as np

MIN_ROWS = 4  # rows of the smallest slab (the library's limit)


def slab_rows(ny: int, world: int, rank: int):
    """Rows [y0, y1) of ``rank``'s slab: ny rows split into ``world`` slabs of
    nearly equal height, rank 0 at the bottom wall."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of %d" % (rank, world))
    if ny < MIN_ROWS * world:
        raise ValueError("%d rows cannot make %d slabs of at least %d rows" % (ny, world, MIN_ROWS))
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def local_rows(ny: int, y0: int, y1: int):
    """Rows of the lattice a slab holds: its own and two ghost rows at every end
    that borders another slab (none at a wall)."""
    return (y0 - 2 if y0 > 0 else 0), (y1 + 2 if y1 < ny else ny)


class SlabExchange:
    """The per-step halo exchange of one rank.  ``handle`` provides halo_bytes,
    pack_halo(face, buf) and unpack_halo(face, buf) (lbfreeze.Solver with
    slab=, or a stand-in with the same calls); ``dist`` is an initialised
    torch.distributed; ``device`` selects CUDA buffers (for NCCL) instead of
    host buffers (for gloo)."""

    def __init__(self, handle, dist, rank: int, world: int, device: bool = False):
        import torch
        self.h, self.dist, self.rank, self.world = handle, dist, rank, world
        self.below = rank - 1 if rank > 0 else None
        self.above = rank + 1 if rank < world - 1 else None
        n = handle.halo_bytes
        kw = dict(dtype=torch.uint8, device="cuda") if device else dict(dtype=torch.uint8)
        self.send = {f: torch.empty(n, **kw) for f in (0, 1)}
        self.recv = {f: torch.empty(n, **kw) for f in (0, 1)}
        self.device = device

    def _buf(self, t):
        return t if self.device else t.numpy()

    def exchange(self):
        """Send the owned boundary rows to both neighbours and receive theirs
        into the ghost rows.  Face 0 talks to the rank below, face 1 to the
        rank above; every send is matched by the neighbour's receive of the
        opposite face."""
        peers = {0: self.below, 1: self.above}
        for f, peer in peers.items():
            if peer is not None:
                self.h.pack_halo(f, self._buf(self.send[f]))
        reqs = []
        for f, peer in peers.items():
            if peer is not None:
                reqs.append(self.dist.isend(self.send[f], dst=peer))
                reqs.append(self.dist.irecv(self.recv[f], src=peer))
        for r in reqs:
            r.wait()
        for f, peer in peers.items():
            if peer is not None:
                self.h.unpack_halo(f, self._buf(self.recv[f]))


class SlabSolver:
    """One rank's slab of a lattice split across ``world`` ranks: the
    library's slab handle plus the exchange.  ``fields`` are the initial fields
    of the whole lattice (ny x nx arrays); each rank keeps its local rows."""

    def __init__(self, grid: dict, params: dict, fields: dict, dist, rank: int, world: int, stream=None,
                 device_exchange: bool = False):
        from . import lbfreeze
        self.ny, self.nx = int(grid["ny"]), int(grid["nx"])
        self.y0, self.y1 = slab_rows(self.ny, world, rank)
        lo, hi = local_rows(self.ny, self.y0, self.y1)
        self.lo = self.y0 - lo  # ghost rows below the owned ones
        local = {k: np.ascontiguousarray(np.asarray(v, dtype=np.float32)[lo:hi]) for k, v in fields.items()
                 if v is not None}
        self.solver = lbfreeze.Solver(grid, params, local, stream=stream, slab=(self.y0, self.y1))
        self.dist, self.rank, self.world = dist, rank, world
        self.x = SlabExchange(self.solver, dist, rank, world, device=device_exchange) if world > 1 else None
        self.V0 = self._allreduce(np.array([self.solver.reduce()[4]]))[0]
        if self.x is not None:
            self.x.exchange()  # ghost rows from the neighbours' initial state

    def _allreduce(self, v: np.ndarray) -> np.ndarray:
        if self.world == 1:
            return v
        import torch
        t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
        self.dist.all_reduce(t)
        return t.numpy()

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.solver.step(1)
            if self.x is not None:
                self.x.exchange()

    def reduce(self) -> np.ndarray:
        """The eight diagnostics of lb_reduce for the whole lattice."""
        r = self.solver.reduce()
        s = self._allreduce(np.array(r[:6]))
        return np.concatenate([s, [s[3] / self.V0, s[4] / self.V0]])

    def fields(self) -> dict:
        """The owned rows of the macroscopic fields, (y1 - y0) x nx arrays."""
        f = self.solver.fields()
        n = self.y1 - self.y0
        return {k: v[self.lo:self.lo + n] for k, v in f.items()}

    def close(self):
        self.solver.close()
