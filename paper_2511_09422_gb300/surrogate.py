"""Learned surrogate of the LB freezing step, with the LB step as fallback.

The surrogate (``cno.Net``) predicts the change of the seven macroscopic
fields (phi, T, f_s, C, u_x, u_y, p; Sec. 2-3) over K_JUMP LB steps.  It is
trained on trajectories the LB solver itself generates (sessile droplets
freezing on a cold wall, Sec. 4.4, at 256^2 with the parameters of the batched
sweep), on the GPU, with the library's own forward and backward kernels.

A jump is accepted only if the predicted state passes two checks against the
state it started from (both computed by ``cno.field_checks`` in FP64):

* mass of the phase-change material, M = rho_s sum f_s + rho_l sum (chi - f_s),
  conserved by the method (Sec. 2.1: the density change on freezing is what
  moves the interface, mass is not created), within ``mass_tol`` relative;
* interface width, W = 2 sum (1 - phi^2) / sum |grad phi| (W for a flat
  profile phi = tanh(2 d / W), Eq. 3 with the workloads' W = 4), within
  ``width_tol`` relative.

An accepted prediction becomes the new LB state through ``lb_set_fields``
(populations at the equilibrium of the predicted fields); a rejected one is
discarded and the LB takes the K_JUMP steps itself, from the unchanged state.
After a rejection the stepper waits for a number of jumps that doubles with
each consecutive rejection before it tries the surrogate again.

Everything numeric runs in the two CUDA libraries; this module orders the
calls and keeps device buffers (torch tensors used as memory).
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import cno, lbfreeze
from . import workloads as W

FIELDS = lbfreeze.FIELD_NAMES  # phi, T, fs, C, ux, uy, p
K_JUMP = 50


@dataclasses.dataclass
class Normaliser:
    """Input x_f = (field_f - offset_f) * inv_scale_f; output: change_f = out_f * out_scale_f."""
    offset: np.ndarray
    inv_scale: np.ndarray
    out_scale: np.ndarray

    def to_arrays(self) -> dict:
        return dict(offset=self.offset, inv_scale=self.inv_scale, out_scale=self.out_scale)

    @classmethod
    def from_arrays(cls, d) -> "Normaliser":
        return cls(np.asarray(d["offset"], np.float32), np.asarray(d["inv_scale"], np.float32),
                   np.asarray(d["out_scale"], np.float32))


@dataclasses.dataclass
class Snapshots:
    """Fields of several trajectories, every `every` steps: data[i, f] is field
    f of snapshot i (device FP32 [ny, nx]); pairs[j] = (i, i + 1) are
    consecutive snapshots of one trajectory; traj[i] its trajectory."""
    data: object
    traj: np.ndarray
    pairs: np.ndarray
    every: int


def generate(n_instances=32, side=256, steps=15000, every=K_JUMP, seed=20251109, log=None) -> Snapshots:
    """Run a batch of freezing sessile droplets (radius, Stefan number,
    Marangoni numbers and solute drawn as in the batched sweep, one lattice
    size) and keep their fields every `every` steps, on the device."""
    import torch
    ws = W.droplet_sweep(n=n_instances, seed=seed, side_min=side, side_max=side)
    b = lbfreeze.Batch(ws)
    nsnap = steps // every + 1
    data = torch.empty((n_instances * nsnap, len(FIELDS), side, side), dtype=torch.float32, device="cuda")

    def grab(slot):
        for i in range(n_instances):
            inst = b.instance(i)
            inst.fields(out={f: data[i * nsnap + slot, k] for k, f in enumerate(FIELDS)})

    t0 = time.time()
    grab(0)
    for s in range(1, nsnap):
        b.step(every)
        grab(s)
    torch.cuda.synchronize()
    b.close()
    if log:
        log("generated %d snapshots (%d droplets x %d) in %.1f s" % (n_instances * nsnap, n_instances, nsnap,
                                                                      time.time() - t0))
    traj = np.repeat(np.arange(n_instances), nsnap)
    pairs = np.array([(i * nsnap + s, i * nsnap + s + 1) for i in range(n_instances) for s in range(nsnap - 1)],
                     dtype=np.int64)
    return Snapshots(data=data, traj=traj, pairs=pairs, every=every)


def fit_normaliser(snaps: Snapshots, sample=64, seed=0) -> Normaliser:
    """Per-field mean and spread of the fields and of their change over one
    pair, from a sample of snapshots (host statistics of device data)."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(snaps.pairs), size=min(sample, len(snaps.pairs)), replace=False)
    cur = snaps.data[snaps.pairs[idx, 0]].cpu().double().numpy()
    nxt = snaps.data[snaps.pairs[idx, 1]].cpu().double().numpy()
    offset = cur.mean(axis=(0, 2, 3))
    spread = cur.std(axis=(0, 2, 3))
    dspread = (nxt - cur).std(axis=(0, 2, 3))
    inv_scale = 1.0 / np.maximum(spread, 1e-6)
    out_scale = np.maximum(dspread, 1e-9)
    return Normaliser(offset.astype(np.float32), inv_scale.astype(np.float32), out_scale.astype(np.float32))


class Trainer:
    """Mini-batch training of a network on snapshot pairs (Adam, cosine
    learning-rate decay); batches are packed on the device by the library."""

    def __init__(self, net: cno.Net, snaps: Snapshots, norm: Normaliser, batch=16, seed=0, holdout=None):
        import torch
        self.net, self.snaps, self.norm, self.batch = net, snaps, norm, batch
        self.rng = np.random.default_rng(seed)
        ny, nx = snaps.data.shape[2:]
        self.x = torch.empty((batch, ny, nx, cno.CIN), dtype=torch.bfloat16, device="cuda")
        self.t = torch.empty((batch, ny, nx, cno.NF), dtype=torch.float32, device="cuda")
        self.inv_out = (1.0 / norm.out_scale).astype(np.float32)
        holdout = set() if holdout is None else set(int(h) for h in holdout)
        tr = np.array([snaps.traj[i] not in holdout for i in snaps.pairs[:, 0]])
        self.train_pairs = snaps.pairs[tr]
        self.val_pairs = snaps.pairs[~tr]

    def _pack(self, pairs):
        d = self.snaps.data
        for b, (i, j) in enumerate(pairs):
            cur = [d[i, k] for k in range(len(FIELDS))]
            nxt = [d[j, k] for k in range(len(FIELDS))]
            cno.pack_fields(cur, self.norm.offset, self.norm.inv_scale, out=self.x[b:b + 1])
            cno.pack_delta(cur, nxt, self.inv_out, self.t[b])

    def fit(self, iters=3000, lr=1e-3, lr_min=1e-5, log_every=0, log=None):
        losses = []
        t0 = time.time()
        for it in range(iters):
            sel = self.train_pairs[self.rng.integers(0, len(self.train_pairs), size=self.batch)]
            self._pack(sel)
            lr_it = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / max(1, iters)))
            want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
            loss = self.net.train_step(self.x, self.t, lr_it, update=True, want_loss=want)
            if want:
                losses.append((it, loss))
                if log:
                    log("iter %5d  lr %.2e  loss %.4e  (%.1f s)" % (it, lr_it, loss, time.time() - t0))
        return losses

    def validation_loss(self, nbatches=4):
        """Mean loss on held-out pairs (no update)."""
        if len(self.val_pairs) == 0:
            return float("nan")
        out = []
        for k in range(nbatches):
            sel = self.val_pairs[self.rng.integers(0, len(self.val_pairs), size=self.batch)]
            self._pack(sel)
            out.append(self.net.train_step(self.x, self.t, 0.0, update=False))
        return float(np.mean(out))


def init_params(seed=0, cin=cno.CIN, widths=cno.WIDTHS, cout=cno.COUT) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 cin))), zero biases, the head scaled by
    0.1 so that the first predictions are small changes."""
    rng = np.random.default_rng(seed)
    out = []
    shapes = cno.layer_shapes(cin, widths, cout)
    for k, (ci, co) in enumerate(shapes):
        w = rng.standard_normal((co, 9, ci)) * math.sqrt(2.0 / (9 * ci))
        if k == len(shapes) - 1:
            w *= 0.1
        out.append((w.astype(np.float32), np.zeros(co, np.float32)))
    return cno.flatten(out)


def save(path, net: cno.Net, norm: Normaliser):
    np.savez(path, params=net.params(), widths=np.array(net.widths), **norm.to_arrays())


def load_model(path):
    d = np.load(path)
    net = cno.Net(widths=tuple(int(v) for v in d["widths"]))
    net.set_params(d["params"])
    return net, Normaliser.from_arrays(d)


class SurrogateStepper:
    """Advance an ``lbfreeze.Solver`` with surrogate jumps of K_JUMP steps,
    each accepted only if the mass and interface-width checks pass, the LB
    step otherwise (see the module text)."""

    def __init__(self, solver: lbfreeze.Solver, net: cno.Net, norm: Normaliser, params: dict, k=K_JUMP,
                 mass_tol=1e-3, width_tol=0.05, max_backoff=8):
        import torch
        self.s, self.net, self.norm, self.k = solver, net, norm, k
        self.rho_s, self.rho_l = float(params["rho_s"]), float(params["rho_l"])
        self.mass_tol, self.width_tol, self.max_backoff = mass_tol, width_tol, max_backoff
        ny, nx = solver.ny, solver.nx
        mk = lambda: {f: torch.empty((ny, nx), dtype=torch.float32, device="cuda") for f in FIELDS}
        self.cur, self.pred = mk(), mk()
        self.x = torch.empty((1, ny, nx, cno.CIN), dtype=torch.bfloat16, device="cuda")
        self.out = torch.empty((1, ny, nx, cno.NF), dtype=torch.float32, device="cuda")
        self.accepted = self.rejected = self.skipped = 0
        self._wait, self._backoff = 0, 1
        self.last = None

    def _measures(self, F):
        s = cno.field_checks(F["phi"], F["fs"])
        mass = self.rho_s * s[2] + self.rho_l * (s[1] - s[2])
        width = 2.0 * s[3] / s[4] if s[4] > 0 else float("nan")
        return mass, width

    def try_jump(self) -> bool:
        """One surrogate jump from the solver's current state; True if it was
        accepted (and the solver now holds the prediction)."""
        self.s.fields(out=self.cur)
        m0, w0 = self._measures(self.cur)
        cno.pack_fields([self.cur[f] for f in FIELDS], self.norm.offset, self.norm.inv_scale, out=self.x)
        self.net.forward(self.x, out=self.out)
        cno.apply_update([self.cur[f] for f in FIELDS], [self.pred[f] for f in FIELDS], self.out,
                         self.norm.out_scale)
        m1, w1 = self._measures(self.pred)
        dm = abs(m1 - m0) / max(abs(m0), 1e-300)
        dw = abs(w1 / w0 - 1.0) if w0 > 0 else float("inf")
        ok = bool(np.isfinite(m1) and np.isfinite(w1) and dm <= self.mass_tol and dw <= self.width_tol)
        self.last = dict(mass_change=dm, width_change=dw, accepted=ok)
        if ok:
            self.s.set_fields(self.pred)
        return ok

    def advance(self, nsteps: int):
        """Advance by nsteps LB-step equivalents."""
        done = 0
        while nsteps - done >= self.k:
            if self._wait > 0:
                self._wait -= 1
                self.skipped += 1
                self.s.step(self.k)
            elif self.try_jump():
                self.accepted += 1
                self._backoff = 1
            else:
                self.rejected += 1
                self.s.step(self.k)
                self._wait = self._backoff
                self._backoff = min(2 * self._backoff, self.max_backoff)
            done += self.k
        if nsteps > done:
            self.s.step(nsteps - done)

    def stats(self) -> dict:
        jumps = self.accepted + self.rejected + self.skipped
        return dict(jumps=jumps, accepted=self.accepted, rejected=self.rejected, skipped=self.skipped,
                    acceptance=self.accepted / jumps if jumps else 0.0)
