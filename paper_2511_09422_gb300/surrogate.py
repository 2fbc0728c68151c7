"""Learned surrogate of the LB freezing step, with the LB step as fallback.

The surrogate (``cno.Net``) predicts the change of the seven macroscopic
fields (phi, T, f_s, C, u_x, u_y, p; Sec. 2-3) over K_JUMP LB steps.  It is
trained on trajectories the LB solver itself generates at 256^2 (sessile
droplets freezing on a cold wall, Sec. 4.4, with the parameters of the
batched sweep, and planar fronts advancing toward an insoluble impurity), on
the GPU, with the library's own forward and backward kernels.

A jump is accepted only if the predicted state passes two checks against the
state it started from (both computed by ``cno.field_checks`` in FP64):

* mass of the phase-change material, M = rho_s sum f_s + rho_l sum (chi - f_s),
  conserved by the method (Sec. 2.1: the density change on freezing is what
  moves the interface, mass is not created), within ``mass_tol`` relative;
* interface width, W = 2 sum (1 - phi^2) / sum |grad phi| (W for a flat
  profile phi = tanh(2 d / W), Eq. 3 with the workloads' W = 4), within
  ``width_tol`` relative;
* enthalpy balance (Sec. 2.3): the change of sum rho H over the jump equals
  the rate measured on the last LB chunk times K_JUMP within ``h_tol``.

With ``h_project`` the predicted change of f_s is first rescaled so that the
enthalpy balance holds (see ``_project_enthalpy``); the check then only
catches what the rescaling cannot fix (clamping).

The predicted change of phi is applied only inside the interface band
(|phi| < phi_band, 0.999 by default): away from the interface the order
parameter sits at its bulk values +-1 and the method keeps it there, while
small errors of the network there would add up over a large lattice.

An accepted prediction becomes the new LB state through ``lb_set_fields``
(populations at the equilibrium of the predicted fields); a rejected one is
discarded and the LB takes the K_JUMP steps itself, from the unchanged state.
After a rejection the stepper runs a number of LB chunks that doubles with
each consecutive rejection (up to ``max_backoff``) before it tries the
surrogate again, so a surrogate that keeps failing costs little.

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


def training_workloads(n_instances=48, side=256, seed=20251109, impurity_fraction=0.5) -> list:
    """Lattices to learn from, all side x side: freezing sessile droplets with
    the parameter ranges of the batched sweep (radius 0.2-0.35 side, Stefan
    0.05-0.5, Ma 0-50, C0 0-0.1), and a fraction of planar fronts advancing
    from the cold wall toward an insoluble circular impurity (radius 0.05-0.15
    side, centre x uniform, y 0.2-0.5 side, density ratio 2; same Stefan, Ma
    and C0 ranges) -- the geometry of the large impurity case at a small size."""
    n_imp = int(round(impurity_fraction * n_instances))
    ws = W.droplet_sweep(n=n_instances - n_imp, seed=seed, side_min=side, side_max=side)
    rng = np.random.default_rng(seed + 1)
    for i in range(n_imp):
        radius = float(rng.uniform(0.05, 0.15)) * side
        cx, cy = float(rng.uniform(0, side)), float(rng.uniform(0.2, 0.5)) * side
        w = W.impurity_front(nx=side, ny=side, radius=radius, center=(cx, cy), c0=float(rng.uniform(0.0, 0.1)),
                             ma=float(rng.uniform(0.0, 50.0)), ste=float(rng.uniform(0.05, 0.5)))
        w["name"] = "impurity_%03d_%d" % (i, side)
        ws.append(w)
    return ws


def generate(n_instances=48, side=256, steps=12000, every=K_JUMP, seed=20251109, impurity_fraction=0.5,
             log=None) -> Snapshots:
    """Run a batch of the training lattices (``training_workloads``) and keep
    their fields every `every` steps, on the device."""
    import torch
    ws = training_workloads(n_instances, side, seed, impurity_fraction)
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
        log("generated %d snapshots (%d lattices x %d) in %.1f s" % (n_instances * nsnap, n_instances, nsnap,
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
    each accepted only if the mass, interface-width and enthalpy-balance
    checks pass, the LB step otherwise (see the module text).

    Between LB chunks at most ``jumps_per_lb`` jumps are tried; every LB chunk
    measures the rate at which the lattice loses enthalpy (through the cold
    wall), and a jump is accepted only if its own enthalpy change matches that
    rate over K_JUMP steps within ``h_tol`` (relative): the latent heat that
    freezing releases has to leave through the wall, so a prediction that
    freezes too fast or too slow breaks the balance."""

    def __init__(self, solver: lbfreeze.Solver, net: cno.Net, norm: Normaliser, params: dict, k=K_JUMP,
                 mass_tol=1e-3, width_tol=0.05, h_tol=0.02, jumps_per_lb=2, max_backoff=64, phi_band=0.999,
                 slow_only=True, h_project=False, device="cuda"):
        import torch
        self.s, self.net, self.norm, self.k = solver, net, norm, k
        self.rho_s, self.rho_l = float(params["rho_s"]), float(params["rho_l"])
        lat = float(params["rho_l"]) * float(params["latent"]) if int(params.get("phase_change_on", 1)) else 0.0
        self.hcoef = (float(params["rho_l"]) * float(params["cp_l"]), float(params["rho_s"]) * float(params["cp_s"]),
                      float(params["rho_g"]) * float(params["cp_g"]), lat)
        self.mass_tol, self.width_tol, self.h_tol = mass_tol, width_tol, h_tol
        self.jumps_per_lb, self.max_backoff = jumps_per_lb, max_backoff
        self.phi_band, self.slow_only, self.h_project = phi_band, slow_only, h_project
        ny, nx = solver.ny, solver.nx
        mk = lambda: {f: torch.empty((ny, nx), dtype=torch.float32, device=device) for f in FIELDS}
        self.cur, self.pred = mk(), mk()
        self.scratch = mk() if h_project else None
        self.x = torch.empty((1, ny, nx, cno.CIN), dtype=torch.bfloat16, device=device)
        self.out = torch.empty((1, ny, nx, cno.NF), dtype=torch.float32, device=device)
        self.accepted = self.rejected = self.lb_chunks = 0
        self._wait, self._backoff, self._jumps = 0, 1, 0
        self.h_rate = None
        self._fresh = False     # the last LB chunk measured the enthalpy rate
        self.last = None

    def _measures(self, F):
        s = cno.field_checks(F["phi"], F["fs"], F["T"], self.hcoef)
        mass = self.rho_s * s[2] + self.rho_l * (s[1] - s[2])
        width = 2.0 * s[3] / s[4] if s[4] > 0 else float("nan")
        return mass, width, (s[5], s[6]), s[7]

    def _lb_chunk(self, measure: bool):
        """K_JUMP LB steps; with measure, also the enthalpy change per step."""
        if measure:
            self.s.fields(out=self.cur)
            h0 = self._measures(self.cur)[3]
        self.s.step(self.k)
        if measure:
            self.s.fields(out=self.cur)
            h1 = self._measures(self.cur)[3]
            self.h_rate = (h1 - h0) / self.k
        self._fresh = measure
        self.lb_chunks += 1
        self._jumps = 0

    def try_jump(self) -> bool:
        """One surrogate jump from the solver's current state; True if it was
        accepted (and the solver now holds the prediction)."""
        self.s.fields(out=self.cur)
        m0, w0, t0, h0 = self._measures(self.cur)
        cno.pack_fields([self.cur[f] for f in FIELDS], self.norm.offset, self.norm.inv_scale, out=self.x)
        self.net.forward(self.x, out=self.out)
        scale = np.array(self.norm.out_scale, np.float32)
        if self.slow_only:
            # the fast fields (velocity, pressure) stay the LB's: they relax within a
            # few steps to the slow fields (phi, T, f_s, C) that the network moves
            scale[[FIELDS.index("ux"), FIELDS.index("uy"), FIELDS.index("p")]] = 0.0
        # projection onto the admissible states: phi in [-1, 1], f_s in [0, 1],
        # C >= 0, and T within its current range (the maximum principle of the
        # heat equation, with the walls and the melting point as the only extremes)
        inf = float("inf")
        lo = [-1.0, t0[0], 0.0, 0.0, -inf, -inf, -inf]
        hi = [1.0, t0[1], 1.0, inf, inf, inf, inf]
        cno.apply_update([self.cur[f] for f in FIELDS], [self.pred[f] for f in FIELDS], self.out, scale,
                         self.phi_band, lo, hi)
        if self.h_project and self._fresh:
            self._project_enthalpy(scale, h0, lo, hi)
        m1, w1, t1, h1 = self._measures(self.pred)
        dm = abs(m1 - m0) / max(abs(m0), 1e-300)
        dw = abs(w1 / w0 - 1.0) if w0 > 0 else float("inf")
        want = (self.h_rate or 0.0) * self.k
        dh = abs((h1 - h0) - want) / max(abs(want), 1e-12 * max(abs(h0), 1.0))
        ok = bool(np.isfinite(m1) and np.isfinite(w1) and np.isfinite(h1) and self._fresh
                  and dm <= self.mass_tol and dw <= self.width_tol and dh <= self.h_tol)
        self.last = dict(mass_change=dm, width_change=dw, enthalpy_mismatch=dh, accepted=ok,
                         fs_scale=getattr(self, "last_c", None) if self.h_project else None)
        if ok:
            self.s.set_fields(self.pred)
        return ok

    def _project_enthalpy(self, scale, h0, lo, hi):
        """Rescale the predicted change of f_s by the factor c that makes the
        jump's enthalpy change equal the rate measured on the last LB chunk:
        at the predicted T the enthalpy is linear in f_s, so with H_a the
        enthalpy of (predicted T, current f_s) and H_b that of the prediction,
        c = (H_0 + rate K - H_a) / (H_b - H_a), clamped to [0, 2].  The front
        then advances at the rate the wall's heat extraction allows (the
        Stefan condition), with the network's shape of the change."""
        F = self.pred
        h_b = cno.field_checks(F["phi"], F["fs"], F["T"], self.hcoef)[7]
        h_a = cno.field_checks(F["phi"], self.cur["fs"], F["T"], self.hcoef)[7]
        want = h0 + self.h_rate * self.k
        c = 1.0 if abs(h_b - h_a) < 1e-12 * max(abs(h0), 1.0) else (want - h_a) / (h_b - h_a)
        c = min(max(c, 0.0), 2.0)
        sc = np.zeros(len(FIELDS), np.float32)
        k = FIELDS.index("fs")
        sc[k] = c * scale[k]
        dst = [self.scratch[f] for f in FIELDS]
        dst[k] = F["fs"]
        cno.apply_update([self.cur[f] for f in FIELDS], dst, self.out, sc, 0.0, lo, hi)
        self.last_c = c

    def advance(self, nsteps: int):
        """Advance by nsteps LB-step equivalents."""
        done = 0
        while nsteps - done >= self.k:
            if self._wait > 0:
                # backing off after a rejection: plain LB chunks; the last one before
                # the next attempt measures the enthalpy rate
                self._wait -= 1
                self._lb_chunk(measure=self._wait == 0)
            elif not self._fresh or self._jumps >= self.jumps_per_lb:
                self._lb_chunk(measure=True)
            elif self.try_jump():
                self.accepted += 1
                self._jumps += 1
                self._backoff = 1
            else:
                self.rejected += 1
                self._lb_chunk(measure=False)
                self._wait = self._backoff
                self._backoff = min(2 * self._backoff, self.max_backoff)
            done += self.k
        if nsteps > done:
            self.s.step(nsteps - done)

    def stats(self) -> dict:
        chunks = self.accepted + self.lb_chunks
        return dict(chunks=chunks, accepted=self.accepted, rejected=self.rejected, lb_chunks=self.lb_chunks,
                    acceptance=self.accepted / chunks if chunks else 0.0)


def train_default(n_instances=48, side=256, steps=12000, iters=3000, lr=3e-4, batch=16, seed=20251109, log=None):
    """Generate the training trajectories, fit the normalisation and train a
    network from the He-normal start; returns (net, normaliser, info)."""
    import torch
    t0 = time.perf_counter()
    snaps = generate(n_instances, side, steps, seed=seed, log=log)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    norm = fit_normaliser(snaps)
    net = cno.Net()
    net.set_params(init_params(0))
    hold = [n_instances // 2 - 1, n_instances - 1]  # one droplet, one impurity front
    tr = Trainer(net, snaps, norm, batch=batch, holdout=hold)
    t1 = time.perf_counter()
    tr.fit(iters=iters, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    info = dict(snapshots=int(snaps.data.shape[0]), lattices=n_instances, side=side, every=snaps.every,
                generate_s=round(t_gen, 2), train_s=round(t_train, 2), iters=iters, batch=batch,
                ms_per_iter=round(1e3 * t_train / iters, 3), val_loss=round(tr.validation_loss(), 5),
                holdout=hold)
    del tr, snaps
    torch.cuda.empty_cache()
    return net, norm, info


def _f32_fields(workload):
    return {k: np.asarray(v, np.float32) for k, v in workload["fields"].items()}


def compare(workload, net, norm, steps, warm=100, **kw) -> dict:
    """The LB alone and the LB with surrogate jumps, from the same state after
    `warm` LB steps, over `steps` LB-step equivalents: wall-clock rate (the
    stepper synchronises for its checks) and the final diagnostics."""
    import torch
    out = {}
    for mode in ("lb", "surrogate"):
        s = lbfreeze.Solver(workload["grid"], workload["params"], _f32_fields(workload))
        s.step(warm)
        st = SurrogateStepper(s, net, norm, workload["params"], **kw) if mode == "surrogate" else None
        torch.cuda.synchronize()
        t = time.perf_counter()
        if st:
            st.advance(steps)
        else:
            s.step(steps)
        r = s.reduce()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        out[mode] = dict(steps_per_s=steps / dt, reduce=r, stats=st.stats() if st else None)
        s.close()
    a, b = out["lb"]["reduce"], out["surrogate"]["reduce"]
    out["front_rel_diff"] = abs(b[5] - a[5]) / max(abs(a[5]), 1e-30)
    out["solid_rel_diff"] = abs(b[3] - a[3]) / max(abs(a[3]), 1e-30)
    return out


def freezing_time(workload, net=None, norm=None, max_steps=60000, frac=0.99, **kw):
    """Steps until sum f_s reaches `frac` of sum chi (checked every K_JUMP steps,
    linear interpolation between checks) with the LB alone (net None) or with
    surrogate jumps; returns (t_f, wall seconds, stepper stats or None)."""
    import torch
    s = lbfreeze.Solver(workload["grid"], workload["params"], _f32_fields(workload))
    st = SurrogateStepper(s, net, norm, workload["params"], **kw) if net is not None else None
    t = time.perf_counter()
    n, prev, tf = 0, (0, 0.0), float("nan")
    try:
        while n < max_steps:
            if st:
                st.advance(K_JUMP)
            else:
                s.step(K_JUMP)
            n += K_JUMP
            r = s.reduce()
            f = r[3] / r[4]
            if f >= frac:
                n0, f0 = prev
                tf = n0 + (frac - f0) / (f - f0) * (n - n0)
                break
            prev = (n, f)
    except lbfreeze.LbError:
        tf = float("nan")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    stats = st.stats() if st else None
    s.close()
    return tf, dt, stats
