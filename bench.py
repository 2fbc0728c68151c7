#!/usr/bin/env python
"""Throughput of the fused diffuse-interface LB freezing step on GB300.

Workload: the 4096 x 4096 planar freezing front advancing into a binary
liquid (C0 = 0.05) toward an insoluble circular impurity of radius 200 cells
(density ratio 2), Marangoni stresses on (Ma = 10), all four coupled D2Q9 sets
active.  One step = one fused kernel launch over the whole lattice.

Metric: MLUPS = lattice cells x steps / time / 1e6 (one update = one cell
advancing all four sets by one step), with the HBM-roofline fraction of the
step kernel against the measured copy bandwidth.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own lattice (replicas; the step
has no data-path exchange in this form) and the whole-job MLUPS is reported.

Besides the headline line's value, roofline, e2e (public API with pinned host
buffers), cpu_baseline (the FP64 oracle on the host cores) and clocks, the
JSON line carries the other forms of the step, each on the same GPU:
fp16_storage (half-precision populations), d2q5_fl (D2Q5 phase-field and
solute sets), batched (256 droplets in one launch per step, FP32 and FP16
storage, against stepping them one by one), droplet_freezing (a 512^2
droplet run to full freezing, FP32 and FP16), and surrogate (the learned
surrogate trained here, its jumps against the LB alone, and its tensor-core
forward pass).  --sur-forward-only times the surrogate's forward pass alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes of one lattice update: 36 populations and 8 lagged fields (f_s,
# Q, u_x, u_y, C, p, S, and phi or T), each read and written once, FP32.  The step
# also keeps the lagged T (phi) beside phi (T) as the reference of its deviation
# storage, 360 bytes in all; that design choice is reported beside the figure.
BYTES_PER_UPDATE = 352
BYTES_MOVED_PER_UPDATE = 360
NAMEPLATE_HBM_GBS = 7900.0  # HBM3e nameplate of one GB300, next to the measured copy bandwidth
WORKLOAD = dict(name="impurity_front", nx=4096, ny=4096)
PROFILE = os.path.join(ROOT, "profiles", "lb_step_kernel_impurity_front.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2511_09422_gb300", "csrc", "lb_kernels.cuh")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _kernel_hash() -> str:
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic_per_launch(cells: int):
    """DRAM bytes per step-kernel launch from the committed ncu summary, scaled
    to this lattice; None if there is none or the kernel changed since."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    kv = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    try:
        return float(kv["dram_bytes_per_cell"]) * cells
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(value: float, dist=None, device="cuda") -> float:
    """The largest value of a per-rank number over all ranks: a job's time is its
    slowest rank's.  dist is torch.distributed (initialised) or None for one rank."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs the same work on its own lattice)."""
    return world * units_per_rank / seconds


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _sample_text(size: int) -> str:
    return ("the benchmark's own impurity_front %dx%d lattice (impurity r=%g at (nx/2, ny/4), same parameters)"
            % (size, size, 200.0 * size / 4096.0))


def _oracle_sample(size: int, steps_min: int, seconds: float, warmup: int = 1, threads: int = 0):
    """The FP64 oracle on the benchmark's size x size impurity-front lattice, timed
    on the host cores (all of them, or ``threads``) after ``warmup`` untimed steps,
    for at least ``steps_min`` steps and ``seconds`` seconds: returns (MLUPS,
    steps, threads used, seconds)."""
    import numpy as np

    import oracle
    from paper_2511_09422_gb300 import workloads as W
    w = W.impurity_front(nx=size, ny=size, radius=200.0 * size / 4096.0)
    f = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in w["fields"].items()}
    if threads:
        oracle.oracle.set_threads(threads)
    o = oracle.Oracle(w["grid"], w["params"], f)
    del f, w
    o.step(max(warmup, 0))
    t0 = time.perf_counter()
    n = 0
    while n < steps_min or time.perf_counter() - t0 < seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    cores = oracle.oracle.num_threads()
    o.close()
    return size * size * n / dt / 1e6, n, cores, dt


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper ships no code) on the same
    lattice, workload and step count as the GPU arm, on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    mlups, n, cores, dt = _oracle_sample(args.size, max(args.steps, 1), 0.0, args.warmup)
    sample = _sample_text(args.size)
    line = {
        "impl": "reference", "metric": "MLUPS (all coupled fields)", "value": round(mlups, 3),
        "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / n * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "impurity_front %dx%d (planar front + insoluble impurity r=%g, C0=0.05, Ma=10), "
                               "FP64 CPU oracle" % (args.size, args.size, 200.0 * args.size / 4096.0),
                   "steps_timed": n},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d oracle steps after %d untimed on %s" % (n, args.warmup, sample)},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


BYTES_PER_UPDATE_F16 = 208  # 36 populations read + written as FP16, 8 lagged FP32 fields read + written
BYTES_PER_UPDATE_Q5 = 288   # D2Q5 f and l: 28 populations + 8 lagged fields, FP32, read + written
BYTES_PER_UPDATE_F16H = 244  # 27 FP16 populations (f, g, l) + 9 FP32 (h) + 8 lagged FP32 fields, read + written
# with the step's ninth lagged field (the deviation reference) 216 and 296 bytes are moved


def _fp16_leg(args, lbfreeze, w, f32, cells, torch, stream, ws, dist, peak_gbs, form=1):
    """The same lattice with half-precision population storage (form 1: every
    set; form 2: f, g, l in half, h in FP32): MLUPS, and achieved bandwidth
    against its own algorithmic bytes (208 or 244 B per update)."""
    nbytes = BYTES_PER_UPDATE_F16 if form == 1 else BYTES_PER_UPDATE_F16H
    s = lbfreeze.Solver(w["grid"], dict(w["params"], pop_storage=form), f32, stream=stream)
    s.step(args.warmup)
    stream.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    s.reduce()  # raises if the half-precision run went non-finite
    s.close()
    mlups = ws * cells * args.steps / (ms * 1e-3) / 1e6
    gbs = nbytes * cells * args.steps / (ms * 1e-3) / 1e9
    what = "FP16 population storage" if form == 1 else "FP16 f, g, l populations, FP32 enthalpy populations"
    return {"metric": "MLUPS (all coupled fields), " + what, "value": round(mlups, 2),
            "unit": "MLUPS", "ms_per_step": round(ms / args.steps, 4), "bytes_per_update": nbytes,
            "bytes_moved_per_update": nbytes + 8,
            "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak_gbs, 4) if peak_gbs else None,
            "dtype": "f32 arithmetic, " + ("f16 populations" if form == 1 else "f16 f/g/l and f32 h populations")}


def _d2q5_leg(args, lbfreeze, w, f32, cells, torch, stream, ws, dist, peak_gbs):
    """The same lattice with D2Q5 for the phase-field and solute sets: MLUPS, and
    achieved bandwidth against its own algorithmic bytes (288 B per update)."""
    s = lbfreeze.Solver(w["grid"], dict(w["params"], lattice_fl=1), f32, stream=stream)
    s.step(args.warmup)
    stream.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    s.reduce()  # raises if the run went non-finite
    s.close()
    mlups = whole_job_rate(cells * args.steps, ms * 1e-3, ws) / 1e6
    gbs = BYTES_PER_UPDATE_Q5 * cells * args.steps / (ms * 1e-3) / 1e9
    return {"metric": "MLUPS (all coupled fields), D2Q5 phase-field and solute sets", "value": round(mlups, 2),
            "unit": "MLUPS", "ms_per_step": round(ms / args.steps, 4), "bytes_per_update": BYTES_PER_UPDATE_Q5,
            "bytes_moved_per_update": BYTES_PER_UPDATE_Q5 + 8,
            "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak_gbs, 4) if peak_gbs else None,
            "dtype": "f32"}


def _batched_leg(args, lbfreeze, W, np, torch, stream, ws, dist):
    """Instance-steps/s of the droplet sweep: the batched persistent launch
    (autotuned segment heights, CUDA graph) against the same instances stepped
    one lattice at a time with the single-lattice launch."""
    sweep = W.droplet_sweep(n=args.batch)
    for w in sweep:
        w["fields"] = {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}
    n = len(sweep)
    b = lbfreeze.Batch(sweep, stream=stream)
    choice = b.tune(trials=3)
    cells = b.cells
    K = args.batch_steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(run):
        run(2)  # warm-up (an even count keeps the instances in step)
        stream.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        run(K)
        e1.record(stream)
        e1.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist)

    inst = [b.instance(i) for i in range(n)]

    def sequential(k):
        for s in inst:
            s.step(k)

    ms_b = timed(b.step)
    ms_s = timed(sequential)
    b.close()
    # the same sweep with half-precision population storage
    sweep16 = [dict(w, params=dict(w["params"], pop_storage=1)) for w in sweep]
    b16 = lbfreeze.Batch(sweep16, stream=stream)
    choice16 = b16.tune(trials=3)
    ms_16 = timed(b16.step)
    b16.close()
    sweep16h = [dict(w, params=dict(w["params"], pop_storage=2)) for w in sweep]
    b16h = lbfreeze.Batch(sweep16h, stream=stream)
    choice16h = b16h.tune(trials=3)
    ms_16h = timed(b16h.step)
    b16h.close()
    v_b = ws * n * K / (ms_b * 1e-3)
    v_s = ws * n * K / (ms_s * 1e-3)
    v_16 = ws * n * K / (ms_16 * 1e-3)
    return {"metric": "instance-steps/s", "value": round(v_b, 1), "unit": "instance-steps/s",
            "workload": "droplet sweep: %d instances, side U[128,512], R U[0.2,0.35] side, Ste U[0.05,0.5], "
                        "Ma U[0,50], C0 U[0,0.1], contact angle U[60,120] deg, seed 20251109" % n,
            "fp16_storage": {"value": round(v_16, 1), "mlups": round(ws * cells * K / (ms_16 * 1e-3) / 1e6, 1),
                             "seg_rows_by_class": choice16},
            "fp16_h32_storage": {"value": round(ws * n * K / (ms_16h * 1e-3), 1),
                                 "mlups": round(ws * cells * K / (ms_16h * 1e-3) / 1e6, 1),
                                 "seg_rows_by_class": choice16h},
            "instances": n, "cells": cells, "steps": K, "mlups": round(ws * cells * K / (ms_b * 1e-3) / 1e6, 1),
            "seg_rows_by_class": choice, "launches_per_step": 1,
            "sequential": {"value": round(v_s, 1), "mlups": round(ws * cells * K / (ms_s * 1e-3) / 1e6, 1),
                           "launches_per_step": n},
            "speedup": round(v_b / v_s, 3)}


def _freezing_leg(args, lbfreeze, W, np, torch):
    """A 512^2 binary sessile droplet (R = 100, 90 degrees, Ste 0.1, C0 0.05,
    Ma 10; gas density ratio 0.1) run until 99 % of the phase-change material
    is solid, with FP32, FP16 and FP16-with-FP32-enthalpy population storage: freezing time
    (diagnostics in FP64 every 500 steps, linear interpolation), final V*_sl,
    and wall time."""
    w = W.sessile_droplet(nx=512, ny=512, radius=100.0, rho_g=0.1, ste=0.1, c0=0.05, ma_T=10.0, ma_C=10.0)
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}
    out = {}
    for name, st in (("f32", 0), ("f16", 1), ("f16_h32", 2)):
        s = lbfreeze.Solver(w["grid"], dict(w["params"], pop_storage=st), f32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n, prev, tf, r = 0, (0, 0.0), float("nan"), None
        while n < args.freeze_max_steps:
            s.step(500)
            n += 500
            r = s.reduce()
            frac = r[3] / r[4]
            if frac >= 0.99:
                tf = prev[0] + (0.99 - prev[1]) / (frac - prev[1]) * (n - prev[0])
                break
            prev = (n, frac)
        dt = time.perf_counter() - t0
        out[name] = {"t_f": round(tf, 1), "steps_run": n, "V_sl": round(float(r[7]), 5), "wall_s": round(dt, 3),
                     "mlups": round(512 * 512 * n / dt / 1e6, 1)}
        s.close()
    out["fp16_rel_error_t_f"] = abs(out["f16"]["t_f"] - out["f32"]["t_f"]) / out["f32"]["t_f"]
    out["fp16_h32_rel_error_t_f"] = abs(out["f16_h32"]["t_f"] - out["f32"]["t_f"]) / out["f32"]["t_f"]
    out["workload"] = "sessile droplet 512x512, R=100, theta=90, Ste=0.1, C0=0.05, Ma_T=Ma_C=10, rho_g/rho_l=0.1"
    return out


def _surrogate_leg(args, torch, peaks):
    """The learned surrogate: trained here on LB trajectories (256^2
    droplets and impurity fronts), then LB alone vs LB with surrogate jumps and
    the enthalpy / mass / width checks on the 4096^2 impurity front, the
    freezing time of a held-out droplet, and the throughput of the tensor-core
    forward pass."""
    from paper_2511_09422_gb300 import cno
    from paper_2511_09422_gb300 import surrogate as S
    from paper_2511_09422_gb300 import workloads as W
    net, norm, info = S.train_default(n_instances=args.sur_lattices, steps=args.sur_steps, iters=args.sur_iters)
    big = W.impurity_front(nx=args.size, ny=args.size, radius=200.0 * args.size / 4096.0)
    cmp = S.compare(big, net, norm, steps=1000)
    cmp_p = S.compare(big, net, norm, steps=1000, h_project=True)
    held = S.training_workloads(args.sur_lattices, 256)[info["holdout"][0]]
    tf_lb, dt_lb, _ = S.freezing_time(held)
    tf_s, dt_s, st_s = S.freezing_time(held, net, norm)
    tf_p, dt_p, st_p = S.freezing_time(held, net, norm, h_project=True)
    # forward pass of the network on the large lattice, timed with CUDA events
    x = torch.zeros((1, args.size, args.size, cno.CIN), dtype=torch.bfloat16, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(0)
    x[..., :cno.NF] = torch.randn((1, args.size, args.size, cno.NF), generator=gen, device="cuda").to(torch.bfloat16)
    out = torch.empty((1, args.size, args.size, cno.NF), dtype=torch.float32, device="cuda")
    for _ in range(2):
        net.forward(x, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        net.forward(x, out=out)
    e1.record()
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 5
    flops = cno.forward_flops(args.size, args.size)
    tflops = flops / (fwd_ms * 1e-3) / 1e12
    peak_tf = peaks.get("bf16_tflops")
    net.close()
    lb, su, sp = cmp["lb"], cmp["surrogate"], cmp_p["surrogate"]
    return {
        "metric": "LB-step equivalents/s on impurity_front %dx%d with surrogate jumps of %d steps (1000 steps)"
                  % (args.size, args.size, S.K_JUMP),
        "value": round(su["steps_per_s"], 1), "lb_alone": round(lb["steps_per_s"], 1),
        "speedup": round(su["steps_per_s"] / lb["steps_per_s"], 3), "stepper": su["stats"],
        "front_rel_diff": cmp["front_rel_diff"], "solid_rel_diff": cmp["solid_rel_diff"],
        "with_enthalpy_projection": {
            "value": round(sp["steps_per_s"], 1), "lb_alone": round(cmp_p["lb"]["steps_per_s"], 1),
            "speedup": round(sp["steps_per_s"] / cmp_p["lb"]["steps_per_s"], 3), "stepper": sp["stats"],
            "front_rel_diff": cmp_p["front_rel_diff"], "solid_rel_diff": cmp_p["solid_rel_diff"]},
        "freezing_time_heldout_droplet": {"lb": round(tf_lb, 1), "surrogate": round(tf_s, 1),
                                          "rel_error": abs(tf_s - tf_lb) / tf_lb, "lb_s": round(dt_lb, 3),
                                          "surrogate_s": round(dt_s, 3), "stepper": st_s,
                                          "with_enthalpy_projection": {
                                              "t_f": round(tf_p, 1), "rel_error": abs(tf_p - tf_lb) / tf_lb,
                                              "s": round(dt_p, 3), "stepper": st_p}},
        "training": info,
        "forward": {"ms": round(fwd_ms, 3), "tflops": round(tflops, 1), "flops": flops,
                    "frac_of_bf16_peak": round(tflops / peak_tf, 4) if peak_tf else None,
                    "dtype": "bf16 operands, f32 accumulate"},
    }


def run_cpu_plan(args):
    """The FP64 oracle timed on the host cores for the small configurations:
    the film-freezing layer (64 x 256, 2000 steps), the heated channel
    (512 x 256, 1000 steps) and the 512^2 sessile droplet (R = 100, 1000
    steps; gas density ratio 0.1), each on all cores and on one core (one core
    runs at least 200 steps and 20 s of the configuration, and its rate is
    reported).  Prints one JSON line; the GPU is not used."""
    import numpy as np

    import oracle
    from paper_2511_09422_gb300 import workloads as W
    cases = [("stefan_layer 64x256", W.stefan_layer(nx=64, ny=256), 2000),
             ("thermocapillary_channel 512x256", W.thermocapillary_channel(nx=512, ny=256), 1000),
             ("sessile_droplet 512x512 R=100", W.sessile_droplet(nx=512, ny=512, radius=100.0, rho_g=0.1), 1000)]
    all_cores = oracle.oracle.num_threads()
    out = []
    for name, w, steps in cases:
        f = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in w["fields"].items()}
        cells = w["grid"]["nx"] * w["grid"]["ny"]
        row = {"config": name, "steps": steps}
        for label, threads in (("all_cores", all_cores), ("one_core", 1)):
            oracle.oracle.set_threads(threads)
            o = oracle.Oracle(w["grid"], w["params"], f)
            o.step(1)
            t0 = time.perf_counter()
            n = 0
            while n < (steps if threads == all_cores else min(steps, 200)) or \
                    (threads == 1 and n < steps and time.perf_counter() - t0 < 20.0):
                o.step(1)
                n += 1
            dt = time.perf_counter() - t0
            row[label] = {"mlups": round(cells * n / dt / 1e6, 3), "steps_timed": n, "s": round(dt, 2),
                          "threads": oracle.oracle.num_threads()}
            o.close()
        out.append(row)
    oracle.oracle.set_threads(all_cores)
    import platform
    print(json.dumps({"metric": "FP64 oracle MLUPS on the host cores", "unit": "MLUPS", "host": platform.machine(),
                      "nproc": os.cpu_count(), "runs": out}))


def run_forward_only(args):
    """The surrogate's forward pass alone: 12 tensor-core convolutions and the
    pooling / upsampling kernels on one size x size image."""
    import numpy as np
    import torch

    from paper_2511_09422_gb300 import cno
    from paper_2511_09422_gb300 import surrogate as S
    net = cno.Net()
    net.set_params(S.init_params(0))
    rng = np.random.default_rng(0)
    x = torch.as_tensor(rng.standard_normal((1, args.size, args.size, cno.CIN)).astype(np.float32)).cuda()
    x = x.to(torch.bfloat16)
    out = torch.empty((1, args.size, args.size, cno.NF), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        net.forward(x, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        net.forward(x, out=out)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    flops = cno.forward_flops(args.size, args.size)
    peak = _peaks()[0].get("bf16_tflops")
    print(json.dumps({"metric": "surrogate forward TFLOP/s", "value": round(flops / (ms * 1e-3) / 1e12, 1),
                      "unit": "TFLOP/s", "ms": round(ms, 4), "size": args.size, "flops": flops,
                      "frac_of_bf16_peak": round(flops / (ms * 1e-3) / 1e12 / peak, 4) if peak else None,
                      "status": cno.read_status()}))
    net.close()


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2511_09422_gb300 import lbfreeze
    from paper_2511_09422_gb300 import workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    nx, ny = args.size, args.size
    w = W.impurity_front(nx=nx, ny=ny, radius=200.0 * nx / 4096.0)
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in w["fields"].items()}
    cells = nx * ny
    stream = torch.cuda.Stream()
    launches_per_step = 1  # one strip-kernel launch per step

    # ---- device-resident throughput -------------------------------------------------------
    solver = lbfreeze.Solver(w["grid"], w["params"], f32, stream=stream)
    solver.step(args.warmup)
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        e0.record(stream)
        solver.step(args.steps)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    red = solver.reduce()
    solver.close()
    if ws > 1:
        dist.barrier()
    ms_max = max_over_ranks(ms_total, dist if ws > 1 else None)
    value = whole_job_rate(cells * args.steps, ms_max * 1e-3, ws) / 1e6
    kernel_ms = ms_total / args.steps

    # ---- end to end through the public API with pinned host buffers ---------------------
    # the initial fields are copied in from pinned host memory, every step's
    # diagnostics (8 doubles) are read back, and the final fields are copied out
    pin_in = {k: torch.from_numpy(v).pin_memory() for k, v in f32.items()}
    pin_out = {k: torch.empty((ny, nx), dtype=torch.float32).pin_memory() for k in lbfreeze.FIELD_NAMES}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s2 = lbfreeze.Solver(w["grid"], w["params"], pin_in, stream=stream)
    for _ in range(args.steps):
        s2.step(1)
        s2.reduce()
    s2.fields(out=pin_out)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    s2.close()
    e2e_value = whole_job_rate(cells * args.steps, max_over_ranks(e2e_s, dist if ws > 1 else None), ws) / 1e6

    # ---- batched form: a sweep of independent droplets in one launch per step -----------
    fp16 = None
    fp16h = None
    if not args.no_fp16:
        fp16 = _fp16_leg(args, lbfreeze, w, f32, cells, torch, stream, ws, dist if ws > 1 else None,
                         _peaks()[0].get("hbm_gbs"))
        fp16h = _fp16_leg(args, lbfreeze, w, f32, cells, torch, stream, ws, dist if ws > 1 else None,
                          _peaks()[0].get("hbm_gbs"), form=2)
    d2q5 = None
    if not args.no_d2q5:
        d2q5 = _d2q5_leg(args, lbfreeze, w, f32, cells, torch, stream, ws, dist if ws > 1 else None,
                         _peaks()[0].get("hbm_gbs"))
    batched = None
    if args.batch > 0:
        batched = _batched_leg(args, lbfreeze, W, np, torch, stream, ws, dist if ws > 1 else None)
    freeze = None
    if not args.no_freeze and ws == 1:
        freeze = _freezing_leg(args, lbfreeze, W, np, torch)
    sur = None
    if args.sur_iters > 0 and ws == 1:
        sur = _surrogate_leg(args, torch, _peaks()[0])
    h2d = sum(v.numel() * 4 for v in pin_in.values()) / args.steps
    d2h = 8 * 8 + sum(v.numel() * 4 for v in pin_out.values()) / args.steps

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    peaks, src = _peaks()
    achieved = BYTES_PER_UPDATE * cells / (kernel_ms * 1e-3) / 1e9
    traffic = _traffic_per_launch(cells)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        mlups, n, cores, dt = _oracle_sample(args.size, 3, 10.0)
        cpu = {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "%d FP64 oracle steps on %s (%.1f s)" % (n, _sample_text(args.size), dt)}
    line = {
        "metric": "MLUPS (all coupled fields)", "value": round(value, 2), "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "impurity_front %dx%d (planar front + insoluble impurity r=%g, C0=0.05, Ma=10)"
                               % (nx, ny, 200.0 * nx / 4096.0),
                   "cells": cells, "l2": "working set %.1f GB >> L2 (inputs larger than L2)" % (cells * BYTES_PER_UPDATE / 2 / 1e9),
                   "parallelism": "replica per GPU" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks.get("hbm_gbs"),
                     "unit": "GB/s", "frac": round(achieved / peaks.get("hbm_gbs"), 4),
                     "peak_source": src, "bytes_per_update": BYTES_PER_UPDATE,
                     "frac_of_nameplate": round(achieved / NAMEPLATE_HBM_GBS, 4),
                     "bytes_moved_per_update": BYTES_MOVED_PER_UPDATE,
                     "frac_at_bytes_moved": round(achieved * BYTES_MOVED_PER_UPDATE / BYTES_PER_UPDATE
                                                  / peaks.get("hbm_gbs"), 4),
                     "traffic": None if traffic is None else round(traffic)},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 2), "unit": "MLUPS", "h2d_bytes_per_step": round(h2d),
                "d2h_bytes_per_step": round(d2h)},
        "gpu_launches": args.steps * launches_per_step,
        "fp16_storage": fp16,
        "fp16_h32_storage": fp16h,
        "d2q5_fl": d2q5,
        "batched": batched,
        "droplet_freezing": freeze,
        "surrogate": sur,
        "clocks": clk.summary(),
        "check": {"sum_phi": red[0], "sum_C": red[2], "front": red[5]},
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="lbfreeze", choices=["lbfreeze", "reference"])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=256, help="droplet-sweep instances of the batched leg (0: skip)")
    ap.add_argument("--no-fp16", action="store_true", help="skip the half-precision population storage leg")
    ap.add_argument("--no-d2q5", action="store_true", help="skip the D2Q5 phase-field / solute lattice leg")
    ap.add_argument("--no-freeze", action="store_true", help="skip the 512^2 droplet run to full freezing")
    ap.add_argument("--freeze-max-steps", type=int, default=600000)
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--sur-iters", type=int, default=3000, help="surrogate training iterations (0: skip the leg)")
    ap.add_argument("--sur-lattices", type=int, default=48, help="LB trajectories the surrogate is trained on")
    ap.add_argument("--sur-steps", type=int, default=12000, help="LB steps per training trajectory")
    ap.add_argument("--sur-forward-only", action="store_true",
                    help="time only the surrogate network's forward pass on a size x size lattice (He-normal "
                         "weights, random input) and print one JSON line")
    ap.add_argument("--cpu-plan", action="store_true",
                    help="time the FP64 oracle on all cores and on one core for the small configurations "
                         "(64x256 layer, 512x256 channel, 512^2 droplet) and print one JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.cpu_plan:
        run_cpu_plan(args)
    elif args.sur_forward_only:
        run_forward_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
