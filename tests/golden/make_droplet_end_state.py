"""Writes droplet_256_end_state.txt: the FP64 oracle's end state of a reduced
sessile-droplet freezing run (the 512^2, R = 100 configuration of Sec. 4.4
halved: 256^2, R = 50), which the GPU tests compare against at 1e-3.

Only the oracle is called.  The workload is seeded and synthetic
(paper_2511_09422_gb300.workloads.sessile_droplet): Ste 0.1, rho_s / rho_l
0.9, C0 0.05, Ma_T = Ma_C = 10, k_p 0.5, 90 degrees, gas density ratio 0.1,
div u the lagged velocity divergence.  The diagnostics are sampled every
SAMPLE steps; the freezing time is the first crossing of sum f_s = 0.99
sum chi, linearly interpolated between the two samples around it; the front
height (solid on the centre column) and V*_s, V*_sl are those of the sample
after the crossing, and of the sample at the end of the run.

    python tests/golden/make_droplet_end_state.py      (about 15 minutes on 8 cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "droplet_256_end_state.txt")
N, RADIUS, SAMPLE, FRAC, TAIL = 256, 50.0, 10, 0.99, 2000


def workload():
    from paper_2511_09422_gb300 import workloads as W
    return W.sessile_droplet(nx=N, ny=N, radius=RADIUS, rho_g=0.1, ste=0.1, c0=0.05, ma_T=10.0, ma_C=10.0)


def main():
    import oracle
    w = workload()
    f = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in w["fields"].items()}
    o = oracle.Oracle(w["grid"], w["params"], f)
    t0 = time.time()
    prev = None
    tf = None
    while tf is None:
        o.step(SAMPLE)
        r = o.reduce()
        g = r[3] - FRAC * r[4]
        if g >= 0.0:
            n = o.steps
            tf = (n - SAMPLE) + SAMPLE * (-prev[0]) / (g - prev[0]) if prev is not None else float(n)
            at_cross = (n, r.copy())
        prev = (g, r)
        if o.steps > 200000:
            raise SystemExit("no full freezing within 200000 steps")
    o.step(TAIL)
    end = (o.steps, o.reduce())
    lines = [
        "# FP64 oracle end state of the 256^2 sessile droplet (R = 50, Ste 0.1, C0 0.05, Ma 10, rho_g/rho_l 0.1,",
        "# divu_mode 1); written by tests/golden/make_droplet_end_state.py (oracle only, %.0f s)." % (time.time() - t0),
        "# diagnostics sampled every %d steps; t_f: first crossing of sum f_s = %.2f sum chi, interpolated" % (SAMPLE, FRAC),
        "sample_every = %d" % SAMPLE,
        "t_f = %.6f" % tf,
        "cross_step = %d" % at_cross[0],
        "front_at_cross = %.9f" % at_cross[1][5],
        "Vs_at_cross = %.9f" % at_cross[1][6],
        "Vsl_at_cross = %.9f" % at_cross[1][7],
        "end_step = %d" % end[0],
        "front_at_end = %.9f" % end[1][5],
        "Vs_at_end = %.9f" % end[1][6],
        "Vsl_at_end = %.9f" % end[1][7],
    ]
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
