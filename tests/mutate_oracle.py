"""Mutation check of the LB oracle's pins (run by hand, not collected by pytest).

Each mutation is a plausible slip in the oracle -- a dropped term, a wrong
sign, index or coefficient -- applied to a copy of oracle/lb_oracle.c; the CPU
pin tests (test_oracle_pins.py, test_wetting_pins.py, test_d2q5_pins.py) are
run against the copy, and the pins that fail are listed.  A slip no pin
catches shows where the oracle is not fixed independently of itself.

    python tests/mutate_oracle.py [--workdir DIR] [index ...]

The copy lives in DIR (default tests/.mutants, which git ignores); the
oracle under oracle/ is never modified.  A full run takes about half an hour
on 8 cores.
"""
import argparse
import os
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PINS = ["conftest.py", "analytic.py", "test_oracle_pins.py", "test_wetting_pins.py", "test_d2q5_pins.py"]

# (name, text in lb_oracle.c, replacement, occurrences replaced)
M = [
 ("capillary force sign (x)", "+ alpha * sigma * muphi * gpx", "- alpha * sigma * muphi * gpx", 1),
 ("Marangoni part dropped", "alpha * (g2 * gs", "0.0 * (g2 * gs", 2),
 ("Marangoni projection sign", "g2 * gsx - gsgp * gpx", "g2 * gsx + gsgp * gpx", 1),
 ("capillary coefficient alpha 3sqrt2 eps/2", "double alpha = 3.0 * sqrt(2.0) * eps / 4.0;", "double alpha = 3.0 * sqrt(2.0) * eps / 2.0;", 1),
 ("chemical potential Laplacian sign", "/ (eps * eps) - lphi;", "/ (eps * eps) + lphi;", 1),
 ("sigma_T gradient dropped", "double gsx = p->sigma_T * gTx + p->sigma_c * gCx;", "double gsx = p->sigma_c * gCx;", 1),
 ("gravity without rho", "double Fx = Fsx + rho * p->gx, Fy = Fsy + rho * p->gy;", "double Fx = Fsx + p->gx, Fy = Fsy + p->gy;", 1),
 ("drag sign", "double ffx = -fs * usx, ffy = -fs * usy;", "double ffx = fs * usx, ffy = fs * usy;", 1),
 ("u = u* + f (no half)", "double ux = usx + 0.5 * ffx, uy = usy + 0.5 * ffy;", "double ux = usx + ffx, uy = usy + ffy;", 1),
 ("S without u.grad rho", "double S = rho * mdot + ux * grx + uy * gry;", "double S = rho * mdot;", 1),
 ("F~ without cs2 grad rho", "double Ftx = Fx - gPx + CS2 * grx + CS2 * gSx;", "double Ftx = Fx - gPx + CS2 * gSx;", 1),
 ("F~ without grad p", " - gP", " + 0.0 * gP", 2),
 ("F~ without grad p (x component only)", "double Ftx = Fx - gPx", "double Ftx = Fx + 0.0 * gPx", 1),
 ("pressure S/2 -> S", "(sg + 0.5 * S + tau_g * G0", "(sg + S + tau_g * G0", 1),
 ("pressure G0 with tau = 1", "tau_g * G0", "1.0 * G0", 1),
 ("pressure G0 with tau_f", "tau_g * G0", "tau_f * G0", 1),
 ("g equilibrium without the rest term", "geq[i] = pr / CS2 * (WT[i] - (i == 0 ? 1.0 : 0.0))", "geq[i] = pr / CS2 * WT[i]", 1),
 ("g source without (1 - 1/2tau)", "(1.0 - 0.5 / tau_g) * Gi[i]", "Gi[i]", 1),
 ("f equilibrium without velocity", "feq[i] = wfl[i] * phi * (1.0 + cu / CS2);", "feq[i] = wfl[i] * phi;", 1),
 ("F_i divergence term dropped", "+ wfl[i] * phi * divu;", ";", 1),
 ("F_i counter term sign", "double ax = dphiux + kf * nx_, ay = dphiuy + kf * ny_;", "double ax = dphiux - kf * nx_, ay = dphiuy - kf * ny_;", 1),
 ("d_t(phi u) dropped", "double dpx = phi * ux - st->phi_prev[c] * st->ux_prev[c];", "double dpx = 0.0;", 1),
 ("h0 equilibrium velocity term dropped", "- WT[0] * rhocp * T * uu / (2.0 * CS2)", "", 1),
 ("TRT times swapped", "(ha - hea) / tau_hb - (hs - hes) / tau_hs", "(ha - hea) / tau_hs - (hs - hes) / tau_hb", 1),
 ("H source factor with tau_bar", "(1.0 - 0.5 / tau_hs) * Hi[i]", "(1.0 - 0.5 / tau_hb) * Hi[i]", 1),
 ("rho H correction dropped", "double e = sh + 0.5 * st->Q_prev[c];", "double e = sh;", 1),
 ("mdot with rho_l/rho_s", "(1.0 - p->rho_s / p->rho_l) * (fs - st->fs_prev[c])", "(1.0 - p->rho_l / p->rho_s) * (fs - st->fs_prev[c])", 1),
 ("phi moment correction sign", "sf / (1.0 - 0.5 * divu)", "sf / (1.0 + 0.5 * divu)", 2),
 ("chi of Eq. Hfl from sum f with the lagged divergence", "chi = chi_of(phi);", "chi = chi_of(sf);", 1),
 ("solute R interface term sign", "(1.0 - phi) * C * nx_ / s2e", "(1.0 + phi) * C * nx_ / s2e", 1),
 ("solute R flux correction sign", "- (p->k_p - 1.0) * C * (-gf", "+ (p->k_p - 1.0) * C * (-gf", 2),
 ("k_eff rule", "double keff = 1.0 - fs * (1.0 - p->k_p);", "double keff = 1.0 - fs * p->k_p;", 1),
 ("tau_l without k_eff", "0.5 + De / (CS2 * keff)", "0.5 + De / CS2", 1),
 ("property rule solid sign", "fs * (zs - zl)", "fs * (zl - zs)", 1),
 ("latent enthalpy with rho_s (inversion only)", "double El = Al * p->T_liq + chi * p->rho_l * p->latent;\n    if (e < Es)", "double El = Al * p->T_liq + chi * p->rho_s * p->latent;\n    if (e < Es)", 1),
 ("mushy f_s without chi", "*fs = chi * (1.0 - r);", "*fs = (1.0 - r);", 1),
 ("Dirichlet stencil ghost = T_w", "return 2.0 * T_wall_bottom(g, xx) - a;", "return T_wall_bottom(g, xx);", 1),
 ("anti-bounce-back T_w at the link crossing", "T_wall_bottom(g, x) :", "T_wall_bottom(g, x + 0.5 * CX[i]) :", 1),
 ("anti-bounce-back factor 2 dropped", "2.0 * WT[i] * rr * Tw", "WT[i] * rr * Tw", 1),
 ("bounce-back without reversal", "int j = OPP[i];\n            st->f2", "int j = i;\n            st->f2", 1),
 ("wetting ghost sign", "if (kind == GHOST_PHI) return a + dphi;", "if (kind == GHOST_PHI) return a - dphi;", 1),
 ("Laplacian weight 2w -> w", "sl += 2.0 * WT[i] * (zi - z0);", "sl += WT[i] * (zi - z0);", 2),
 ("velocity wall ghost mirror", "if (kind == GHOST_VELOCITY) return -a;", "if (kind == GHOST_VELOCITY) return a;", 2),
 ("D2Q5 weights 1/4", "static const double W5[9] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0,", "static const double W5[9] = {0.0, 1.0 / 4.0, 1.0 / 4.0, 1.0 / 4.0, 1.0 / 4.0,", 1),
]


def _prepare(work):
    if os.path.exists(work):
        shutil.rmtree(work)
    os.makedirs(os.path.join(work, "tests"))
    os.makedirs(os.path.join(work, "paper_2511_09422_gb300"))
    shutil.copytree(os.path.join(HERE, "golden"), os.path.join(work, "tests", "golden"))
    for f in PINS:
        shutil.copy(os.path.join(HERE, f), os.path.join(work, "tests", f))
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2511_09422_gb300", f), os.path.join(work, "paper_2511_09422_gb300", f))
    os.makedirs(os.path.join(work, "oracle"))
    for f in ("__init__.py", "oracle.py", "cno.py", "lb_oracle.h", "lb_oracle.c"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(work, "oracle", f))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workdir", default=os.path.join(HERE, ".mutants"))
    ap.add_argument("only", nargs="*", type=int)
    args = ap.parse_args()
    work = os.path.abspath(args.workdir)
    _prepare(work)
    src = os.path.join(work, "oracle", "lb_oracle.c")
    orig = open(src).read()
    for k, (name, a, b, cnt) in enumerate(M):
        if args.only and k not in args.only:
            continue
        n = orig.count(a)
        if n != cnt:
            print("%2d %-44s SKIPPED: text found %d times, expected %d" % (k, name, n, cnt), flush=True)
            continue
        open(src, "w").write(orig.replace(a, b))
        lib = os.path.join(work, "oracle", "liblboracle.so")
        if os.path.exists(lib):
            os.remove(lib)
        t0 = time.time()
        r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                           cwd=work, capture_output=True, text=True, timeout=1800)
        fails = sorted({l.split(" ")[1].split("::")[1].split("[")[0] for l in r.stdout.splitlines()
                        if l.startswith("FAILED")})
        verdict = ("caught by " + ", ".join(fails)) if fails else "NOT CAUGHT"
        print("%2d %-44s %s (%.0f s)" % (k, name, verdict, time.time() - t0), flush=True)
    open(src, "w").write(orig)


if __name__ == "__main__":
    main()
