/*
 * lb_oracle.c -- FP64 CPU oracle of one time step of the diffuse-interface
 * lattice Boltzmann (LB) method for gas-liquid-solid freezing of a binary
 * fluid with Marangoni flow (Huang, Chai, Liu, Huang, arXiv 2511.09422).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the GPU library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the GPU
 * library never links it and shares no code, table or header with it.
 *
 * Everything is IEEE double precision, compiled without fast-math and with
 * FMA contraction disabled, so x86 and Arm hosts give the same bits.
 *
 * Method, in the paper's order (Sec. 3):
 *   - four D2Q9 distribution sets: phase field f (Sec. 3.1, BGK),
 *     pressure-based flow g (Sec. 3.2, BGK), total enthalpy h (Sec. 3.3,
 *     two-relaxation-time), solute l (Sec. 3.4, BGK);
 *   - macroscopic variables from the moments of the post-streaming
 *     populations, the temperature and solid fraction from the enthalpy
 *     (Eq. Hfl), properties by the linear rule zeta(phi, f_s) (end of Sec. 2);
 *   - gradients and Laplacians by the second-order isotropic difference
 *     schemes on the D2Q9 neighbourhood (end of Sec. 3.4);
 *   - forces: continuum surface force split into Marangoni and capillary
 *     parts (Eq. Fs), body force, solid-liquid interaction force (Sec. 3.2);
 *   - collision, then streaming with half-way bounce-back walls (no slip,
 *     no flux) and anti-bounce-back for a Dirichlet temperature (Sec. 4.5),
 *     periodic in x.
 *
 * Where the paper is silent or garbled, the reading taken is stated at the
 * line that uses it.  State layout: populations post-streaming, [i*n + c]
 * with c = y*nx + x; lagged auxiliary fields of the previous step.
 *
 * Parity pins (what fixes each part independently of this code) live in the
 * CPU test-suite; every function here is pinned there, and
 * tests/mutate_oracle.py lists which planted slips the pins catch.  One term
 * is parity unpinned on its own: the x component of -grad p in the effective
 * force F~ of pass_local (no closed form puts a steady pressure gradient along
 * the periodic x beside a flow along x); its y component, the same arithmetic,
 * is pinned by a body force across a channel flow.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lb_oracle.h"

/* D2Q9 velocity set: c_0 = (0,0); c_1..4 = (1,0),(0,1),(-1,0),(0,-1);
 * c_5..8 = (1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36; c_s^2 = 1/3. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
#define CS2 (1.0 / 3.0)
#define PI_D 3.14159265358979323846

struct orc_state {
    orc_grid g;
    orc_params p;
    long n;
    long step;
    double *f, *gq, *h, *l;     /* post-streaming populations, 9*n each */
    double *f2, *g2, *h2, *l2;  /* streaming destinations */
    /* lagged auxiliary state written by the previous step */
    double *fs_prev, *Q_prev, *phi_prev, *C_prev;
    double *ux_prev, *uy_prev, *p_prev, *S_prev;
    double *ux_new, *uy_new, *p_new, *S_new;
    /* per-step local macroscopic fields */
    double *phi, *T, *fs, *C, *rhoH, *mdot, *divu, *rho;
    double V0;
};

/* ------------------------------------------------------------------ */
/* Properties, enthalpy relation                                        */
/* ------------------------------------------------------------------ */

/* Linear interpolation rule for rho, mu, lambda, C_p (end of Sec. 2):
 * zeta = phi (zl - zg)/2 + f_s (zs - zl) + (zl + zg)/2. */
double orc_zeta(double phi, double fs, double zl, double zs, double zg)
{
    return 0.5 * phi * (zl - zg) + fs * (zs - zl) + 0.5 * (zl + zg);
}

/* Volumetric heat capacity rho C_p of the advective terms of the enthalpy set
 * (the h equilibrium and the source Q).  rhocp_rule 0 (the reading taken):
 * the linear property rule applied to the product rho C_p of each phase.
 * rhocp_rule 1 (the literal reading, for comparison only): the rule applied
 * to rho and to C_p apart and the two multiplied, which peaks inside the
 * interface when the phases have equal rho C_p but different densities. */
static double rhocp_of(const orc_params *p, double phi, double fs)
{
    if (p->rhocp_rule == 1)
        return orc_zeta(phi, fs, p->rho_l, p->rho_s, p->rho_g) * orc_zeta(phi, fs, p->cp_l, p->cp_s, p->cp_g);
    return orc_zeta(phi, fs, p->rho_l * p->cp_l, p->rho_s * p->cp_s, p->rho_g * p->cp_g);
}

/* Fraction of phase-change material from the order parameter, clamped. */
static double chi_of(double phi)
{
    double c = 0.5 * (1.0 + phi);
    return c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
}

/* Enthalpy -> (T, f_s), Eq. Hfl.  The paper writes it for the pure
 * phase-change material (chi = 1).  Reading taken for the interface and gas:
 * the solidus/liquidus enthalpies are chi-weighted mixtures,
 *   A_s = chi rho_s Cp_s + (1-chi) rho_g Cp_g,  E_s = A_s T_s,
 *   A_l = chi rho_l Cp_l + (1-chi) rho_g Cp_g,  E_l = A_l T_l + chi rho_l L,
 * and f_s ranges over [0, chi] (no solid in the gas).  At chi = 1 this is
 * Eq. Hfl exactly, with f_s = 1 - f_l.  With phase change switched off the
 * latent term is dropped and f_s = 0. */
void orc_enthalpy_invert(const orc_params *p, double e, double chi, double *T, double *fs)
{
    double Al = chi * p->rho_l * p->cp_l + (1.0 - chi) * p->rho_g * p->cp_g;
    if (!p->phase_change_on) {
        *T = e / Al;
        *fs = 0.0;
        return;
    }
    double As = chi * p->rho_s * p->cp_s + (1.0 - chi) * p->rho_g * p->cp_g;
    double Es = As * p->T_sol;
    double El = Al * p->T_liq + chi * p->rho_l * p->latent;
    if (e < Es) {
        *fs = chi;
        *T = e / As;
    } else if (e > El) {
        *fs = 0.0;
        *T = p->T_liq + (e - El) / Al;
    } else {
        double d = El - Es, r;
        double scale = fabs(e) > 1.0 ? fabs(e) : 1.0;
        if (d < 1e-14 * scale)
            r = 1.0; /* degenerate mushy range (gas, or T_s = T_l with L = 0) */
        else
            r = (e - Es) / d;
        *fs = chi * (1.0 - r);
        *T = p->T_sol + r * (p->T_liq - p->T_sol);
    }
}

/* Forward map (T, chi) -> enthalpy, the inverse of orc_enthalpy_invert on
 * its range; a temperature exactly at T_s = T_l is taken as liquid. */
double orc_enthalpy_forward(const orc_params *p, double T, double chi)
{
    double Al = chi * p->rho_l * p->cp_l + (1.0 - chi) * p->rho_g * p->cp_g;
    if (!p->phase_change_on) return Al * T;
    double As = chi * p->rho_s * p->cp_s + (1.0 - chi) * p->rho_g * p->cp_g;
    double Es = As * p->T_sol;
    double El = Al * p->T_liq + chi * p->rho_l * p->latent;
    if (T >= p->T_liq) return El + Al * (T - p->T_liq);
    if (T < p->T_sol) return As * T;
    double r = (T - p->T_sol) / (p->T_liq - p->T_sol);
    return Es + r * (El - Es);
}

/* Reference heat capacity of Sec. 3.3: C_p,ref = 2 Cp_s Cp_l / (Cp_s + Cp_l).
 * rho_ref is not defined by the paper; it is taken as rho_l, which makes the
 * enthalpy equilibria sum to rho H exactly (see orc_equilibria). */
static double rhocp_ref(const orc_params *p)
{
    double cpref = 2.0 * p->cp_s * p->cp_l / (p->cp_s + p->cp_l);
    return p->rho_l * cpref;
}

/* ------------------------------------------------------------------ */
/* Equilibria and discrete source terms (Sec. 3.1 - 3.4)                */
/* ------------------------------------------------------------------ */

/* s_i(u) of Sec. 3.2. */
static double s_of(int i, double ux, double uy)
{
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WT[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* All four equilibria of one cell.
 *  f_eq = w phi (1 + c.u/cs2)                                  (Sec. 3.1)
 *  g_eq = p/cs2 (w_i - 1[i=0]) + rho s_i(u)                    (Sec. 3.2)
 *  h_eq_0 = rhoH - rRef T + w_0 rRef T - w_0 rhoCp T u.u/(2cs2)
 *  h_eq_i = w_i [rRef T + rhoCp T (c.u/cs2 + ((c.u)^2 - cs2 u.u)/(2 cs2^2))]
 *          with rRef = rho_ref Cp_ref                           (Sec. 3.3)
 *  l_eq = w C (1 + c.u/cs2)                                     (Sec. 3.4)
 * The i = 0 enthalpy term is printed "rho H - rho C_p,ref T"; it is read with
 * rho_ref so that sum_i h_eq_i = rho H holds exactly. */
/* Weights of the phase-field and solute sets.  The paper does not name their
 * lattice (D2Q9 is read everywhere; Sec. 3).  D2Q5 is the five velocities
 * c_0 .. c_4 of D2Q9 with weights 1/3 and 1/6: written here as D2Q9 with zero
 * diagonal weights, whose populations 5 .. 8 then stay zero; both lattices have
 * c_s^2 = 1/3 and the same first moments, which is all the equilibria and
 * sources of f and l use. */
static const double W5[9] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 0.0, 0.0, 0.0, 0.0};
static const double *weights_fl(const orc_params *p) { return p->lattice_fl == 1 ? W5 : WT; }

static void equilibria_w(const orc_params *p, const double *wfl, double phi, double C, double rhoH, double T,
                         double pr, double ux, double uy, double rho, double rhocp,
                         double feq[9], double geq[9], double heq[9], double leq[9]);

void orc_equilibria(const orc_params *p, double phi, double C, double rhoH, double T,
                    double pr, double ux, double uy, double rho, double rhocp,
                    double feq[9], double geq[9], double heq[9], double leq[9])
{
    equilibria_w(p, WT, phi, C, rhoH, T, pr, ux, uy, rho, rhocp, feq, geq, heq, leq);
}

static void equilibria_w(const orc_params *p, const double *wfl, double phi, double C, double rhoH, double T,
                         double pr, double ux, double uy, double rho, double rhocp,
                         double feq[9], double geq[9], double heq[9], double leq[9])
{
    double rr = rhocp_ref(p);
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = wfl[i] * phi * (1.0 + cu / CS2);
        leq[i] = wfl[i] * C * (1.0 + cu / CS2);
        geq[i] = pr / CS2 * (WT[i] - (i == 0 ? 1.0 : 0.0)) + rho * s_of(i, ux, uy);
        if (i == 0)
            heq[i] = rhoH - rr * T + WT[0] * rr * T - WT[0] * rhocp * T * uu / (2.0 * CS2);
        else
            heq[i] = WT[i] * (rr * T + rhocp * T * (cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2)));
    }
}

/* Discrete sources of one cell.
 *  F_i = w c.[d_t(phi u) + cs2 n (1-phi^2)/(sqrt2 eps)]/cs2 + w phi div u  (Sec. 3.1)
 *  G_i = w [S + c.(F + rho f)/cs2 + (u Ft + Ft u):(c c - cs2 I)/(2 cs2^2)] (Sec. 3.2)
 *  H_i = w Q,  Q = rho Cp T div u                                         (Sec. 3.3)
 *  L_i = w c.[d_t(C u) + cs2 R]/cs2                                       (Sec. 3.4)
 * H_i is printed without the weight w_i, which is read as a typo (its zeroth
 * moment must be Q).  ``divu`` is the velocity divergence (see pass_local). */
static void sources_w(const double *wfl, double dphiux, double dphiuy, double nx_, double ny_, double phi,
                      double eps, double divu, double S, double Fx, double Fy, double rfx, double rfy,
                      double Ftx, double Fty, double ux, double uy, double Q,
                      double dCux, double dCuy, double Rx, double Ry,
                      double Fi[9], double Gi[9], double Hi[9], double Li[9]);

void orc_sources(double dphiux, double dphiuy, double nx_, double ny_, double phi, double eps,
                 double divu, double S, double Fx, double Fy, double rfx, double rfy,
                 double Ftx, double Fty, double ux, double uy, double Q,
                 double dCux, double dCuy, double Rx, double Ry,
                 double Fi[9], double Gi[9], double Hi[9], double Li[9])
{
    sources_w(WT, dphiux, dphiuy, nx_, ny_, phi, eps, divu, S, Fx, Fy, rfx, rfy, Ftx, Fty, ux, uy, Q, dCux, dCuy,
              Rx, Ry, Fi, Gi, Hi, Li);
}

static void sources_w(const double *wfl, double dphiux, double dphiuy, double nx_, double ny_, double phi,
                      double eps, double divu, double S, double Fx, double Fy, double rfx, double rfy,
                      double Ftx, double Fty, double ux, double uy, double Q,
                      double dCux, double dCuy, double Rx, double Ry,
                      double Fi[9], double Gi[9], double Hi[9], double Li[9])
{
    double kf = CS2 * (1.0 - phi * phi) / (sqrt(2.0) * eps);
    double ax = dphiux + kf * nx_, ay = dphiuy + kf * ny_;
    double bx = dCux + CS2 * Rx, by = dCuy + CS2 * Ry;
    double uF = ux * Ftx + uy * Fty;
    for (int i = 0; i < 9; i++) {
        double cx = CX[i], cy = CY[i];
        double cu = cx * ux + cy * uy, cF = cx * Ftx + cy * Fty;
        Fi[i] = wfl[i] * (cx * ax + cy * ay) / CS2 + wfl[i] * phi * divu;
        /* (u Ft + Ft u):(c c - cs2 I) = 2 (c.u)(c.Ft) - 2 cs2 u.Ft */
        Gi[i] = WT[i] * (S + (cx * (Fx + rfx) + cy * (Fy + rfy)) / CS2 +
                         (2.0 * cu * cF - 2.0 * CS2 * uF) / (2.0 * CS2 * CS2));
        Hi[i] = WT[i] * Q;
        Li[i] = wfl[i] * (cx * bx + cy * by) / CS2;
    }
}

/* ------------------------------------------------------------------ */
/* Neighbourhood access with the wall ghosts used by the stencils        */
/* ------------------------------------------------------------------ */

/* Wall temperature of the bottom wall at continuous abscissa x
 * (cell centres at integer x): T_b + A cos(2 pi m x / nx). */
static double T_wall_bottom(const orc_grid *g, double x)
{
    if (g->T_bottom_amp == 0.0) return g->T_bottom;
    return g->T_bottom + g->T_bottom_amp * cos(2.0 * PI_D * g->T_bottom_modes * x / g->nx);
}

/* Value of field v at (x + dx, y + dy), x periodic.  Rows outside the domain
 * are ghosts of the half-way walls at y = -1/2 and y = ny - 1/2, built by
 * linear extrapolation through the wall value: 2 v_w - v_adjacent for a field
 * with a prescribed wall value (the temperature at a Dirichlet wall; the
 * velocity, v_w = 0 at a no-slip wall), and a mirror v_adjacent for a field
 * with zero normal gradient (everything else; for phi and rho this is the
 * 90-degree contact angle, other angles are in nb_st below). */
#define GHOST_MIRROR 0
#define GHOST_TEMPERATURE 1
#define GHOST_VELOCITY 2
static double nb(const orc_grid *g, const double *v, int x, int y, int dx, int dy, int kind)
{
    int xx = ((x + dx) % g->nx + g->nx) % g->nx;
    int yy = y + dy;
    if (yy < 0) {
        double a = v[(long)0 * g->nx + xx];
        if (kind == GHOST_TEMPERATURE && g->bc_bottom == ORC_WALL_DIRICHLET_T)
            return 2.0 * T_wall_bottom(g, xx) - a;
        if (kind == GHOST_VELOCITY) return -a;
        return a;
    }
    if (yy >= g->ny) {
        double a = v[(long)(g->ny - 1) * g->nx + xx];
        if (kind == GHOST_TEMPERATURE && g->bc_top == ORC_WALL_DIRICHLET_T)
            return 2.0 * g->T_top - a;
        if (kind == GHOST_VELOCITY) return -a;
        return a;
    }
    return v[(long)yy * g->nx + xx];
}

/* Wetting (contact angle theta at a wall, Sec. 3.4; the paper cites the
 * treatment without printing it).  For the equilibrium profile
 * phi = tanh(2 d / W) = tanh(d / (sqrt 2 eps)) meeting the wall at angle
 * theta (measured inside the phi = 1 phase), the derivative along the wall
 * normal n_w pointing into the fluid is
 *     n_w . grad phi = -cos(theta) (1 - phi^2) / (sqrt 2 eps).
 * The ghost of phi beyond the half-way wall follows from that derivative
 * across the half cell on each side of the wall, with phi at the wall taken
 * as the adjacent value a:  phi_ghost = a + cos(theta) (1 - a^2) / (sqrt 2 eps)
 * (cos theta = 0 is the mirror, 90 degrees).  The density ghost follows
 * from the phi ghost by the linear rule: rho_ghost = rho_a + (rho_l - rho_g)/2
 * (phi_ghost - a).  Other fields keep the ghosts of nb(). */
#define GHOST_PHI 3
#define GHOST_RHO 4
static double nb_st(const orc_state *st, const double *v, int x, int y, int dx, int dy, int kind)
{
    const orc_grid *g = &st->g;
    int yy = y + dy;
    if ((kind != GHOST_PHI && kind != GHOST_RHO) || (yy >= 0 && yy < g->ny))
        return nb(g, v, x, y, dx, dy, kind == GHOST_PHI || kind == GHOST_RHO ? GHOST_MIRROR : kind);
    int xx = ((x + dx) % g->nx + g->nx) % g->nx;
    int ya = yy < 0 ? 0 : g->ny - 1;
    double ct = yy < 0 ? g->cos_theta_bottom : g->cos_theta_top;
    double phi_a = st->phi[(long)ya * g->nx + xx];
    double dphi = ct * (1.0 - phi_a * phi_a) / (sqrt(2.0) * st->p.eps);
    double a = v[(long)ya * g->nx + xx];
    if (kind == GHOST_PHI) return a + dphi;
    return a + 0.5 * (st->p.rho_l - st->p.rho_g) * dphi;
}

/* Second-order isotropic schemes (end of Sec. 3.4), dx = dt = 1:
 *   grad z = sum_{i != 0} w_i c_i z(x + c_i) / cs2
 *   lap  z = sum_{i != 0} 2 w_i [z(x + c_i) - z(x)] / cs2                  */
static void stencil(const orc_grid *g, const double *v, int x, int y, int kind,
                    double *gx, double *gy, double *lap)
{
    double z0 = v[(long)y * g->nx + x];
    double sx = 0, sy = 0, sl = 0;
    for (int i = 1; i < 9; i++) {
        double zi = nb(g, v, x, y, CX[i], CY[i], kind);
        sx += WT[i] * CX[i] * zi;
        sy += WT[i] * CY[i] * zi;
        sl += 2.0 * WT[i] * (zi - z0);
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
    if (lap) *lap = sl / CS2;
}

/* The same schemes with the wetting ghosts of nb_st(). */
static void stencil_st(const orc_state *st, const double *v, int x, int y, int kind,
                       double *gx, double *gy, double *lap)
{
    double z0 = v[(long)y * st->g.nx + x];
    double sx = 0, sy = 0, sl = 0;
    for (int i = 1; i < 9; i++) {
        double zi = nb_st(st, v, x, y, CX[i], CY[i], kind);
        sx += WT[i] * CX[i] * zi;
        sy += WT[i] * CY[i] * zi;
        sl += 2.0 * WT[i] * (zi - z0);
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
    if (lap) *lap = sl / CS2;
}

void orc_stencil_field(const orc_grid *g, const double *v, int kind, double *gx, double *gy, double *lap)
{
    for (int y = 0; y < g->ny; y++)
        for (int x = 0; x < g->nx; x++) {
            long c = (long)y * g->nx + x;
            stencil(g, v, x, y, kind, &gx[c], &gy[c], &lap[c]);
        }
}

/* ------------------------------------------------------------------ */
/* Creation                                                             */
/* ------------------------------------------------------------------ */

static double *alloc0(long n)
{
    return (double *)calloc((size_t)n, sizeof(double));
}

orc_state *orc_create(const orc_grid *g, const orc_params *p, const double *phi0,
                      const double *T0, const double *C0, const double *ux0, const double *uy0)
{
    if (g->nx < 1 || g->ny < 1) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    st->g = *g;
    st->p = *p;
    long n = (long)g->nx * g->ny;
    st->n = n;
    st->f = alloc0(9 * n); st->gq = alloc0(9 * n); st->h = alloc0(9 * n); st->l = alloc0(9 * n);
    st->f2 = alloc0(9 * n); st->g2 = alloc0(9 * n); st->h2 = alloc0(9 * n); st->l2 = alloc0(9 * n);
    st->fs_prev = alloc0(n); st->Q_prev = alloc0(n); st->phi_prev = alloc0(n); st->C_prev = alloc0(n);
    st->ux_prev = alloc0(n); st->uy_prev = alloc0(n); st->p_prev = alloc0(n); st->S_prev = alloc0(n);
    st->ux_new = alloc0(n); st->uy_new = alloc0(n); st->p_new = alloc0(n); st->S_new = alloc0(n);
    st->phi = alloc0(n); st->T = alloc0(n); st->fs = alloc0(n); st->C = alloc0(n);
    st->rhoH = alloc0(n); st->mdot = alloc0(n); st->divu = alloc0(n); st->rho = alloc0(n);

    /* Initial state: post-streaming populations equal to the equilibria of
     * the initial fields with p = 0; the enthalpy from the forward map;
     * lagged fields consistent with a state at rest in time. */
    double V0 = 0.0;
    for (long c = 0; c < n; c++) {
        double ph = phi0[c], T = T0[c], C = C0[c];
        double ux = ux0 ? ux0[c] : 0.0, uy = uy0 ? uy0[c] : 0.0;
        double chi = chi_of(ph);
        double e = orc_enthalpy_forward(p, T, chi);
        double Tc, fs;
        orc_enthalpy_invert(p, e, chi, &Tc, &fs);
        double rho = orc_zeta(ph, fs, p->rho_l, p->rho_s, p->rho_g);
        double rhocp = rhocp_of(p, ph, fs);
        double feq[9], geq[9], heq[9], leq[9];
        equilibria_w(p, weights_fl(p), ph, C, e, Tc, 0.0, ux, uy, rho, rhocp, feq, geq, heq, leq);
        for (int i = 0; i < 9; i++) {
            st->f[i * n + c] = feq[i];
            st->gq[i * n + c] = geq[i];
            st->h[i * n + c] = heq[i];
            st->l[i * n + c] = leq[i];
        }
        st->fs_prev[c] = fs;
        st->Q_prev[c] = 0.0;
        st->phi_prev[c] = ph;
        st->C_prev[c] = C;
        st->ux_prev[c] = ux;
        st->uy_prev[c] = uy;
        V0 += chi;
    }
    st->V0 = V0;
    return st;
}

void orc_destroy(orc_state *st)
{
    if (!st) return;
    double *ptrs[] = {st->f, st->gq, st->h, st->l, st->f2, st->g2, st->h2, st->l2,
                      st->fs_prev, st->Q_prev, st->phi_prev, st->C_prev, st->ux_prev,
                      st->uy_prev, st->p_prev, st->S_prev, st->ux_new, st->uy_new, st->p_new,
                      st->S_new, st->phi, st->T, st->fs, st->C, st->rhoH, st->mdot, st->divu,
                      st->rho};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); k++) free(ptrs[k]);
    free(st);
}

/* ------------------------------------------------------------------ */
/* Step, part 1: local macroscopic variables of every cell              */
/* ------------------------------------------------------------------ */

/* Per cell, in this order:
 *   rho H = sum h_i + Q^{n-1}/2  (Sec. 3.3; the correction needs this step's
 *           T, which depends on rho H, so the previous step's Q is used);
 *   T, f_s from the enthalpy (Eq. Hfl) with the material fraction chi =
 *           clamp((1 + phi)/2): phi from the moment below when div u is the
 *           lagged velocity divergence (known before the enthalpy), sum f_i in
 *           place of phi when div u = mdot (which needs f_s first);
 *   mdot = (1 - rho_s/rho_l) d_t f_s, backward difference (Eq. NS1);
 *   div u, the velocity divergence in the phase-field and enthalpy sources
 *           and moment corrections (Sec. 3.1, 3.3): by default the model
 *           value mdot of Eq. NS1, which keeps sum phi exactly conserved
 *           without phase change (the conservative phase-field model).  With
 *           divu_mode = 1 it is the isotropic divergence of the previous
 *           step's velocity instead (this step's velocity is not known at the
 *           neighbours yet), which also follows the compression of the
 *           surrounding phase by the volume change in a closed box;
 *   phi = sum f_i + phi div u / 2, solved for phi (Sec. 3.1);
 *   C = sum l_i (Sec. 3.4);  rho = zeta(phi, f_s).
 * The source Q = rho Cp T div u is formed in the collision pass. */
static void pass_local(orc_state *st)
{
    const orc_params *p = &st->p;
    const orc_grid *g = &st->g;
    long n = st->n;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) {
        int x = (int)(c % g->nx), y = (int)(c / g->nx);
        double sf = 0, sh = 0, sl = 0;
        for (int i = 0; i < 9; i++) {
            sf += st->f[i * n + c];
            sh += st->h[i * n + c];
            sl += st->l[i * n + c];
        }
        double e = sh + 0.5 * st->Q_prev[c];
        double T, fs, divu = 0.0, phi = 0.0, chi;
        if (p->divu_mode == 1) {
            /* div u known before the enthalpy: phi first, and the material
             * fraction of the enthalpy relation from phi itself, as in the
             * property rule */
            double dxx, dxy, dyx, dyy;
            stencil(g, st->ux_prev, x, y, GHOST_VELOCITY, &dxx, &dxy, NULL);
            stencil(g, st->uy_prev, x, y, GHOST_VELOCITY, &dyx, &dyy, NULL);
            divu = dxx + dyy;
            phi = sf / (1.0 - 0.5 * divu);
            chi = chi_of(phi);
        } else {
            /* div u = mdot needs f_s, which needs the enthalpy relation: the
             * material fraction is taken from sum f_i */
            chi = chi_of(sf);
        }
        orc_enthalpy_invert(p, e, chi, &T, &fs);
        double mdot = p->phase_change_on ? (1.0 - p->rho_s / p->rho_l) * (fs - st->fs_prev[c]) : 0.0;
        if (p->divu_mode != 1) {
            divu = mdot;
            phi = sf / (1.0 - 0.5 * divu);
        }
        st->divu[c] = divu;
        st->rhoH[c] = e;
        st->T[c] = T;
        st->fs[c] = fs;
        st->mdot[c] = mdot;
        st->phi[c] = phi;
        st->C[c] = sl;
        st->rho[c] = orc_zeta(phi, fs, p->rho_l, p->rho_s, p->rho_g);
    }
}

/* ------------------------------------------------------------------ */
/* Step, part 2: gradients, forces, velocity, pressure, collision        */
/* ------------------------------------------------------------------ */

typedef struct {
    double ux, uy, p, S, Q;
    double fpc[9], gpc[9], hpc[9], lpc[9]; /* post-collision populations */
} cell_out;

static void cell_dynamics(const orc_state *st, int x, int y, cell_out *o)
{
    const orc_grid *g = &st->g;
    const orc_params *p = &st->p;
    long n = st->n;
    long c = (long)y * g->nx + x;
    double phi = st->phi[c], T = st->T[c], fs = st->fs[c], C = st->C[c];
    double rhoH = st->rhoH[c], mdot = st->mdot[c], divu = st->divu[c], rho = st->rho[c];
    double eps = p->eps;

    /* stencils of the current fields and of the lagged p, S */
    double gpx, gpy, lphi, gTx, gTy, gCx, gCy, gfx, gfy, grx, gry, gPx, gPy, gSx, gSy;
    stencil_st(st, st->phi, x, y, GHOST_PHI, &gpx, &gpy, &lphi);
    stencil(g, st->T, x, y, GHOST_TEMPERATURE, &gTx, &gTy, NULL);
    stencil(g, st->C, x, y, GHOST_MIRROR, &gCx, &gCy, NULL);
    stencil(g, st->fs, x, y, GHOST_MIRROR, &gfx, &gfy, NULL);
    stencil_st(st, st->rho, x, y, GHOST_RHO, &grx, &gry, NULL);
    stencil(g, st->p_prev, x, y, GHOST_MIRROR, &gPx, &gPy, NULL);
    stencil(g, st->S_prev, x, y, GHOST_MIRROR, &gSx, &gSy, NULL);

    /* properties */
    double mu = orc_zeta(phi, fs, p->mu_l, p->mu_s, p->mu_g);
    double lam = orc_zeta(phi, fs, p->lam_l, p->lam_s, p->lam_g);
    /* The linear rule is applied to the volumetric heat capacity rho C_p,
     * the product that enters Eq. Tem; interpolating rho and C_p separately
     * and multiplying would make rho C_p peak inside the interface when the
     * phases have equal rho C_p but very different densities.  This is the
     * same chi-weighted mixture that the enthalpy relation uses. */
    double rhocp = rhocp_of(p, phi, fs);

    /* unit normal n = grad phi / |grad phi| (Eq. 1), undefined where
     * grad phi = 0.  Regularised as grad phi / sqrt(|grad phi|^2 + 1e-6): the
     * normal only matters in the interface, where the counter term's factor
     * (1 - phi^2)/(sqrt2 eps) equals |grad phi| on the equilibrium profile, so
     * for |phi| < 0.99 the normal is unbiased to better than 1%; away from the
     * interface the product (1 - phi^2) n fades smoothly instead of taking a
     * random direction from round-off gradients, which would make the scheme
     * amplify 1e-7 perturbations to 1e-3 within 100 steps. */
    double g2 = gpx * gpx + gpy * gpy;
    double inv = 1.0 / sqrt(g2 + 1e-6);
    double nx_ = gpx * inv, ny_ = gpy * inv;

    /* chemical potential with phi1 = 1, phi2 = -1, k = 1, beta = 1/(4 eps^2):
     * mu_phi = (phi^3 - phi)/eps^2 - lap phi */
    double muphi = (phi * phi * phi - phi) / (eps * eps) - lphi;

    /* surface tension, linear equation of state, and its gradient */
    double sigma = p->sigma0 + p->sigma_T * (T - p->T_ref) + p->sigma_c * (C - p->c_ref);
    double gsx = p->sigma_T * gTx + p->sigma_c * gCx;
    double gsy = p->sigma_T * gTy + p->sigma_c * gCy;

    /* Eq. Fs with alpha = 3 sqrt(2) eps / 4.  The capillary part is printed
     * with an extra sigma/eps^2 factor although mu_phi already carries
     * 1/eps^2; it is read as alpha sigma mu_phi grad phi, which is the
     * preceding line of Eq. Fs on the equilibrium profile and gives the
     * Laplace jump sigma/R.  Multiplied by (1 - f_s) when the modified
     * surface tension of Sec. 4.5 is selected. */
    double alpha = 3.0 * sqrt(2.0) * eps / 4.0;
    double gsgp = gsx * gpx + gsy * gpy;
    double Fsx = alpha * (g2 * gsx - gsgp * gpx) + alpha * sigma * muphi * gpx;
    double Fsy = alpha * (g2 * gsy - gsgp * gpy) + alpha * sigma * muphi * gpy;
    if (p->fs_modulated_st) {
        Fsx *= (1.0 - fs);
        Fsy *= (1.0 - fs);
    }
    /* total force F = F_s + F_b, body force rho g */
    double Fx = Fsx + rho * p->gx, Fy = Fsy + rho * p->gy;

    /* velocity: rho u* = sum c_i g_i + F/2; f = f_s (0 - u*); u = u* + f/2 */
    double jx = 0, jy = 0, sg = 0;
    for (int i = 0; i < 9; i++) {
        double gi = st->gq[i * n + c];
        jx += CX[i] * gi;
        jy += CY[i] * gi;
        if (i) sg += gi;
    }
    double usx = (jx + 0.5 * Fx) / rho, usy = (jy + 0.5 * Fy) / rho;
    double ffx = -fs * usx, ffy = -fs * usy;
    double ux = usx + 0.5 * ffx, uy = usy + 0.5 * ffy;
    double rfx = rho * ffx, rfy = rho * ffy;

    /* mass source S = rho mdot + u.grad rho */
    double S = rho * mdot + ux * grx + uy * gry;

    /* effective force Ft = F - grad p + cs2 grad rho + cs2 grad S.  grad p and
     * grad S need p and S of the neighbours, which in turn need Ft; the
     * previous step's p and S are used.  The printed "cs2 div S" of a scalar
     * is read as cs2 grad S. */
    double Ftx = Fx - gPx + CS2 * grx + CS2 * gSx;
    double Fty = Fy - gPy + CS2 * gry + CS2 * gSy;

    /* relaxation times (Sec. 3.1-3.4), with eta = 1 in M = eta cs2 (tau_f - 1/2) */
    double tau_f = 0.5 + p->mobility / CS2;
    double tau_g = 0.5 + mu / (rho * CS2);
    double tau_hb = 0.5 + lam / (rhocp_ref(p) * CS2);
    double tau_hs = 1.0 / (2.0 - 1.0 / tau_hb);
    double keff = 1.0 - fs * (1.0 - p->k_p);
    double De = fs * p->k_p * p->D_s + (1.0 - fs) * p->D_l;
    double tau_l = 0.5 + De / (CS2 * keff);

    /* pressure (Sec. 3.2), G_0 = w_0 [S - u.Ft/cs2], tau = tau_g */
    double G0 = WT[0] * (S - (ux * Ftx + uy * Fty) / CS2);
    double pr = CS2 / (1.0 - WT[0]) * (sg + 0.5 * S + tau_g * G0 + rho * s_of(0, ux, uy));

    /* time derivatives by backward differences over one step */
    double dpx = phi * ux - st->phi_prev[c] * st->ux_prev[c];
    double dpy = phi * uy - st->phi_prev[c] * st->uy_prev[c];
    double dcx = C * ux - st->C_prev[c] * st->ux_prev[c];
    double dcy = C * uy - st->C_prev[c] * st->uy_prev[c];

    /* solute flux correction R (Sec. 3.4), as printed */
    double s2e = sqrt(2.0) * eps;
    double Rx = (1.0 - phi) * C * nx_ / s2e - (p->k_p - 1.0) * C * (-gfx) / keff;
    double Ry = (1.0 - phi) * C * ny_ / s2e - (p->k_p - 1.0) * C * (-gfy) / keff;

    double Q = rhocp * T * divu;

    double feq[9], geq[9], heq[9], leq[9], Fi[9], Gi[9], Hi[9], Li[9];
    equilibria_w(p, weights_fl(p), phi, C, rhoH, T, pr, ux, uy, rho, rhocp, feq, geq, heq, leq);
    sources_w(weights_fl(p), dpx, dpy, nx_, ny_, phi, eps, divu, S, Fx, Fy, rfx, rfy, Ftx, Fty, ux, uy, Q,
              dcx, dcy, Rx, Ry, Fi, Gi, Hi, Li);

    double hloc[9];
    for (int i = 0; i < 9; i++) hloc[i] = st->h[i * n + c];
    for (int i = 0; i < 9; i++) {
        double fi = st->f[i * n + c], gi = st->gq[i * n + c], li = st->l[i * n + c];
        o->fpc[i] = fi - (fi - feq[i]) / tau_f + (1.0 - 0.5 / tau_f) * Fi[i];
        o->gpc[i] = gi - (gi - geq[i]) / tau_g + (1.0 - 0.5 / tau_g) * Gi[i];
        o->lpc[i] = li - (li - leq[i]) / tau_l + (1.0 - 0.5 / tau_l) * Li[i];
        /* two-relaxation-time enthalpy collision: antisymmetric part with
         * tau_bar (sets the conductivity), symmetric part with tau_tilde,
         * 1/tau_tilde + 1/tau_bar = 2.  The isotropic source H_i is purely
         * symmetric and is weighted with (1 - 1/(2 tau_tilde)); the printed
         * tau_bar there would break rho H = sum h + Q/2 at second order. */
        int j = OPP[i];
        double hs = 0.5 * (hloc[i] + hloc[j]), ha = 0.5 * (hloc[i] - hloc[j]);
        double hes = 0.5 * (heq[i] + heq[j]), hea = 0.5 * (heq[i] - heq[j]);
        o->hpc[i] = hloc[i] - (ha - hea) / tau_hb - (hs - hes) / tau_hs + (1.0 - 0.5 / tau_hs) * Hi[i];
    }
    o->ux = ux;
    o->uy = uy;
    o->p = pr;
    o->S = S;
    o->Q = Q;
}

/* ------------------------------------------------------------------ */
/* Step, part 3: streaming with wall rules                               */
/* ------------------------------------------------------------------ */

/* Push the post-collision populations of cell (x, y) to their destinations.
 * A population whose destination is beyond a wall returns to its own cell in
 * the opposite direction (half-way bounce-back: no slip, no flux).  For the
 * enthalpy at a Dirichlet wall it returns with the anti-bounce-back rule
 *   h_opp(x) = -h_i*(x) + 2 w_i rho_ref Cp_ref T_w,
 * (Sec. 4.5) with T_w the wall temperature at the foot of the cell, (x, -1/2)
 * for the bottom wall, for all three links that cross the wall there.  The
 * paper does not say where T_w is sampled; taking it at each link's own
 * crossing point x +- 1/2 instead doubles the O(k^2) error of the steady
 * temperature under a wall of wavenumber k against the closed-form solution.
 * At an adiabatic wall the enthalpy bounces back like the others. */
static void push_cell(orc_state *st, int x, int y, const cell_out *o)
{
    const orc_grid *g = &st->g;
    long n = st->n;
    long c = (long)y * g->nx + x;
    double rr = rhocp_ref(&st->p);
    for (int i = 0; i < 9; i++) {
        int yy = y + CY[i];
        if (yy >= 0 && yy < g->ny) {
            int xx = ((x + CX[i]) % g->nx + g->nx) % g->nx;
            long d = (long)yy * g->nx + xx;
            st->f2[i * n + d] = o->fpc[i];
            st->g2[i * n + d] = o->gpc[i];
            st->h2[i * n + d] = o->hpc[i];
            st->l2[i * n + d] = o->lpc[i];
        } else {
            int j = OPP[i];
            st->f2[j * n + c] = o->fpc[i];
            st->g2[j * n + c] = o->gpc[i];
            st->l2[j * n + c] = o->lpc[i];
            int bottom = yy < 0;
            int dirichlet = bottom ? (g->bc_bottom == ORC_WALL_DIRICHLET_T) : (g->bc_top == ORC_WALL_DIRICHLET_T);
            if (dirichlet) {
                double Tw = bottom ? T_wall_bottom(g, x) : g->T_top;
                st->h2[j * n + c] = -o->hpc[i] + 2.0 * WT[i] * rr * Tw;
            } else {
                st->h2[j * n + c] = o->hpc[i];
            }
        }
    }
}

static void swap_ptr(double **a, double **b)
{
    double *t = *a;
    *a = *b;
    *b = t;
}

void orc_step(orc_state *st, int nsteps)
{
    const orc_grid *g = &st->g;
    for (int s = 0; s < nsteps; s++) {
        pass_local(st);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < g->ny; y++) {
            for (int x = 0; x < g->nx; x++) {
                long c = (long)y * g->nx + x;
                cell_out o;
                cell_dynamics(st, x, y, &o);
                push_cell(st, x, y, &o);
                /* lagged state for the next step: fields read only at the
                 * own cell are overwritten in place; u, p and S, which the
                 * neighbours still read in this pass, go to new arrays */
                st->fs_prev[c] = st->fs[c];
                st->Q_prev[c] = o.Q;
                st->phi_prev[c] = st->phi[c];
                st->C_prev[c] = st->C[c];
                st->ux_new[c] = o.ux;
                st->uy_new[c] = o.uy;
                st->p_new[c] = o.p;
                st->S_new[c] = o.S;
            }
        }
        swap_ptr(&st->f, &st->f2);
        swap_ptr(&st->gq, &st->g2);
        swap_ptr(&st->h, &st->h2);
        swap_ptr(&st->l, &st->l2);
        swap_ptr(&st->ux_prev, &st->ux_new);
        swap_ptr(&st->uy_prev, &st->uy_new);
        swap_ptr(&st->p_prev, &st->p_new);
        swap_ptr(&st->S_prev, &st->S_new);
        st->step++;
    }
}

/* ------------------------------------------------------------------ */
/* Observables                                                           */
/* ------------------------------------------------------------------ */

/* Macroscopic fields of the current state: the quantities the next step
 * computes before it collides (phi, T, f_s, C, u, p, rho H).  Any pointer may
 * be NULL. */
void orc_fields(orc_state *st, double *phi, double *T, double *fs, double *C, double *ux,
                double *uy, double *pr, double *rhoH)
{
    const orc_grid *g = &st->g;
    pass_local(st);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < g->ny; y++)
        for (int x = 0; x < g->nx; x++) {
            long c = (long)y * g->nx + x;
            cell_out o;
            cell_dynamics(st, x, y, &o);
            if (phi) phi[c] = st->phi[c];
            if (T) T[c] = st->T[c];
            if (fs) fs[c] = st->fs[c];
            if (C) C[c] = st->C[c];
            if (ux) ux[c] = o.ux;
            if (uy) uy[c] = o.uy;
            if (pr) pr[c] = o.p;
            if (rhoH) rhoH[c] = st->rhoH[c];
        }
}

/* Global diagnostics of the current state, summed in row-major order:
 *   out[0] sum phi, out[1] sum rho H, out[2] sum C, out[3] sum f_s,
 *   out[4] sum chi with chi = clamp((1 + phi)/2, 0, 1),
 *   out[5] freezing-front height = sum_y f_s on the column x = nx/2,
 *   out[6] V*_s = sum f_s / V_0, out[7] V*_sl = sum chi / V_0,
 * V_0 = sum chi of the initial fields. */
void orc_reduce(orc_state *st, double out[8])
{
    const orc_grid *g = &st->g;
    pass_local(st);
    double a[6] = {0, 0, 0, 0, 0, 0};
    int xc = g->nx / 2;
    for (int y = 0; y < g->ny; y++)
        for (int x = 0; x < g->nx; x++) {
            long c = (long)y * g->nx + x;
            a[0] += st->phi[c];
            a[1] += st->rhoH[c];
            a[2] += st->C[c];
            a[3] += st->fs[c];
            a[4] += chi_of(st->phi[c]);
            if (x == xc) a[5] += st->fs[c];
        }
    for (int k = 0; k < 6; k++) out[k] = a[k];
    out[6] = st->V0 > 0 ? a[3] / st->V0 : 0.0;
    out[7] = st->V0 > 0 ? a[4] / st->V0 : 0.0;
}

long orc_step_count(const orc_state *st) { return st->step; }

/* Population access for invariant checks: set 0..3 = f, g, h, l; layout
 * [i * n + c].  Copies out 9 n values. */
void orc_get_populations(const orc_state *st, int set, double *out)
{
    const double *src = set == 0 ? st->f : set == 1 ? st->gq : set == 2 ? st->h : st->l;
    memcpy(out, src, sizeof(double) * 9 * (size_t)st->n);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
