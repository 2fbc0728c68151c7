/*
 * lb_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use it.  It shares nothing with the GPU library's headers.
 */
#ifndef LB_ORACLE_H
#define LB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_WALL_DIRICHLET_T 0
#define ORC_WALL_ADIABATIC 1

typedef struct {
    int nx, ny;            /* lattice, x periodic, walls at y = -1/2 and ny - 1/2 */
    int bc_bottom, bc_top; /* ORC_WALL_DIRICHLET_T or ORC_WALL_ADIABATIC */
    double T_bottom, T_top;
    double T_bottom_amp;   /* bottom wall T_bottom + amp cos(2 pi modes x / nx) */
    int T_bottom_modes;
    double cos_theta_bottom, cos_theta_top; /* wetting: cosine of the contact angle (0: 90 degrees) */
} orc_grid;

typedef struct {
    double rho_l, rho_s, rho_g;
    double mu_l, mu_s, mu_g;
    double lam_l, lam_s, lam_g;
    double cp_l, cp_s, cp_g;
    double latent, T_sol, T_liq;
    double k_p, D_l, D_s;
    double eps, mobility;
    double sigma0, sigma_T, sigma_c, T_ref, c_ref;
    double gx, gy;
    int fs_modulated_st, phase_change_on;
    int divu_mode; /* 0: div u = mdot (model value); 1: lagged velocity divergence */
    int lattice_fl; /* lattice of the phase-field and solute sets: 0 D2Q9, 1 D2Q5 */
    int rhocp_rule; /* 0: the property rule on rho C_p; 1: on rho and C_p apart, multiplied */
} orc_params;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_grid *g, const orc_params *p, const double *phi0,
                      const double *T0, const double *C0, const double *ux0, const double *uy0);
void orc_destroy(orc_state *st);
void orc_step(orc_state *st, int nsteps);
void orc_fields(orc_state *st, double *phi, double *T, double *fs, double *C, double *ux,
                double *uy, double *pr, double *rhoH);
void orc_reduce(orc_state *st, double out[8]);
long orc_step_count(const orc_state *st);
void orc_get_populations(const orc_state *st, int set, double *out);
int orc_num_threads(void);
void orc_set_num_threads(int k);

/* building blocks, exported for the invariant pins */
double orc_zeta(double phi, double fs, double zl, double zs, double zg);
void orc_enthalpy_invert(const orc_params *p, double e, double chi, double *T, double *fs);
double orc_enthalpy_forward(const orc_params *p, double T, double chi);
void orc_equilibria(const orc_params *p, double phi, double C, double rhoH, double T,
                    double pr, double ux, double uy, double rho, double rhocp,
                    double feq[9], double geq[9], double heq[9], double leq[9]);
void orc_sources(double dphiux, double dphiuy, double nx_, double ny_, double phi, double eps,
                 double mdot, double S, double Fx, double Fy, double rfx, double rfy,
                 double Ftx, double Fty, double ux, double uy, double Q,
                 double dCux, double dCuy, double Rx, double Ry,
                 double Fi[9], double Gi[9], double Hi[9], double Li[9]);
void orc_stencil_field(const orc_grid *g, const double *v, int kind, double *gx, double *gy,
                       double *lap);

#ifdef __cplusplus
}
#endif
#endif
