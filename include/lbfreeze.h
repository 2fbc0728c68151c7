/*
 * lbfreeze.h -- C ABI of the GB300 (sm_103a) fused diffuse-interface lattice
 * Boltzmann step for gas-liquid-solid freezing of a binary fluid with
 * thermal and solutal Marangoni flow (Huang, Chai, Liu, Huang,
 * arXiv 2511.09422).
 *
 * The library evolves, on one GPU, the four coupled D2Q9 distribution sets of
 * Sec. 3 of the paper on a 2-D lattice:
 *   f  conservative Allen-Cahn phase field (Sec. 3.1, Eq. ACE),
 *   g  pressure-based flow with the solid-liquid interaction force and the
 *      volume-change source (Sec. 3.2, Eqs. NS1-NS2),
 *   h  total enthalpy, two-relaxation-time (Sec. 3.3, Eqs. Tem and Hfl),
 *   l  solute with the pseudo-potential concentration (Sec. 3.4, Eq. c),
 * coupled through the continuum surface force with Marangoni and capillary
 * parts (Eq. Fs), the linear surface-tension equation of state, and the
 * property rule zeta(phi, f_s) (end of Sec. 2).  Gradients use the isotropic
 * schemes at the end of Sec. 3.4.  x is periodic; the walls at y = -1/2 and
 * y = ny - 1/2 are half-way bounce-back (no slip, no flux) with
 * anti-bounce-back for a Dirichlet temperature (Sec. 4.5).
 *
 * Conventions
 *   - Fields are nx*ny arrays, row-major with x fastest: v[y*nx + x].
 *   - All calls return an lb_status code; nothing throws across the ABI.
 *   - A handle owns all of its device memory.  Pointers passed in are
 *     borrowed for the duration of the call only.
 *   - Work is enqueued on the handle's stream (the legacy default stream
 *     until lb_set_stream).  lb_step is asynchronous; lb_get_fields with host
 *     outputs, lb_reduce, lb_save and lb_load synchronise that stream.
 *   - The first error is sticky: once a call has failed with LB_ERR_CUDA or
 *     LB_ERR_UNSTABLE, later calls on the handle return the same code.
 *   - Arithmetic is FP32 with FP64 global sums.
 */
#ifndef LBFREEZE_H
#define LBFREEZE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID_ARG = 1, /* null pointer, empty or oversized lattice, tau <= 1/2, eps <= 0 ... */
    LB_ERR_CUDA = 2,        /* a CUDA runtime call failed (message via lb_last_error) */
    LB_ERR_OOM = 3,         /* device allocation failed */
    LB_ERR_UNSTABLE = 4     /* a non-finite value was produced by the step */
} lb_status;

#define LB_WALL_DIRICHLET_T 0 /* anti-bounce-back to the wall temperature */
#define LB_WALL_ADIABATIC 1   /* bounce-back for the enthalpy as well */

/* Lattice and walls (problem statement, Sec. 2, Fig. 1; boundary
 * treatment of Sec. 4.5).  The bottom-wall temperature may vary along x as
 * T_bottom + T_bottom_amp * cos(2 pi T_bottom_modes x / nx) (the heated
 * channel of Sec. 4.1), with cell centres at integer x.
 * cos_theta_bottom, cos_theta_top: wettability of each wall (Sec. 3.4), the
 * cosine of the contact angle measured inside the phi = 1 phase, in [-1, 1];
 * 0 (the zero-initialised value) is 90 degrees.  The wall condition is the
 * normal derivative of the equilibrium profile at that angle,
 * n_w . grad phi = -cos(theta) (1 - phi^2) / (sqrt 2 eps), imposed on the
 * ghost of phi beyond the half-way wall: phi_ghost = phi_adjacent +
 * cos(theta) (1 - phi_adjacent^2) / (sqrt 2 eps); the density gradient
 * follows by the linear property rule. */
typedef struct {
    int nx, ny;             /* 1 <= nx, ny; nx*ny <= LB_MAX_CELLS */
    int bc_bottom, bc_top;  /* LB_WALL_DIRICHLET_T or LB_WALL_ADIABATIC */
    double T_bottom, T_top;
    double T_bottom_amp;
    int T_bottom_modes;
    double cos_theta_bottom, cos_theta_top;
} lb_grid;

#define LB_MAX_CELLS (1L << 28)

/* Model constants (Sec. 2 and 3).  Suffix _l liquid, _s solid, _g the
 * surrounding phase (phi = -1).  mu is the dynamic viscosity, lam the
 * conductivity, cp the specific heat; the property rule interpolates rho,
 * mu, lam and the volumetric heat capacity rho*cp.  latent is L of
 * H = Cp T + L f_l; T_sol, T_liq the solidus and liquidus; k_p the partition
 * coefficient and D_l, D_s the solute diffusivities of Eq. c; eps the
 * interface parameter of Eq. 3 and mobility M of Eq. ACE
 * (tau_f = 1/2 + M/cs^2); sigma0, sigma_T, sigma_c, T_ref, c_ref the linear
 * equation of state sigma = sigma0 + sigma_T (T - T_ref) + sigma_c (C - c_ref);
 * (gx, gy) the body-force acceleration (F_b = rho g).
 * fs_modulated_st: 1 multiplies the surface force by (1 - f_s) (Sec. 4.5).
 * phase_change_on: 0 drops the latent heat and keeps f_s = 0.
 * divu_mode: which velocity divergence enters the div u terms of Sec. 3.1
 * (the source w_i phi div u of F_i and the moment phi = sum f_i + phi div u/2)
 * and Sec. 3.3 (H_i and rho H = sum h_i + rho Cp T div u/2).  0: the model
 * value mdot of Eq. NS1.  1: the isotropic divergence (end of Sec. 3.4) of
 * the previous step's velocity, with the ghost -u beyond a no-slip wall; the
 * compression of the surrounding phase by the volume change then reaches the
 * interface, which reproduces the final heights of Table 1 and the final
 * droplet volume of Sec. 4.4.  Other values are rejected.
 * pop_storage: how the 36 population planes are stored.  LB_STORAGE_F32 (0):
 * FP32 deviations from lagged references.  LB_STORAGE_F16 (1): the same
 * deviations times 2^8 in IEEE half precision (the solute set shifted by
 * w_i c_ref as well), which halves the population bytes; the arithmetic stays
 * FP32 and the lagged fields stay FP32.  Half storage rounds every stored
 * population to 11 bits, so its results differ from the FP32 ones (tests state
 * the difference per field); a deviation beyond 2^8 x 65504 becomes infinite and
 * is reported as LB_ERR_UNSTABLE.  LB_STORAGE_F16_H32 (2): f, g and l as with
 * LB_STORAGE_F16, the enthalpy set h in FP32 as with LB_STORAGE_F32 (252
 * instead of 360 bytes per update); the rounding of the stored enthalpy
 * deviations is what moves the freezing time of a long run in half storage, so
 * this form keeps it at the FP32 level. */
#define LB_STORAGE_F32 0
#define LB_STORAGE_F16 1
#define LB_STORAGE_F16_H32 2
/* lattice_fl: velocity set of the phase-field (f) and solute (l) sets.  The
 * paper does not name it; LB_LATTICE_D2Q9 (0) uses D2Q9 for all four sets.
 * LB_LATTICE_D2Q5 (1) uses D2Q5 for f and l: the five velocities c_0 .. c_4
 * with weights 1/3, 1/6 (c_s^2 = 1/3, the same equilibria and sources of
 * Sec. 3.1 and 3.4 with these weights); g and h stay D2Q9.  f and l then
 * move 5 instead of 9 populations each (296 instead of 360 bytes per update).
 * Needs pop_storage = LB_STORAGE_F32. */
#define LB_LATTICE_D2Q9 0
#define LB_LATTICE_D2Q5 1
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
    int divu_mode;
    int pop_storage;
    int lattice_fl;
} lb_params;

/* Initial fields, nx*ny floats each, host or device memory (on_device = 0/1).
 * ux, uy may be NULL (fluid at rest). */
typedef struct {
    const float *phi, *T, *C, *ux, *uy;
    int on_device;
} lb_fields;

typedef struct lb_handle lb_handle;

/* Allocate the state and initialise it at rest in time: post-streaming
 * populations equal to the equilibria of the initial fields with p = 0,
 * the enthalpy from (T, chi) by the inverse of Eq. Hfl.
 * Returns LB_ERR_INVALID_ARG for null pointers, nx or ny < 1, nx*ny above
 * LB_MAX_CELLS, a padded plane (nx rounded up to a multiple of 32, times ny)
 * of 2^31 floats or more, eps <= 0, non-positive densities, a relaxation time <= 1/2
 * anywhere in the property range, or divu_mode not 0 or 1.  *out is set only on
 * success.  Synchronises the device. */
lb_status lb_create(const lb_grid *grid, const lb_params *params, const lb_fields *init,
                    lb_handle **out);

/* Use a CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later work of the handle; NULL selects the legacy default stream. */
lb_status lb_set_stream(lb_handle *h, void *cuda_stream);

/* Enqueue n >= 0 time steps (one fused kernel launch each).  Asynchronous.
 * One step is the LB update of Sec. 3 for all four sets: streaming with the
 * wall rules of Sec. 4.5 (half-way bounce-back; anti-bounce-back of the
 * enthalpy at a Dirichlet wall), the moments of Sec. 3.1-3.4 (phi, rho u*,
 * u, p, rho H, C), the enthalpy relation Eq. Hfl, the property rule of
 * Sec. 2, the isotropic stencils at the end of Sec. 3.4, the forces of
 * Eq. Fs and Sec. 3.2, and the collisions (BGK for f, g, l; two relaxation
 * times for h).  A non-finite result sets a sticky status that lb_reduce
 * returns as LB_ERR_UNSTABLE; an error of an earlier call is returned
 * unchanged and nothing is enqueued. */
lb_status lb_step(lb_handle *h, int n);

/* Macroscopic fields of the current state -- the values the next step
 * computes before it collides (the moments of Sec. 3.1-3.4 and Eq. Hfl):
 * order parameter phi, temperature T, solid fraction f_s, concentration C,
 * velocity (ux, uy) (the corrected velocity u = u* + f/2 of Sec. 3.2),
 * pressure p.  Each output is nx*ny floats, row-major with x fastest, host or
 * device memory as on_device says, owned by the caller; any may be NULL.
 * With host outputs the call synchronises the stream. */
lb_status lb_get_fields(lb_handle *h, float *phi, float *T, float *fs, float *C, float *ux,
                        float *uy, float *p, int on_device);

/* Replace the current state by the equilibrium state of the given fields
 * (the inverse of lb_get_fields): populations at the equilibria of (phi, u, p,
 * C) and of the enthalpy, lagged fields set from the inputs.  Same layout as
 * lb_get_fields (nx*ny floats each, host or device memory); phi, T, C are
 * required.  fs: the solid fraction, clamped to [0, chi]; the enthalpy is
 * then the latent part rho_l L (chi - f_s) plus the sensible part with the
 * mixture rule T (f_s (rho Cp)_s + (chi - f_s) (rho Cp)_l + (1 - chi)
 * (rho Cp)_g).  fs = NULL derives f_s from (T, chi) as lb_create does.
 * ux, uy, p = NULL mean 0.  With divu_mode = 1 the rest population of the
 * phase-field set is lowered by phi div u / 2 (div u of the given velocity),
 * so that the moment phi = sum f_i + phi div u / 2 of Sec. 3.1 returns the
 * given phi.  The step count and V_0 are kept.  This is how a
 * learned surrogate's prediction of the fields is handed back to the method;
 * the paper has no counterpart.  With host inputs the call synchronises the
 * stream. */
lb_status lb_set_fields(lb_handle *h, const float *phi, const float *T, const float *fs, const float *C,
                        const float *ux, const float *uy, const float *p, int on_device);

/* Global diagnostics of the current state in FP64, summed in a fixed order
 * (the conservation checks of Sec. 2 and the freezing measures of Sec. 4.2
 * and 4.4: solid height on the centre column, the solid and the total
 * phase-change volume relative to the initial one, V*_s and V*_sl):
 *   out[0] sum phi     out[1] sum rho H    out[2] sum C     out[3] sum f_s
 *   out[4] sum chi, chi = clamp((1 + phi)/2, 0, 1)
 *   out[5] front height: sum over y of f_s on the column x = nx/2
 *   out[6] V*_s  = sum f_s / V_0     out[7] V*_sl = sum chi / V_0
 * with V_0 = sum chi of the initial state.  Synchronises the stream; returns
 * LB_ERR_UNSTABLE if the step has produced a non-finite value. */
lb_status lb_reduce(lb_handle *h, double out[8]);

/* The diagnostics of lb_reduce (same eight values, summed per lattice row
 * and then over the rows, so they can differ from lb_reduce in the last
 * digits), computed without allocating any device memory: for callers that
 * cannot allocate at this point, e.g. because another allocator holds the
 * device's memory or the surrounding code forbids allocation.  The paper has
 * no counterpart of this call.  Its scratch is a fixed device array of
 * (LB_NOALLOC_MAX_ROWS + 1) x 6 doubles (196,656 bytes) that every GPU using
 * the library keeps until exit; lattices with more than LB_NOALLOC_MAX_ROWS
 * rows get LB_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address, so make that first call before any stream capture,
 * with the handle's device current.  All calls share the array: calls that
 * run on the GPU at the same time race and must be serialised by the caller.
 * Synchronises the stream; out is host memory. */
#define LB_NOALLOC_MAX_ROWS 4096
lb_status lb_reduce_noalloc(lb_handle *h, double out[8]);

/* Number of steps taken since lb_create (or restored by lb_load). */
lb_status lb_steps_taken(lb_handle *h, long *out);

/* Checkpoint: write / read the complete state of the time stepping of Sec. 3
 * (the stored populations of the four sets, the lagged fields the next step
 * reads, the step count and V_0) to / from a file at path.  lb_load requires
 * a file written for the same nx, ny, population storage and lattice_fl
 * (LB_ERR_INVALID_ARG otherwise, state unchanged); the run then continues
 * bit-for-bit as the saved run would have.  Both synchronise the stream. */
lb_status lb_save(lb_handle *h, const char *path);
lb_status lb_load(lb_handle *h, const char *path);

/* Free the handle and its device memory; NULL is a no-op. */
void lb_destroy(lb_handle *h);

/* ---- Batched instances -------------------------------------------------------
 * Many independent lattices ("instances", each with its own lb_grid, lb_params
 * and initial fields, as in a parameter sweep over droplets of uneven sizes)
 * advanced together: one persistent kernel launch per step covers all of them,
 * its warps taking (instance, 30-column strip, row segment) work items from a
 * shared counter.  Every instance evolves exactly as a single-lattice handle
 * created from the same inputs (bit for bit).  The paper runs its cases one at
 * a time; this is the throughput form of the same step (Sec. 3). */
typedef struct lb_batch lb_batch;

/* Create n >= 1 instances: grids[i], params[i], init[i] as for lb_create (the
 * same checks and errors; a failure names the instance in
 * lb_batch_last_error(NULL)).  All instances use the same pop_storage
 * (LB_ERR_INVALID_ARG otherwise).  Synchronises the device. */
lb_status lb_batch_create(int n, const lb_grid *grids, const lb_params *params, const lb_fields *init,
                          lb_batch **out);

/* Stream for the batch and all of its instances (NULL: legacy default stream). */
lb_status lb_batch_set_stream(lb_batch *b, void *cuda_stream);

/* Enqueue n >= 0 steps of every instance.  Pairs of steps are replayed from a
 * CUDA graph captured on first use (lb_batch_use_graph(b, 0) launches them one
 * by one instead).  Asynchronous.  Returns LB_ERR_INVALID_ARG if instances were
 * stepped separately (lb_step on an instance handle) by different counts. */
lb_status lb_batch_step(lb_batch *b, int n);
lb_status lb_batch_use_graph(lb_batch *b, int on);

/* Autotuner: for each size class (lattice rows < 192, < 320, >= 320) time
 * `trials` batched launches with inner row segments of 8, 12, 16, 24, 32 and 64 rows
 * and keep the fastest; seg_rows (3 ints, may be NULL) receives the choice per
 * class (0 for an empty class).  The trial launches do not advance the state.
 * Synchronises the stream. */
lb_status lb_batch_tune(lb_batch *b, int trials, int seg_rows[3]);

/* Handle of instance i (0 <= i < n), owned by the batch: use it with
 * lb_get_fields, lb_reduce, lb_save..., but do not destroy it. */
lb_status lb_batch_instance(lb_batch *b, int i, lb_handle **out);

/* Number of instances and total cells (either pointer may be NULL). */
lb_status lb_batch_size(const lb_batch *b, int *n, long long *cells);

/* Message of the last failure on the batch (or of the calling thread's last
 * failed lb_batch_create when b is NULL); never NULL. */
const char *lb_batch_last_error(const lb_batch *b);

/* Free the batch and all of its instances; NULL is a no-op. */
void lb_batch_destroy(lb_batch *b);

/* ---- Slabs of one lattice (y-slab decomposition, one slab per GPU) -----------
 * The step of Sec. 3 is local: a cell's update reads its own populations and
 * those of its eight neighbours, and the isotropic stencils at the end of
 * Sec. 3.4 reach one cell further.  A lattice cut into slabs of whole rows
 * therefore advances exactly as one lattice when, before every step, each
 * slab holds copies of the two rows of state (stored populations and lagged
 * fields) next to it on either side: its ghost rows.  The result is bit for
 * bit that of the whole lattice.  x stays periodic within every slab.
 *
 * lb_slab_create: the slab of rows [y0, y1) of the lattice `global` (walls,
 * parameters and storage as for lb_create).  init holds the initial fields of
 * rows [y0 - 2, y1 + 2) of the lattice, (y1 - y0 + 4) * nx values each,
 * without the two rows below when y0 = 0 or above when y1 = global->ny (those
 * ends are the lattice's walls); the handle's local lattice has those rows.
 * Every slab, and so every neighbour, needs at least 4 rows: y1 - y0 >= 4,
 * and y0 = 0 or y0 >= 4, and y1 = ny or ny - y1 >= 4 (LB_ERR_INVALID_ARG
 * otherwise).  The handle works with every single-lattice call; lb_step,
 * lb_reduce, lb_reduce_noalloc and lb_get_fields update, sum or read only the
 * owned rows (the ghost rows of lb_get_fields's outputs hold no meaningful values;
 * the diagnostics are the slab's share of the lattice's sums, with V_0 the
 * slab's own).  Ghost rows are filled by lb_slab_unpack only. */
lb_status lb_slab_create(const lb_grid *global, const lb_params *params, const lb_fields *init, int y0, int y1,
                         lb_handle **out);

/* Bytes of one face's halo message: 2 rows x nx values of the 36 population
 * planes (4 bytes each, 2 with half storage) followed by the 9 lagged planes
 * (FP32), plane by plane.  0 for a handle from lb_create. */
size_t lb_slab_halo_bytes(const lb_handle *h);

/* lb_slab_pack: the two owned rows next to face 0 (low y) or 1 (high y) of
 * the current state into dst (lb_slab_halo_bytes bytes, caller-owned; host
 * memory with on_device = 0, then the call synchronises the stream, or device
 * memory, then it is asynchronous on the handle's stream).  After a step,
 * the message of face 0 goes to the slab below, that of face 1 to the slab
 * above.  lb_slab_unpack: a neighbour's message into the ghost rows at face
 * (0: from the slab below, 1: from the slab above), same memory rules.  A
 * face without a neighbouring slab is LB_ERR_INVALID_ARG. */
lb_status lb_slab_pack(lb_handle *h, int face, void *dst, int on_device);
lb_status lb_slab_unpack(lb_handle *h, int face, const void *src, int on_device);

/* Static description of a status code. */
const char *lb_error_string(int status);

/* Message of the last failure on this handle (or of the calling thread's
 * last failed lb_create when h is NULL); never NULL. */
const char *lb_last_error(const lb_handle *h);

/* Device bytes held by the handle. */
size_t lb_device_bytes(const lb_handle *h);

#ifdef __cplusplus
}
#endif
#endif
