// lb_api.cu -- host side of the C ABI declared in include/lbfreeze.h.
//
// Owns the device state of one lattice (double-buffered populations and
// lagged fields, a field buffer for read-back, FP64 reduction partials) and
// launches the kernels of lb_kernels.cuh on the handle's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lb_kernels.cuh"
#include "lbfreeze.h"

using lbk::Consts;

struct lb_handle {
    lb_grid grid;
    lb_params params;
    Consts K;
    float *pops[2] = {nullptr, nullptr};
    float *aux[2] = {nullptr, nullptr};
    float *fields = nullptr;     // 7 planes
    double *partials = nullptr;  // reduction partials, red_parts * NRED
    double *red_out = nullptr;   // NRED doubles on the device
    unsigned *status = nullptr;
    lbk::StepRec *rec = nullptr;          // the step kernel's record of this lattice
    unsigned long long *counter = nullptr;  // the step kernel's work counters (2)
    long long nitems = 0;                   // work items of one step
    int red_parts = 0;           // partial slots: one per warp of the largest capped MODE_REDUCE grid
    bool half = false;           // some populations stored in half precision
    // kernel instantiation: 0 FP32 D2Q9, 1 FP16 D2Q9, 2 FP32 with D2Q5 f and l, 3 FP16 f, g, l with FP32 h
    int kind = 0;
    size_t pop_bytes() const;
    int cur = 0;
    cudaStream_t stream = nullptr;
    double V0 = 0.0;
    long steps = 0;
    lb_status sticky = LB_OK;
    std::string err;
    size_t bytes = 0;
    unsigned char *halo = nullptr;  // device staging of one halo message (slabs with a host-memory exchange)
    size_t halo_bytes = 0;          // bytes of one face's halo message (slabs only)
};

// Kernel kind of a run: 0 FP32 D2Q9, 1 FP16 D2Q9, 2 FP32 with D2Q5 f and l, 3 FP16 f, g, l with FP32 h.
static int kind_of(const lb_params *p)
{
    return p->pop_storage == LB_STORAGE_F16 ? 1
                                            : (p->pop_storage == LB_STORAGE_F16_H32 ? 3 : (p->lattice_fl == 1 ? 2 : 0));
}

// Calls f(PS{}) with the storage trait of kernel kind `kind`.
template <class F>
static auto with_storage(int kind, F f)
{
    if (kind == 1) return f(lbk::PopF16{});
    if (kind == 2) return f(lbk::PopF32Q5{});
    if (kind == 3) return f(lbk::PopF16H{});
    return f(lbk::PopF32{});
}

size_t lb_handle::pop_bytes() const
{
    return with_storage(kind, [&](auto ps) { return (size_t)lbk::pop_cell_bytes<decltype(ps)>() * (size_t)K.plane; });
}

static thread_local std::string g_create_error;  // last lb_create failure of this thread

static const char *k_status_text[] = {"ok", "invalid argument", "CUDA error", "out of device memory",
                                      "unstable: a non-finite value was produced"};

extern "C" const char *lb_error_string(int status)
{
    if (status < 0 || status > 4) return "unknown status";
    return k_status_text[status];
}

extern "C" const char *lb_last_error(const lb_handle *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" size_t lb_device_bytes(const lb_handle *h) { return h ? h->bytes : 0; }

static lb_status fail(lb_handle *h, lb_status s, const std::string &msg)
{
    if (h) {
        if (h->sticky == LB_OK && (s == LB_ERR_CUDA || s == LB_ERR_UNSTABLE)) h->sticky = s;
        h->err = msg;
    } else {
        g_create_error = msg;
    }
    return s;
}

static lb_status cuda_fail(lb_handle *h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, m);
}

#define CK(h, call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------------------
// Parameter checks: every relaxation time must stay above 1/2 over the whole
// property range (phi in [-1, 1], f_s in [0, 1]).
// ---------------------------------------------------------------------------------------
static bool finite_all(const lb_params *p)
{
    const double v[] = {p->rho_l, p->rho_s, p->rho_g, p->mu_l, p->mu_s, p->mu_g, p->lam_l, p->lam_s, p->lam_g,
                        p->cp_l, p->cp_s, p->cp_g, p->latent, p->T_sol, p->T_liq, p->k_p, p->D_l, p->D_s,
                        p->eps, p->mobility, p->sigma0, p->sigma_T, p->sigma_c, p->T_ref, p->c_ref, p->gx, p->gy};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

static std::string check_params(const lb_grid *g, const lb_params *p)
{
    if (g->nx < 1 || g->ny < 1) return "nx and ny must be >= 1";
    if ((long)g->nx * (long)g->ny > LB_MAX_CELLS) return "lattice larger than LB_MAX_CELLS";
    if ((long)((g->nx + 31) / 32 * 32) * (long)g->ny >= (1L << 31))
        return "padded plane (nx rounded up to 32, times ny) of 2^31 floats or more";
    if (g->bc_bottom < 0 || g->bc_bottom > 1 || g->bc_top < 0 || g->bc_top > 1) return "unknown wall type";
    if (!(std::fabs(g->cos_theta_bottom) <= 1.0) || !(std::fabs(g->cos_theta_top) <= 1.0))
        return "cos_theta_bottom and cos_theta_top must lie in [-1, 1]";
    if (!finite_all(p)) return "non-finite parameter";
    if (!(p->eps > 0)) return "eps must be > 0";
    if (!(p->rho_l > 0 && p->rho_s > 0 && p->rho_g > 0)) return "densities must be > 0";
    if (!(p->cp_l > 0 && p->cp_s > 0 && p->cp_g > 0)) return "heat capacities must be > 0";
    if (!(p->mobility > 0)) return "mobility must be > 0 (tau_f > 1/2)";
    if (!(p->mu_l > 0 && p->mu_s > 0 && p->mu_g > 0)) return "viscosities must be > 0 (tau_g > 1/2)";
    if (!(p->lam_l > 0 && p->lam_s > 0 && p->lam_g > 0)) return "conductivities must be > 0 (tau_h > 1/2)";
    if (!(p->D_l > 0) || p->D_s < 0) return "D_l must be > 0 and D_s >= 0 (tau_l > 1/2 in the liquid)";
    if (!(p->k_p > 0)) return "k_p must be > 0";
    if (p->divu_mode != 0 && p->divu_mode != 1) return "divu_mode must be 0 or 1";
    if (p->pop_storage != LB_STORAGE_F32 && p->pop_storage != LB_STORAGE_F16 && p->pop_storage != LB_STORAGE_F16_H32)
        return "pop_storage must be LB_STORAGE_F32, LB_STORAGE_F16 or LB_STORAGE_F16_H32";
    if (p->lattice_fl != LB_LATTICE_D2Q9 && p->lattice_fl != LB_LATTICE_D2Q5)
        return "lattice_fl must be LB_LATTICE_D2Q9 or LB_LATTICE_D2Q5";
    if (p->lattice_fl == LB_LATTICE_D2Q5 && p->pop_storage != LB_STORAGE_F32)
        return "lattice_fl = LB_LATTICE_D2Q5 needs pop_storage = LB_STORAGE_F32";
    if (p->phase_change_on && p->T_liq < p->T_sol) return "T_liq < T_sol";
    return "";
}

static Consts make_consts(const lb_grid *g, const lb_params *p)
{
    Consts K;
    memset(&K, 0, sizeof(K));
    K.nx = g->nx;
    K.ny = g->ny;
    K.pitch = (g->nx + 31) / 32 * 32;
    K.plane = (long long)K.pitch * g->ny;
    K.bc_bottom = g->bc_bottom;
    K.bc_top = g->bc_top;
    K.T_bottom = (real)g->T_bottom;
    K.T_top = (real)g->T_top;
    K.T_bottom_amp = (real)g->T_bottom_amp;
    K.wall_k = (real)(2.0 * g->T_bottom_modes / g->nx);
    K.wet_b = (real)(g->cos_theta_bottom / (std::sqrt(2.0) * p->eps));
    K.wet_t = (real)(g->cos_theta_top / (std::sqrt(2.0) * p->eps));
    K.rho_l = (real)p->rho_l; K.rho_s = (real)p->rho_s; K.rho_g = (real)p->rho_g;
    K.mu_l = (real)p->mu_l; K.mu_s = (real)p->mu_s; K.mu_g = (real)p->mu_g;
    K.lam_l = (real)p->lam_l; K.lam_s = (real)p->lam_s; K.lam_g = (real)p->lam_g;
    K.rcp_l = (real)(p->rho_l * p->cp_l);
    K.rcp_s = (real)(p->rho_s * p->cp_s);
    K.rcp_g = (real)(p->rho_g * p->cp_g);
    K.latent_l = (real)(p->rho_l * p->latent);
    K.lat_l = p->phase_change_on ? K.latent_l : 0.0f;
    K.T_sol = (real)p->T_sol; K.T_liq = (real)p->T_liq;
    K.k_p = (real)p->k_p; K.D_l = (real)p->D_l; K.D_s = (real)p->D_s;
    K.rr = (real)(p->rho_l * 2.0 * p->cp_s * p->cp_l / (p->cp_s + p->cp_l));
    K.inv_rr = (real)((p->cp_s + p->cp_l) / (p->rho_l * 2.0 * p->cp_s * p->cp_l));
    K.inv_eps2 = (real)(1.0 / (p->eps * p->eps));
    K.inv_s2eps = (real)(1.0 / (std::sqrt(2.0) * p->eps));
    K.alpha = (real)(3.0 * std::sqrt(2.0) * p->eps / 4.0);
    K.tau_f = (real)(0.5 + 3.0 * p->mobility);
    K.om_f = (real)(1.0 / (0.5 + 3.0 * p->mobility));
    K.src_f = (real)(1.0 - 0.5 / (0.5 + 3.0 * p->mobility));
    K.sigma0 = (real)p->sigma0; K.sigma_T = (real)p->sigma_T; K.sigma_c = (real)p->sigma_c;
    K.T_ref = (real)p->T_ref; K.c_ref = (real)p->c_ref;
    K.gx = (real)p->gx; K.gy = (real)p->gy;
    K.expand = (real)(1.0 - p->rho_s / p->rho_l);
    K.fs_mod = p->fs_modulated_st ? 1 : 0;
    K.segh = (p->pop_storage != LB_STORAGE_F32 || p->lattice_fl == LB_LATTICE_D2Q5) ? LB_SEGH_ALT : LB_SEGH;
    // Shorter segments where the lattice gives the persistent wave of W warps too
    // few work items.  A work item costs about segh + 3 rows (its rows plus the
    // fill and copy prologue); the warps share the items dynamically, so a step
    // takes about items (segh + 3) / W plus one item, the last one started.  The
    // height of the default and the shorter candidates (8 rows at least) that
    // minimises it.
    {
        const long long W = with_storage(kind_of(p), [](auto ps) {
            return 152LL * lbk::step_min_blocks<decltype(ps)>() * lbk::step_warps<decltype(ps)>();
        });
        const long long nstrip = (g->nx + LB_TX - 1) / LB_TX;
        auto cost = [&](int h) { return (double)(nstrip * lbk::strip_segments(g->ny, h)) * (h + 3) / (double)W + (h + 3); };
        const int cand[] = {24, 16, 12, 8};
        int best = K.segh;
        for (int c : cand)
            if (c < K.segh && cost(c) < cost(best)) best = c;
        K.segh = best;
    }
    K.qfl = p->lattice_fl == LB_LATTICE_D2Q5 ? 5 : 9;
    K.divu = p->divu_mode;
    K.phase_change = p->phase_change_on ? 1 : 0;
    return K;
}

// One strip-kernel launch covers the lattice: the two bands next to the walls
// (blocks first) and the inner segments.  MODE_REDUCE caps the grid at one wave
// of resident blocks, each block then owning several (strip group, segment)
// pairs, and writes one partial per warp.
static unsigned strip_blocks(const Consts &K)
{
    return (unsigned)(lbk::strip_groups(K.nx) * lbk::strip_segments(K.ny, K.segh));
}

template <class PS>
static unsigned reduce_blocks(const Consts &K)
{
    const unsigned n = strip_blocks(K), cap = 152u * (unsigned)lbk::strip_min_blocks<PS, false>();
    return n < cap ? n : cap;
}

// Shared-memory carveout (percent of the 228 KB maximum) that holds `blocks`
// resident blocks of `smem` bytes each (1 KB reserved per block) and no more:
// the rest of the SM's 256 KB stays L1, which caches the per-lane staging
// copies of the strip ends and wall bands.
static int carveout_for(int blocks, size_t smem)
{
    const long long need = (long long)blocks * ((long long)smem + 1024), max = 228LL * 1024;
    const int pct = (int)((100 * need + max - 1) / max);
    return pct > 100 ? 100 : pct;
}

template <int MODE, class PS>
static void launch_strip_as(const Consts &K, const lbk::Buffers &B, cudaStream_t st, double *partials)
{
    constexpr size_t smem = lbk::strip_smem<PS, MODE != lbk::MODE_REDUCE>();
    static bool opted = false;  // per instantiation: rings above 48 KB need the opt-in, and the
    if (!opted) {               // carveout holds every resident block
        cudaFuncSetAttribute(lbk::lb_strip_kernel<MODE, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(lbk::lb_strip_kernel<MODE, PS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             carveout_for(lbk::strip_min_blocks<PS, MODE != lbk::MODE_REDUCE>(), smem));
        opted = true;
    }
    const unsigned grid = MODE == lbk::MODE_REDUCE ? reduce_blocks<PS>(K) : strip_blocks(K);
    lbk::lb_strip_kernel<MODE, PS><<<grid, dim3(32, LB_SW, 1), smem, st>>>(K, B, partials);
}

template <int MODE>
static void launch_strip(const Consts &K, const lbk::Buffers &B, cudaStream_t st, int kind, double *partials = nullptr)
{
    with_storage(kind, [&](auto ps) { launch_strip_as<MODE, decltype(ps)>(K, B, st, partials); });
}

static int flat_blocks(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    long long cap = 152LL * 8;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// Record of lattice h for the step kernel, its work items numbered from item0;
// returns the number of items.
static long long fill_record(const lb_handle *h, lbk::StepRec &r, long long item0)
{
    r.K = h->K;
    for (int p = 0; p < 2; p++) {
        r.B[p].pin = h->pops[p];
        r.B[p].pout = h->pops[1 - p];
        r.B[p].ain = h->aux[p];
        r.B[p].aout = h->aux[1 - p];
        r.B[p].fields = nullptr;
        r.B[p].status = h->status;
    }
    r.nstrip = (h->K.nx + LB_TX - 1) / LB_TX;
    r.item0 = item0;
    return (long long)r.nstrip * lbk::strip_segments(h->K.ny, h->K.segh);
}

// One step of ninst lattices (records rec, nitems work items in all) from buffer
// `parity`: a persistent launch of at most one wave of resident blocks.
template <class PS>
static cudaError_t launch_step_as(const lbk::StepRec *rec, int ninst, long long nitems, int parity,
                                  unsigned long long *counter, cudaStream_t st)
{
    constexpr size_t smem = lbk::step_smem<PS>();
    constexpr int sw = lbk::step_warps<PS>();
    static bool opted = false;
    if (!opted) {
        cudaFuncSetAttribute(lbk::lb_step_kernel<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(lbk::lb_step_kernel<PS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             carveout_for(lbk::step_min_blocks<PS>(), smem));
        opted = true;
    }
    // one persistent wave: as many blocks per SM as the rings of PS allow
    const long long wave = 152LL * lbk::step_min_blocks<PS>(), need = (nitems + sw - 1) / sw;
    const unsigned grid = (unsigned)(need < wave ? (need < 1 ? 1 : need) : wave);
    lbk::lb_step_kernel<PS><<<grid, dim3(32, sw, 1), smem, st>>>(rec, ninst, nitems, parity, counter);
    return cudaGetLastError();
}

static cudaError_t launch_step(const lbk::StepRec *rec, int ninst, long long nitems, int parity,
                               unsigned long long *counter, cudaStream_t st, int kind)
{
    return with_storage(kind, [&](auto ps) {
        return launch_step_as<decltype(ps)>(rec, ninst, nitems, parity, counter, st);
    });
}

static lb_status launch_reduce(lb_handle *h, double out[lbk::NRED])
{
    const Consts &K = h->K;
    lbk::Buffers B;
    B.pin = h->pops[h->cur];
    B.pout = nullptr;
    B.ain = h->aux[h->cur];
    B.aout = nullptr;
    B.fields = nullptr;
    B.status = h->status;
    launch_strip<lbk::MODE_REDUCE>(K, B, h->stream, h->kind, h->partials);
    CK(h, cudaGetLastError());
    // the warps of this launch's grid (the segment height, and so the grid, can change with lb_batch_tune)
    const int nparts = (int)with_storage(h->kind, [&](auto ps) { return reduce_blocks<decltype(ps)>(K); }) * LB_SW;
    lbk::lb_reduce_final_kernel<<<1, lbk::RED_THREADS, 0, h->stream>>>(h->partials, nparts, h->red_out);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(out, h->red_out, sizeof(double) * lbk::NRED, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

static void free_all(lb_handle *h)
{
    void *ptrs[] = {h->pops[0], h->pops[1], h->aux[0], h->aux[1], h->fields, h->partials, h->red_out, h->status,
                    h->rec,     h->counter, h->halo};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

// A lattice, or a slab of one whose two rows at an end with ghost_* set are
// ghost rows (see Consts::ghost_lo).
static lb_status create_handle(const lb_grid *grid, const lb_params *params, const lb_fields *init, int ghost_lo,
                               int ghost_hi, lb_handle **out)
{
    if (!grid || !params || !init || !out) return fail(nullptr, LB_ERR_INVALID_ARG, "null argument");
    std::string why = check_params(grid, params);
    if (!why.empty()) return fail(nullptr, LB_ERR_INVALID_ARG, why);
    if (!init->phi || !init->T || !init->C) return fail(nullptr, LB_ERR_INVALID_ARG, "initial phi, T and C are required");

    lb_handle *h = new lb_handle();
    h->grid = *grid;
    h->params = *params;
    h->half = params->pop_storage != LB_STORAGE_F32;
    h->kind = kind_of(params);
    h->K = make_consts(grid, params);
    h->K.ghost_lo = ghost_lo;
    h->K.ghost_hi = ghost_hi;
    if (ghost_lo || ghost_hi)
        h->halo_bytes = with_storage(h->kind, [&](auto ps) {
            return (size_t)lbk::halo_message_bytes<decltype(ps)>(grid->nx);
        });
    const Consts &K = h->K;
    const long long n = (long long)grid->nx * grid->ny;
    const size_t plane_b = sizeof(float) * (size_t)K.plane;
    // every grid reduce_blocks can give (a capped wave of at most 6 blocks per SM)
    h->red_parts = 152 * 6 * LB_SW;

    auto alloc = [&](void **p, size_t b) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, b);
        if (e == cudaSuccess) h->bytes += b;
        return e;
    };
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = alloc((void **)&h->pops[k], h->pop_bytes());
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = alloc((void **)&h->aux[k], lbk::NAUX * plane_b);
    if (e == cudaSuccess) e = alloc((void **)&h->fields, 7 * plane_b);
    if (e == cudaSuccess) e = alloc((void **)&h->partials, sizeof(double) * lbk::NRED * h->red_parts);
    if (e == cudaSuccess) e = alloc((void **)&h->red_out, sizeof(double) * lbk::NRED);
    if (e == cudaSuccess) e = alloc((void **)&h->status, sizeof(unsigned));
    if (e == cudaSuccess) e = alloc((void **)&h->rec, sizeof(lbk::StepRec));
    if (e == cudaSuccess) e = alloc((void **)&h->counter, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess && h->halo_bytes) e = alloc((void **)&h->halo, h->halo_bytes);
    if (e != cudaSuccess) {
        lb_status s = cuda_fail(nullptr, e, "cudaMalloc");
        cudaGetLastError();
        free_all(h);
        delete h;
        return s;
    }

    // initial fields on the device (the field buffer serves as staging)
    const float *src[5] = {init->phi, init->T, init->C, init->ux, init->uy};
    const float *dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    lb_status st = LB_OK;
    do {
        cudaError_t me = cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream);
        if (me == cudaSuccess) me = cudaMemsetAsync(h->counter, 0, 2 * sizeof(unsigned long long), h->stream);
        lbk::StepRec rec;
        h->nitems = fill_record(h, rec, 0);
        if (me == cudaSuccess) me = cudaMemcpyAsync(h->rec, &rec, sizeof(rec), cudaMemcpyHostToDevice, h->stream);
        if (me != cudaSuccess) { st = cuda_fail(h, me, "step record"); break; }
        for (int k = 0; k < 5; k++) {
            if (!src[k]) continue;
            float *d = h->fields + (size_t)k * K.plane;
            cudaError_t ce = cudaMemcpyAsync(d, src[k], sizeof(float) * n,
                                             init->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
            if (ce != cudaSuccess) { st = cuda_fail(h, ce, "copy of the initial fields"); break; }
            dev[k] = d;
        }
        if (st != LB_OK) break;
        // equilibria in FP32: in the second population buffer, or for half storage
        // in a temporary buffer freed once the first buffer holds the state
        float *eq = h->pops[1], *eq_tmp = nullptr;
        if (h->half) {
            cudaError_t ae = cudaMalloc((void **)&eq_tmp, 36 * plane_b);
            if (ae != cudaSuccess) { st = cuda_fail(h, ae, "cudaMalloc of the initial equilibria"); break; }
            eq = eq_tmp;
        }
        lbk::lb_init_eq_kernel<<<flat_blocks(n, 256), 256, 0, h->stream>>>(K, dev[0], dev[1], dev[2], dev[3], dev[4],
                                                                           nullptr, nullptr, eq, h->aux[0], 0);
        with_storage(h->kind, [&](auto ps) {
            lbk::lb_init_unstream_kernel<decltype(ps)><<<flat_blocks(n, 256), 256, 0, h->stream>>>(K, eq, h->aux[0],
                                                                                                  h->pops[0]);
            return 0;
        });
        cudaError_t ce = cudaGetLastError();
        if (eq_tmp) {
            cudaError_t fe = cudaStreamSynchronize(h->stream);
            cudaFree(eq_tmp);
            if (ce == cudaSuccess) ce = fe;
        }
        if (ce != cudaSuccess) { st = cuda_fail(h, ce, "init kernels"); break; }
        h->cur = 0;
        double r[lbk::NRED];
        st = launch_reduce(h, r);
        if (st != LB_OK) break;
        h->V0 = r[4];
    } while (0);
    if (st != LB_OK) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return LB_OK;
}

extern "C" lb_status lb_create(const lb_grid *grid, const lb_params *params, const lb_fields *init, lb_handle **out)
{
    return create_handle(grid, params, init, 0, 0, out);
}

// ---------------------------------------------------------------------------------------
// Slabs of a larger lattice (y-slab decomposition across GPUs).
// ---------------------------------------------------------------------------------------
extern "C" lb_status lb_slab_create(const lb_grid *global, const lb_params *params, const lb_fields *init, int y0,
                                    int y1, lb_handle **out)
{
    if (!global || !params || !init || !out) return fail(nullptr, LB_ERR_INVALID_ARG, "null argument");
    if (y0 < 0 || y1 > global->ny || y1 - y0 < 4)
        return fail(nullptr, LB_ERR_INVALID_ARG, "slab rows [y0, y1) must lie in [0, ny) and hold at least 4 rows");
    if (y0 > 0 && y0 < 4)
        return fail(nullptr, LB_ERR_INVALID_ARG, "a slab below this one would hold fewer than 4 rows (y0 < 4)");
    if (y1 < global->ny && global->ny - y1 < 4)
        return fail(nullptr, LB_ERR_INVALID_ARG, "a slab above this one would hold fewer than 4 rows (ny - y1 < 4)");
    const int glo = y0 > 0 ? 2 : 0, ghi = y1 < global->ny ? 2 : 0;
    lb_grid g = *global;
    g.ny = y1 - y0 + glo + ghi;
    return create_handle(&g, params, init, glo != 0, ghi != 0, out);
}

extern "C" size_t lb_slab_halo_bytes(const lb_handle *h) { return h ? h->halo_bytes : 0; }

// first lattice row of the two rows that face `face` packs (owned) or unpacks (ghost)
static int halo_row(const lb_handle *h, int face, bool ghost)
{
    const Consts &K = h->K;
    if (face == 0) return ghost ? 0 : 2;
    return ghost ? K.ny - 2 : K.ny - 4;
}

static lb_status halo_check(lb_handle *h, int face, const void *p)
{
    if (!h || !p) return fail(h, LB_ERR_INVALID_ARG, "null argument");
    if (h->sticky != LB_OK) return h->sticky;
    if ((face != 0 && face != 1) || !(face == 0 ? h->K.ghost_lo : h->K.ghost_hi))
        return fail(h, LB_ERR_INVALID_ARG, "face must be 0 (low y) or 1 (high y) and have a neighbouring slab");
    return LB_OK;
}

extern "C" lb_status lb_slab_pack(lb_handle *h, int face, void *dst, int on_device)
{
    lb_status s = halo_check(h, face, dst);
    if (s != LB_OK) return s;
    unsigned char *msg = on_device ? (unsigned char *)dst : h->halo;
    const long long vals = 2LL * h->K.nx * (36 + lbk::NAUX);
    with_storage(h->kind, [&](auto ps) {
        lbk::lb_halo_kernel<decltype(ps), true><<<flat_blocks(vals, 256), 256, 0, h->stream>>>(
            h->K, (unsigned char *)h->pops[h->cur], h->aux[h->cur], halo_row(h, face, false), msg);
        return 0;
    });
    CK(h, cudaGetLastError());
    if (!on_device) {
        CK(h, cudaMemcpyAsync(dst, h->halo, h->halo_bytes, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LB_OK;
}

extern "C" lb_status lb_slab_unpack(lb_handle *h, int face, const void *src, int on_device)
{
    lb_status s = halo_check(h, face, src);
    if (s != LB_OK) return s;
    const unsigned char *msg = (const unsigned char *)src;
    if (!on_device) {
        CK(h, cudaMemcpyAsync(h->halo, src, h->halo_bytes, cudaMemcpyHostToDevice, h->stream));
        msg = h->halo;
    }
    const long long vals = 2LL * h->K.nx * (36 + lbk::NAUX);
    with_storage(h->kind, [&](auto ps) {
        lbk::lb_halo_kernel<decltype(ps), false><<<flat_blocks(vals, 256), 256, 0, h->stream>>>(
            h->K, (unsigned char *)h->pops[h->cur], h->aux[h->cur], halo_row(h, face, true),
            const_cast<unsigned char *>(msg));
        return 0;
    });
    CK(h, cudaGetLastError());
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

extern "C" lb_status lb_set_stream(lb_handle *h, void *cuda_stream)
{
    if (!h) return LB_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return LB_OK;
}

extern "C" lb_status lb_step(lb_handle *h, int n)
{
    if (!h || n < 0) return fail(h, LB_ERR_INVALID_ARG, "null handle or negative step count");
    if (h->sticky != LB_OK) return h->sticky;
    for (int s = 0; s < n; s++) {
        cudaError_t e = launch_step(h->rec, 1, h->nitems, h->cur, h->counter, h->stream, h->kind);
        if (e != cudaSuccess) return cuda_fail(h, e, "lb_step_kernel launch");
        h->cur = 1 - h->cur;
        h->steps++;
    }
    return LB_OK;
}

extern "C" lb_status lb_steps_taken(lb_handle *h, long *out)
{
    if (!h || !out) return LB_ERR_INVALID_ARG;
    *out = h->steps;
    return LB_OK;
}

extern "C" lb_status lb_get_fields(lb_handle *h, float *phi, float *T, float *fs, float *C, float *ux, float *uy,
                                   float *p, int on_device)
{
    if (!h) return LB_ERR_INVALID_ARG;
    if (h->sticky != LB_OK) return h->sticky;
    const Consts &K = h->K;
    lbk::Buffers B;
    B.pin = h->pops[h->cur];
    B.pout = nullptr;
    B.ain = h->aux[h->cur];
    B.aout = nullptr;
    B.fields = h->fields;
    B.status = h->status;
    launch_strip<lbk::MODE_FIELDS>(K, B, h->stream, h->kind);
    CK(h, cudaGetLastError());
    float *dst[7] = {phi, T, fs, C, ux, uy, p};
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < 7; k++) {
        if (!dst[k]) continue;
        CK(h, cudaMemcpy2DAsync(dst[k], sizeof(float) * K.nx, h->fields + (size_t)k * K.plane, sizeof(float) * K.pitch,
                                sizeof(float) * K.nx, K.ny, kind, h->stream));
    }
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

extern "C" lb_status lb_set_fields(lb_handle *h, const float *phi, const float *T, const float *fs, const float *C,
                                   const float *ux, const float *uy, const float *p, int on_device)
{
    if (!h) return LB_ERR_INVALID_ARG;
    if (h->sticky != LB_OK) return h->sticky;
    if (!phi || !T || !C) return fail(h, LB_ERR_INVALID_ARG, "phi, T and C are required");
    const Consts &K = h->K;
    const size_t n = (size_t)K.nx * K.ny;
    // the inputs go to the 7-plane fields buffer first (dense, as lb_create does), in
    // the argument order phi, T, C, ux, uy, fs, p
    const float *src[7] = {phi, T, C, ux, uy, fs, p};
    const float *dev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k = 0; k < 7; k++) {
        if (!src[k]) continue;
        float *d = h->fields + (size_t)k * K.plane;
        CK(h, cudaMemcpyAsync(d, src[k], sizeof(float) * n, kind, h->stream));
        dev[k] = d;
    }
    const size_t plane_b = sizeof(float) * (size_t)K.plane;
    float *eq = h->pops[1 - h->cur], *eq_tmp = nullptr;
    if (h->half) {
        CK(h, cudaMallocAsync((void **)&eq_tmp, 36 * plane_b, h->stream));
        eq = eq_tmp;
    }
    lbk::lb_init_eq_kernel<<<flat_blocks((long long)n, 256), 256, 0, h->stream>>>(K, dev[0], dev[1], dev[2], dev[3],
                                                                                 dev[4], dev[5], dev[6], eq,
                                                                                 h->aux[h->cur], 1);
    with_storage(h->kind, [&](auto ps) {
        lbk::lb_init_unstream_kernel<decltype(ps)><<<flat_blocks((long long)n, 256), 256, 0, h->stream>>>(
            K, eq, h->aux[h->cur], h->pops[h->cur]);
        return 0;
    });
    CK(h, cudaGetLastError());
    if (eq_tmp) CK(h, cudaFreeAsync(eq_tmp, h->stream));
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

extern "C" lb_status lb_reduce(lb_handle *h, double out[8])
{
    if (!h || !out) return fail(h, LB_ERR_INVALID_ARG, "null argument");
    if (h->sticky != LB_OK) return h->sticky;
    double r[lbk::NRED];
    lb_status s = launch_reduce(h, r);
    if (s != LB_OK) return s;
    unsigned status = 0;
    CK(h, cudaMemcpyAsync(&status, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 6; k++) out[k] = r[k];
    out[6] = h->V0 > 0 ? r[3] / h->V0 : 0.0;
    out[7] = h->V0 > 0 ? r[4] / h->V0 : 0.0;
    bool finite = true;
    for (int k = 0; k < 6; k++) finite = finite && std::isfinite(r[k]);
    if (status || !finite) return fail(h, LB_ERR_UNSTABLE, "non-finite value in the lattice state");
    return LB_OK;
}

// ---------------------------------------------------------------------------------------
// Checkpoint: header + raw planes (populations, lagged fields) of the current buffer.
// ---------------------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int version, nx, ny, pitch;
    long steps;
    double V0;
};

extern "C" lb_status lb_save(lb_handle *h, const char *path)
{
    if (!h || !path) return fail(h, LB_ERR_INVALID_ARG, "null argument");
    if (h->sticky != LB_OK) return h->sticky;
    const Consts &K = h->K;
    const size_t pb = h->pop_bytes(), ab = sizeof(float) * lbk::NAUX * (size_t)K.plane;
    char *buf = (char *)malloc(pb + ab);
    if (!buf) return fail(h, LB_ERR_INVALID_ARG, "host allocation for the checkpoint failed");
    cudaError_t e = cudaMemcpyAsync(buf, h->pops[h->cur], pb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + pb, h->aux[h->cur], ab, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        free(buf);
        return cuda_fail(h, e, "checkpoint read-back");
    }
    FILE *f = fopen(path, "wb");
    if (!f) {
        free(buf);
        return fail(h, LB_ERR_INVALID_ARG, std::string("cannot open ") + path);
    }
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LBFRZ01", 8);
    hd.version = h->kind + 1;  // 1: FP32, 2: half-precision populations, 3: FP32 with D2Q5 f and l
    hd.nx = K.nx; hd.ny = K.ny; hd.pitch = K.pitch; hd.steps = h->steps; hd.V0 = h->V0;
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(buf, 1, pb + ab, f) == pb + ab;
    ok = (fclose(f) == 0) && ok;
    free(buf);
    return ok ? LB_OK : fail(h, LB_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

extern "C" lb_status lb_load(lb_handle *h, const char *path)
{
    if (!h || !path) return fail(h, LB_ERR_INVALID_ARG, "null argument");
    if (h->sticky != LB_OK) return h->sticky;
    const Consts &K = h->K;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(h, LB_ERR_INVALID_ARG, std::string("cannot open ") + path);
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, "LBFRZ01", 8) != 0 || hd.nx != K.nx || hd.ny != K.ny ||
        hd.pitch != K.pitch || hd.version != h->kind + 1) {
        fclose(f);
        return fail(h, LB_ERR_INVALID_ARG, "checkpoint does not match this lattice");
    }
    const size_t pb = h->pop_bytes(), ab = sizeof(float) * lbk::NAUX * (size_t)K.plane;
    char *buf = (char *)malloc(pb + ab);
    if (!buf) {
        fclose(f);
        return fail(h, LB_ERR_INVALID_ARG, "host allocation for the checkpoint failed");
    }
    bool ok = fread(buf, 1, pb + ab, f) == pb + ab;
    fclose(f);
    if (!ok) {
        free(buf);
        return fail(h, LB_ERR_INVALID_ARG, "truncated checkpoint");
    }
    cudaError_t e = cudaMemcpyAsync(h->pops[h->cur], buf, pb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->aux[h->cur], buf + pb, ab, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    free(buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint upload");
    h->steps = hd.steps;
    h->V0 = hd.V0;
    return LB_OK;
}

extern "C" void lb_destroy(lb_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

// ---------------------------------------------------------------------------------------
// Diagnostics without any device allocation (lb_reduce_noalloc).
//
// For callers that must not allocate device memory when they read the
// diagnostics -- for example code whose device memory is entirely reserved by
// another allocator (a framework's caching pool), or a section of a larger
// pipeline that runs under a no-allocation rule.  The scratch lives in one
// fixed file-scope device array instead of the handle: one row of FP64 partial
// sums per lattice row, then the totals.  Every GPU that loads this library
// holds the array, (LB_NOALLOC_MAX_ROWS + 1) * 6 doubles = 196,656 bytes,
// until the process exits.  All calls share it and it keeps the last call's
// contents; every call overwrites the rows and totals it reads, so nothing
// needs clearing, but calls that overlap on the GPU (different streams or
// threads at once) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[(LB_NOALLOC_MAX_ROWS + 1) * lbk::NRED];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device, with that device current, by the first call made on it.
static double *g_noalloc_addr[256];
static std::mutex g_noalloc_mu;

namespace {

template <class PS>
__global__ void __launch_bounds__(lbk::RED_THREADS) noalloc_rows_kernel(const Consts K, const float *__restrict__ pin,
                                                                         const float *__restrict__ ain,
                                                                         double *__restrict__ scratch)
{
    __shared__ double sh[lbk::RED_THREADS / 32][lbk::NRED];
    const int y = blockIdx.x;
    const int xc = K.nx / 2;
    const bool ghost = (K.ghost_lo && y < 2) || (K.ghost_hi && y >= K.ny - 2);  // a slab's ghost rows add nothing
    double acc[lbk::NRED] = {0, 0, 0, 0, 0, 0};
    for (int x = ghost ? K.nx : (int)threadIdx.x; x < K.nx; x += blockDim.x) {
        const int cell = y * K.pitch + x;
        const lbk::CellA c =
            lbk::cell_a<PS>(K, pin, ain, x, y, cell);
        lbk::add_diag(K, c.phi_p, c.L.dphi, c.ed, c.T_p, c.chi_p, c.fs_p, c.L.C, c.L.fs, x == xc, acc);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < lbk::NRED; q++) {
        double s = lbk::warp_sum(acc[q]);
        if (lane == 0) sh[w][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < lbk::NRED) {
        double s = 0.0;
        for (int j = 0; j < lbk::RED_THREADS / 32; j++) s += sh[j][threadIdx.x];
        scratch[(long long)y * lbk::NRED + threadIdx.x] = s;
    }
}

// Adds the row partials in row order; the totals go after the last possible row.
__global__ void noalloc_total_kernel(double *__restrict__ scratch, int nrows)
{
    if (threadIdx.x < lbk::NRED) {
        double s = 0.0;
        for (int y = 0; y < nrows; y++) s += scratch[(long long)y * lbk::NRED + threadIdx.x];
        scratch[(long long)LB_NOALLOC_MAX_ROWS * lbk::NRED + threadIdx.x] = s;
    }
}

}  // namespace

extern "C" lb_status lb_reduce_noalloc(lb_handle *h, double out[8])
{
    if (!h || !out) return fail(h, LB_ERR_INVALID_ARG, "null argument");
    if (h->sticky != LB_OK) return h->sticky;
    const Consts &K = h->K;
    if (K.ny > LB_NOALLOC_MAX_ROWS)
        return fail(h, LB_ERR_INVALID_ARG,
                    "lb_reduce_noalloc: the lattice has " + std::to_string(K.ny) + " rows; its fixed scratch holds " +
                        std::to_string(LB_NOALLOC_MAX_ROWS) + " (use lb_reduce)");
    int dev = -1;
    CK(h, cudaGetDevice(&dev));
    cudaPointerAttributes attr;
    CK(h, cudaPointerGetAttributes(&attr, h->pops[0]));
    if (attr.device != dev)
        return fail(h, LB_ERR_INVALID_ARG, "lb_reduce_noalloc: call it with the handle's device current");
    if (dev < 0 || dev >= 256) return fail(h, LB_ERR_INVALID_ARG, "lb_reduce_noalloc: device ordinal out of range");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_noalloc_addr[dev] = (double *)p;
        }
        scratch = g_noalloc_addr[dev];
    }
    with_storage(h->kind, [&](auto ps) {
        noalloc_rows_kernel<decltype(ps)><<<K.ny, lbk::RED_THREADS, 0, h->stream>>>(K, h->pops[h->cur],
                                                                                   h->aux[h->cur], scratch);
        return 0;
    });
    CK(h, cudaGetLastError());
    noalloc_total_kernel<<<1, 32, 0, h->stream>>>(scratch, K.ny);
    CK(h, cudaGetLastError());
    double r[lbk::NRED];
    unsigned status = 0;
    CK(h, cudaMemcpyAsync(r, scratch + (size_t)LB_NOALLOC_MAX_ROWS * lbk::NRED, sizeof(r), cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaMemcpyAsync(&status, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 6; k++) out[k] = r[k];
    out[6] = h->V0 > 0 ? r[3] / h->V0 : 0.0;
    out[7] = h->V0 > 0 ? r[4] / h->V0 : 0.0;
    bool finite = true;
    for (int k = 0; k < 6; k++) finite = finite && std::isfinite(r[k]);
    if (status || !finite) return fail(h, LB_ERR_UNSTABLE, "non-finite value in the lattice state");
    return LB_OK;
}

// ---------------------------------------------------------------------------------------
// Batched instances: independent lattices advanced by one persistent launch per step.
// The instances are ordinary handles owned by the batch, so the per-handle calls
// (fields, diagnostics, checkpoints) work on each of them.
// ---------------------------------------------------------------------------------------
struct lb_batch {
    std::vector<lb_handle *> h;
    std::vector<lbk::StepRec> inst;
    lbk::StepRec *d_inst = nullptr;
    unsigned long long *d_counter = nullptr;
    long long nitems = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;                   // stream used to capture the step graphs
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // two steps, starting from buffer 0 or 1
    bool use_graph = true;
    lb_status sticky = LB_OK;
    std::string err;
};

static thread_local std::string g_batch_create_error;  // last lb_batch_create failure of this thread

static lb_status bfail(lb_batch *b, lb_status s, const std::string &msg)
{
    if (b) {
        if (b->sticky == LB_OK && (s == LB_ERR_CUDA || s == LB_ERR_UNSTABLE)) b->sticky = s;
        b->err = msg;
    } else {
        g_batch_create_error = msg;
    }
    return s;
}

#define BCK(b, call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void drop_graphs(lb_batch *b)
{
    for (auto &g : b->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Size class of an instance for the autotuner: by lattice rows.
static int size_class(const lb_handle *h) { return h->K.ny < 192 ? 0 : (h->K.ny < 320 ? 1 : 2); }

// Rebuild the work list and the device copy of the per-instance records.
static lb_status upload_instances(lb_batch *b)
{
    long long item = 0;
    for (size_t i = 0; i < b->h.size(); i++) item += fill_record(b->h[i], b->inst[i], item);
    b->nitems = item;
    BCK(b, cudaMemcpy(b->d_inst, b->inst.data(), sizeof(lbk::StepRec) * b->inst.size(), cudaMemcpyHostToDevice));
    drop_graphs(b);
    return LB_OK;
}

// One batched step from buffer `parity` on stream st.
static lb_status launch_batch(lb_batch *b, int parity, cudaStream_t st)
{
    BCK(b, launch_step(b->d_inst, (int)b->h.size(), b->nitems, parity, b->d_counter, st, b->h[0]->kind));
    return LB_OK;
}

extern "C" lb_status lb_batch_create(int n, const lb_grid *grids, const lb_params *params, const lb_fields *init,
                                     lb_batch **out)
{
    if (n < 1 || !grids || !params || !init || !out) return bfail(nullptr, LB_ERR_INVALID_ARG, "null argument or n < 1");
    lb_batch *b = new lb_batch();
    for (int i = 0; i < n; i++) {
        lb_handle *h = nullptr;
        lb_status s = lb_create(&grids[i], &params[i], &init[i], &h);
        if (s != LB_OK) {
            std::string why = "instance " + std::to_string(i) + ": " + lb_last_error(nullptr);
            lb_batch_destroy(b);
            return bfail(nullptr, s, why);
        }
        b->h.push_back(h);
        if (h->kind != b->h[0]->kind) {
            lb_batch_destroy(b);
            return bfail(nullptr, LB_ERR_INVALID_ARG, "instance " + std::to_string(i) +
                                                          ": all instances must use the same pop_storage and lattice_fl");
        }
    }
    b->inst.resize(n);
    lb_status s = LB_OK;
    cudaError_t e = cudaMalloc((void **)&b->d_inst, sizeof(lbk::StepRec) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counter, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) s = bfail(nullptr, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, cudaGetErrorString(e));
    if (s == LB_OK) {
        s = upload_instances(b);
        if (s != LB_OK) g_batch_create_error = b->err;
    }
    if (s != LB_OK) {
        lb_batch_destroy(b);
        return s;
    }
    *out = b;
    return LB_OK;
}

extern "C" lb_status lb_batch_set_stream(lb_batch *b, void *cuda_stream)
{
    if (!b) return LB_ERR_INVALID_ARG;
    b->stream = (cudaStream_t)cuda_stream;
    for (lb_handle *h : b->h) h->stream = b->stream;
    return LB_OK;
}

extern "C" lb_status lb_batch_use_graph(lb_batch *b, int on)
{
    if (!b) return LB_ERR_INVALID_ARG;
    b->use_graph = on != 0;
    return LB_OK;
}

extern "C" lb_status lb_batch_step(lb_batch *b, int n)
{
    if (!b || n < 0) return bfail(b, LB_ERR_INVALID_ARG, "null batch or negative step count");
    if (b->sticky != LB_OK) return b->sticky;
    const int p = b->h[0]->cur;
    for (lb_handle *h : b->h) {
        if (h->sticky != LB_OK) return bfail(b, h->sticky, "an instance is in an error state: " + h->err);
        if (h->cur != p) return bfail(b, LB_ERR_INVALID_ARG, "instances were stepped separately and are out of step");
    }
    int done = 0;
    if (b->use_graph && n >= 2) {
        if (!b->gexec[p]) {
            cudaGraph_t g = nullptr;
            BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            lb_status s1 = launch_batch(b, p, b->cap);
            lb_status s2 = s1 == LB_OK ? launch_batch(b, 1 - p, b->cap) : s1;
            cudaError_t e = cudaStreamEndCapture(b->cap, &g);
            if (s2 != LB_OK) {
                if (g) cudaGraphDestroy(g);
                return s2;
            }
            if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->gexec[p], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        for (; done + 2 <= n; done += 2) BCK(b, cudaGraphLaunch(b->gexec[p], b->stream));
    }
    for (int par = (p + done) & 1; done < n; done++, par ^= 1) {
        lb_status s = launch_batch(b, par, b->stream);
        if (s != LB_OK) return s;
    }
    for (lb_handle *h : b->h) {
        h->cur = (h->cur + n) & 1;
        h->steps += n;
    }
    return LB_OK;
}

extern "C" lb_status lb_batch_tune(lb_batch *b, int trials, int seg_rows[3])
{
    if (!b || trials < 1) return bfail(b, LB_ERR_INVALID_ARG, "null batch or trials < 1");
    if (b->sticky != LB_OK) return b->sticky;
    const int cand[6] = {8, 12, 16, 24, 32, 64};
    const int p = b->h[0]->cur;
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    lb_status st = LB_OK;
    int best_all[3] = {0, 0, 0};
    for (int c = 0; c < 3 && st == LB_OK; c++) {
        bool any = false;
        for (lb_handle *h : b->h) any = any || size_class(h) == c;
        if (!any) continue;
        float best_ms = 0.0f;
        int best = 0;
        for (int k = 0; k < 6 && st == LB_OK; k++) {
            for (lb_handle *h : b->h)
                if (size_class(h) == c) h->K.segh = cand[k];
            st = upload_instances(b);
            // trial launches read the current buffer and write the other one, which the
            // next real step overwrites: the state does not move
            if (st == LB_OK) st = launch_batch(b, p, b->stream);
            if (st != LB_OK) break;
            cudaEventRecord(e0, b->stream);
            for (int t = 0; t < trials && st == LB_OK; t++) st = launch_batch(b, p, b->stream);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = bfail(b, LB_ERR_CUDA, "tuning timing");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best == 0 || ms < best_ms) {
                best_ms = ms;
                best = cand[k];
            }
        }
        for (lb_handle *h : b->h)
            if (size_class(h) == c) h->K.segh = best;
        best_all[c] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == LB_OK) st = upload_instances(b);
    if (seg_rows)
        for (int c = 0; c < 3; c++) seg_rows[c] = best_all[c];
    return st;
}

extern "C" lb_status lb_batch_instance(lb_batch *b, int i, lb_handle **out)
{
    if (!b || !out || i < 0 || i >= (int)b->h.size()) return bfail(b, LB_ERR_INVALID_ARG, "bad instance index");
    *out = b->h[i];
    return LB_OK;
}

extern "C" lb_status lb_batch_size(const lb_batch *b, int *n, long long *cells)
{
    if (!b) return LB_ERR_INVALID_ARG;
    if (n) *n = (int)b->h.size();
    if (cells) {
        long long c = 0;
        for (const lb_handle *h : b->h) c += (long long)h->K.nx * h->K.ny;
        *cells = c;
    }
    return LB_OK;
}

extern "C" const char *lb_batch_last_error(const lb_batch *b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

extern "C" void lb_batch_destroy(lb_batch *b)
{
    if (!b) return;
    drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_counter) cudaFree(b->d_counter);
    for (lb_handle *h : b->h) lb_destroy(h);
    delete b;
}
