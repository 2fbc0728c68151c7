// lb_kernels.cuh -- sm_103a kernels of the fused diffuse-interface LB freezing step.
//
// One launch of lb_step_kernel advances a lattice -- or a batch of independent
// lattices -- by one time step of the four coupled D2Q9 sets of arXiv
// 2511.09422, Sec. 3: phase field f (BGK, Sec. 3.1), pressure-based flow g
// (BGK, Sec. 3.2), total enthalpy h (two-relaxation-time, Sec. 3.3) and solute
// l (BGK, Sec. 3.4).  lb_strip_kernel runs the same sweep to read out the
// macroscopic fields or the diagnostics sums.
//
// Memory layout (HBM): structure of arrays.  Every population direction and
// every lagged field is a plane of pitch*ny floats (row pitch a multiple of
// 32 floats, so each warp row access is one aligned 128-byte line).  The
// state is double-buffered: the kernel pulls post-collision populations of
// the previous step from buffer A (stream-then-collide, "pull" form) and
// writes this step's post-collision populations to buffer B at the own cell.
// Lagged fields (plane index):
//   0 f_s  1 Q = rho Cp T div u  2 u_x  3 u_y  4 phi  5 C  6 p  7 S  8 T
// are read from A and written to B the same way.
//
// Storage form.  The phase-field, flow and enthalpy populations are stored
// as deviations from a reference rebuilt exactly on reading, so that FP32
// rounding at storage applies to the small non-equilibrium part instead of
// the whole value:
//   f_i   stored as f_i* - w_i phi^n(s)
//   g_i   stored as g_i* - 3 p^n(s) (w_i - [i = 0])
//   h_i   stored as h_i* - w_i rr T^n(s)                     (i > 0)
//   h_0   stored as h_0* - w_0 rr T^n(s) - rho_l L (chi(phi^n(s)) - f_s^n(s))
// with s the cell that wrote the value, rr = rho_ref Cp_ref, and phi^n, p^n,
// T^n, f_s^n the lagged fields written by the same step.  The step's
// arithmetic carries phi, p and T as (lagged value, small change) pairs, so
// that the large parts -- phi ~ 1, the pressure, T, and the latent enthalpy
// ~ rho_l L -- cancel analytically instead of in FP32.
//
// Strip form (lb_step_kernel, lb_strip_kernel): each warp owns a strip of 30 columns plus a
// one-column halo on each side (32 lanes) and walks down a segment of rows.
// Per row y it runs phase A -- the local fields of the step (T, f_s, mdot,
// phi, C) from the pulled f, h, l -- into per-warp shared-memory rings, and
// then phase B for row y - 1, whose neighbours are all in the rings: the
// isotropic gradients, the forces, velocity and pressure, and the collision
// of the four sets.  The pulled f, h, l are read from global memory once, the
// halo costs 2 rows per segment and two columns per 30, and the warps of a
// CTA never synchronise with one another (only __syncwarp).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

// Arithmetic type of the step (FP32; the diagnostics sums are FP64).
typedef float real;
#define R(x) ((real)(x))

#define LB_TX 30  // interior columns of a warp strip (32 lanes less a halo column on each side)

namespace lbk {

// ---------------------------------------------------------------------------------------
// D2Q9: 0 rest; 1 (+1,0) 2 (0,+1) 3 (-1,0) 4 (0,-1); 5 (+1,+1) 6 (-1,+1) 7 (-1,-1) 8 (+1,-1)
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
// c_iy of a direction known only at run time: a 2-bit table (c_iy + 1 for i = 0 .. 8).
__device__ __forceinline__ int cy_rt(int i) { return ((0x2865 >> (2 * i)) & 3) - 1; }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
__host__ __device__ constexpr real wgt(int i) { return i == 0 ? (R(4.0) / R(9.0)) : (i <= 4 ? (R(1.0) / R(9.0)) : (R(1.0) / R(36.0))); }
// Weights of the phase-field and solute sets on a lattice of Q = 9 or 5
// velocities (D2Q5: the first five D2Q9 velocities, weights 1/3 and 1/6, the
// same c_s^2 = 1/3).
template <int Q>
__host__ __device__ constexpr real wfl(int i)
{
    return Q == 9 ? wgt(i) : (i == 0 ? (R(1.0) / R(3.0)) : (i <= 4 ? (R(1.0) / R(6.0)) : R(0.0)));
}
__host__ __device__ inline real wfl_rt(int q, int i) { return q == 5 ? wfl<5>(i) : wfl<9>(i); }

constexpr int SET_F = 0, SET_G = 1, SET_H = 2, SET_L = 3;

// Storage of the 36 population planes, per set (f, g, h, l).  PopF32: FP32
// deviations (see the top of this file).  PopF16: the same deviations times 2^8
// in IEEE half precision, the solute set additionally shifted by w_i c_ref,
// halving the population bytes.  PopF16H: f, g and l as PopF16, the enthalpy set
// h in FP32 (its rounding sets the freezing-time error of half storage).  The
// arithmetic is FP32 in every form.  A half deviation beyond 2^8 * 65504
// overflows to infinity, which the step reports as non-finite.  esize(s) is the
// bytes of one stored value of set s; the sets' planes follow each other in the
// order f, g, h, l, nine planes each.
struct PopF32 {
    static constexpr bool kHalf = false;  // some set stored in half precision
    static constexpr int QFL = 9;         // lattice of the phase-field and solute sets
    __host__ __device__ static constexpr int esize(int) { return 4; }
};
struct PopF16 {
    static constexpr bool kHalf = true;
    static constexpr int QFL = 9;
    __host__ __device__ static constexpr int esize(int) { return 2; }
};
struct PopF16H {
    static constexpr bool kHalf = true;
    static constexpr int QFL = 9;
    __host__ __device__ static constexpr int esize(int s) { return s == SET_H ? 4 : 2; }
};
// FP32 storage with D2Q5 for the phase-field and solute sets (lb_params.lattice_fl
// = 1): their populations 5 .. 8 are neither read nor written.
struct PopF32Q5 : PopF32 {
    static constexpr int QFL = 5;
};

// Element type of set S under storage PS, and the encoding of a deviation.
template <class PS, int S>
using SetT = typename std::conditional<PS::esize(S) == 2, __half, float>::type;

// v 2^-8 + c in one mixed-precision FMA (sm_100+: half multiplicands, FP32
// addend and result).  The product of two halves is exact in FP32, so this is
// the FP32 sum of the decoded deviation and c, rounded once; c = -0 gives the
// deviation itself with the sign of a zero kept.
__device__ __forceinline__ float dec_fma(__half v, float c)
{
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(__half_as_ushort(v)), "h"((unsigned short)0x1C00), "f"(c));
    return d;
}
__device__ __forceinline__ real dec_val(float v) { return v; }
__device__ __forceinline__ real dec_val(__half v) { return dec_fma(v, -0.0f); }
template <class T>
__device__ __forceinline__ T enc_val(real d);
template <>
__device__ __forceinline__ float enc_val<float>(real d) { return d; }
template <>
__device__ __forceinline__ __half enc_val<__half>(real d) { return __float2half_rn(d * R(256.0)); }

// Bytes per cell of the planes before set s.
template <class PS>
__host__ __device__ constexpr int set_bytes_before(int s)
{
    return s <= 0 ? 0 : set_bytes_before<PS>(s - 1) + 9 * PS::esize(s - 1);
}
// Bytes per cell of all 36 planes.
template <class PS>
__host__ __device__ constexpr int pop_cell_bytes() { return set_bytes_before<PS>(4); }

constexpr int AUX_FS = 0, AUX_Q = 1, AUX_UX = 2, AUX_UY = 3, AUX_PHI = 4, AUX_C = 5, AUX_P = 6, AUX_S = 7, AUX_T = 8;
constexpr int NAUX = 9;
constexpr int WALL_DIRICHLET = 0;

// Constants of one run, precomputed on the host from lb_params.
struct Consts {
    int nx, ny, pitch;
    long long plane;          // floats per plane (pitch * ny)
    int bc_bottom, bc_top;
    real T_bottom, T_top, T_bottom_amp, wall_k;  // wall_k = 2 * modes / nx (argument of cospi)
    real wet_b, wet_t;          // cos(theta) / (sqrt 2 eps) of the bottom and top walls (0: 90 degrees)
    real rho_l, rho_s, rho_g, mu_l, mu_s, mu_g, lam_l, lam_s, lam_g;
    real rcp_l, rcp_s, rcp_g;   // volumetric heat capacities rho*Cp
    real latent_l;              // rho_l * L
    real lat_l;                 // rho_l * L if phase change is on, else 0 (latent reference of h_0)
    real T_sol, T_liq, k_p, D_l, D_s;
    real rr;                    // rho_ref Cp_ref
    real inv_eps2, inv_s2eps, alpha;
    real tau_f, om_f, src_f;    // tau_f, 1/tau_f, 1 - 1/(2 tau_f)
    real inv_rr;                // 1 / (rho_ref Cp_ref)
    real sigma0, sigma_T, sigma_c, T_ref, c_ref, gx, gy;
    real expand;                // 1 - rho_s / rho_l
    int fs_mod, phase_change;
    int segh;                   // rows of an inner segment of the strip sweep
    int qfl;                    // lattice of the phase-field and solute sets: 9 or 5 velocities
    int divu;                   // div u in the phi and h sources: 0 the model value mdot, 1 the lagged velocity divergence
    // Slab of a larger lattice (y-slab decomposition): 1 when the two rows at
    // this end are ghost rows holding the neighbouring slab's state instead of
    // rows next to a wall.  Ghost rows are read by the sweep but never updated,
    // summed or read out; the sweep then has no wall at that end.
    int ghost_lo, ghost_hi;
};

struct Buffers {
    const float *__restrict__ pin;
    float *__restrict__ pout;
    const float *__restrict__ ain;
    float *__restrict__ aout;
    float *__restrict__ fields;  // 7 planes, fields mode only
    unsigned *status;
};

__device__ __forceinline__ real zeta(real phi, real fs, real zl, real zs, real zg)
{
    return R(0.5) * phi * (zl - zg) + fs * (zs - zl) + R(0.5) * (zl + zg);
}

__device__ __forceinline__ int wrapx(int x, int nx)
{
    return x < 0 ? x + nx : (x >= nx ? x - nx : x);
}

// Start of plane k of a buffer.  A plane holds fewer than 2^31 floats (the
// host rejects larger ones), so offsets within a plane are 32-bit.
template <class T>
__device__ __forceinline__ T *plane_ptr(T *base, int k, const Consts &K)
{
    return base + (size_t)(unsigned)K.plane * (unsigned)k;
}

// Plane i of set S in a population buffer (base: the buffer's first byte).
template <class PS, int S>
__device__ __forceinline__ const SetT<PS, S> *set_plane(const float *base, int i, const Consts &K)
{
    const char *b = reinterpret_cast<const char *>(base) + (size_t)(unsigned)K.plane * (unsigned)set_bytes_before<PS>(S);
    return reinterpret_cast<const SetT<PS, S> *>(b) + (size_t)(unsigned)K.plane * (unsigned)i;
}
template <class PS, int S>
__device__ __forceinline__ SetT<PS, S> *set_plane(float *base, int i, const Consts &K)
{
    char *b = reinterpret_cast<char *>(base) + (size_t)(unsigned)K.plane * (unsigned)set_bytes_before<PS>(S);
    return reinterpret_cast<SetT<PS, S> *>(b) + (size_t)(unsigned)K.plane * (unsigned)i;
}

__device__ __forceinline__ real clamp01(real v) { return fmin(fmax(v, R(0.0)), R(1.0)); }

// Correctly rounded reciprocal (a division a / b below is a * rcp(b), within
// one unit in the last place of the quotient).
__device__ __forceinline__ float rcp(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp(double v) { return 1.0 / v; }

// Asynchronous 4-byte global -> shared copies (sm_80+ cp.async, cached in L1):
// the strip sweep stages the next row's inputs with them, so their latency
// overlaps the current row's arithmetic without holding registers.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// 16-byte form, cached in L2 only: both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Packed FP32 pairs for the sm_100+ f32x2 instructions, which add, subtract,
// multiply or fuse-multiply-add both halves of a 64-bit register at once
// (each half rounded as its FP32 counterpart).
typedef unsigned long long pf2;
__device__ __forceinline__ pf2 pk2(float lo, float hi)
{
    pf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(__float_as_uint(lo)), "r"(__float_as_uint(hi)));
    return r;
}
__device__ __forceinline__ pf2 pk2(float2 v) { return pk2(v.x, v.y); }
__device__ __forceinline__ pf2 splat2(float v) { return pk2(v, v); }
__device__ __forceinline__ float2 up2(pf2 v)
{
    unsigned lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(v));
    return make_float2(__uint_as_float(lo), __uint_as_float(hi));
}
__device__ __forceinline__ pf2 add2(pf2 a, pf2 b)
{
    pf2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ pf2 sub2(pf2 a, pf2 b)
{
    pf2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ pf2 mul2(pf2 a, pf2 b)
{
    pf2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ pf2 fma2(pf2 a, pf2 b, pf2 c)  // a * b + c
{
    pf2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Bottom-wall temperature at continuous abscissa x.
__device__ __forceinline__ real wall_T_bottom(const Consts &K, real x)
{
    return K.T_bottom_amp == R(0.0) ? K.T_bottom : K.T_bottom + K.T_bottom_amp * cospi(K.wall_k * x);
}

// Enthalpy -> (T, f_s) of Eq. Hfl with chi-weighted solidus / liquidus
// enthalpies (Eq. Hfl at chi = 1), f_s in [0, chi].  The enthalpy is passed
// as rho H = ed + rr T_p + rho_l L (chi_p - fs_p) with ed small, and chi with
// its change dchi = chi - chi_p formed from small terms, so that e - E_l,
// e - E_s and T - T_p are free of the large magnitudes.  Returns dT = T - T_p.
__device__ __forceinline__ void invert_enthalpy(const Consts &K, real ed, real T_p, real chi_p, real fs_p, real chi,
                                                real dchi, real &dT, real &fs)
{
    const real Al = chi * K.rcp_l + (R(1.0) - chi) * K.rcp_g;
    if (!K.phase_change) {
        dT = (ed + (K.rr - Al) * T_p) * rcp(Al);
        fs = R(0.0);
        return;
    }
    const real As = chi * K.rcp_s + (R(1.0) - chi) * K.rcp_g;
    const real lat_p = K.lat_l * (chi_p - fs_p);
    const real em_s = ed + K.rr * T_p + lat_p - As * K.T_sol;                   // e - E_s
    const real em_l = ed + K.rr * T_p - K.lat_l * (dchi + fs_p) - Al * K.T_liq;  // e - E_l
    if (em_s < R(0.0)) {
        fs = chi;
        dT = (ed + lat_p + (K.rr - As) * T_p) * rcp(As);
    } else if (em_l > R(0.0)) {
        fs = R(0.0);
        dT = (ed - K.lat_l * (dchi + fs_p) + (K.rr - Al) * T_p) * rcp(Al);
    } else {
        const real d = Al * K.T_liq - As * K.T_sol + chi * K.latent_l;
        const real r = (d < R(1e-14) * fmax(R(1.0), fabs(em_s))) ? R(1.0) : em_s * rcp(d);
        fs = chi * (R(1.0) - r);
        dT = (K.T_sol - T_p) + r * (K.T_liq - K.T_sol);
    }
}

// Forward map (T, chi) -> sensible enthalpy e - rho_l L (chi - f_s) and f_s;
// T exactly at T_s = T_l counts as liquid.
__device__ __forceinline__ real forward_sensible(const Consts &K, real T, real chi, real &fs)
{
    const real Al = chi * K.rcp_l + (R(1.0) - chi) * K.rcp_g;
    if (!K.phase_change) {
        fs = R(0.0);
        return Al * T;
    }
    const real As = chi * K.rcp_s + (R(1.0) - chi) * K.rcp_g;
    if (T >= K.T_liq) {
        fs = R(0.0);
        return Al * T;
    }
    if (T < K.T_sol) {
        fs = chi;
        return As * T;
    }
    const real r = (T - K.T_sol) / (K.T_liq - K.T_sol);
    fs = chi * (R(1.0) - r);
    return As * K.T_sol + r * (Al * K.T_liq - As * K.T_sol);
}

// Pull one stored post-collision population of set S into direction I at cell
// (x, y): from (x - c_I) in the bulk; from the own cell's opposite direction
// at a wall (half-way bounce-back).  For the enthalpy at a Dirichlet wall the
// anti-bounce-back rule h_I = -h*_opp + 2 w rr T_w (Sec. 4.5; the wall
// temperature at the foot of the cell on the wall, for all three links that
// cross it there) is applied in deviation form relative to w rr T_own.
// pull_src gives the address read, abb_fix the wall rule applied to its value.
template <class PS, int S, int I, bool W>
__device__ __forceinline__ const SetT<PS, S> *pull_src(const Consts &K, const float *__restrict__ pin, int x, int y,
                                                       int cell)
{
    constexpr int ys_off = -cy(I);
    const int ys = y + ys_off;
    if (W && ys_off != 0 && (ys < 0 || ys >= K.ny)) return set_plane<PS, S>(pin, opp(I), K) + cell;
    return set_plane<PS, S>(pin, I, K) + (ys * K.pitch + wrapx(x - cx(I), K.nx));
}

template <int S, int I, bool W>
__device__ __forceinline__ real abb_fix(const Consts &K, real v, int x, int y, real T_own)
{
    constexpr int ys_off = -cy(I);
    const int ys = y + ys_off;
    if (S == SET_H && W && ys_off != 0 && (ys < 0 || ys >= K.ny)) {
        const bool bottom = ys < 0;
        if ((bottom ? K.bc_bottom : K.bc_top) == WALL_DIRICHLET) {
            const real Tw = bottom ? wall_T_bottom(K, (real)x) : K.T_top;
            return -v + R(2.0) * wgt(I) * K.rr * (Tw - T_own);
        }
    }
    return v;
}

// Decoded stored value of set S, direction i: the deviation, and for the solute
// set in half storage the w_i c_ref shift added back.
template <class PS, int S>
__device__ __forceinline__ real dec_pop(const Consts &K, int i, SetT<PS, S> v)
{
    if constexpr (PS::esize(S) == 2 && S == SET_L)
        return dec_fma(v, wgt(i) * K.c_ref);
    else
        return dec_val(v);
}

template <class PS, int S>
__device__ __forceinline__ SetT<PS, S> enc_pop(const Consts &K, int i, real v)
{
    return enc_val<SetT<PS, S>>((PS::esize(S) == 2 && S == SET_L) ? v - wgt(i) * K.c_ref : v);
}

// Store population (set S, direction i) of cell into the output planes.
template <class PS, int S>
__device__ __forceinline__ void put_pop(const Consts &K, float *pout, int i, int cell, real v)
{
    set_plane<PS, S>(pout, i, K)[cell] = enc_pop<PS, S>(K, i, v);
}

template <class PS, int S, int I, bool W>
__device__ __forceinline__ real pull(const Consts &K, const float *__restrict__ pin, int x, int y, int cell, real T_own)
{
    return abb_fix<S, I, W>(K, dec_pop<PS, S>(K, I, __ldg(pull_src<PS, S, I, W>(K, pin, x, y, cell))), x, y, T_own);
}

// W = false: the caller guarantees that no source row lies beyond a wall.
template <class PS, int S, bool W = true>
__device__ __forceinline__ void pull9(const Consts &K, const float *__restrict__ pin, int x, int y, int cell, real v[9],
                                      real T_own = R(0.0))
{
    v[0] = pull<PS, S, 0, W>(K, pin, x, y, cell, T_own);
    v[1] = pull<PS, S, 1, W>(K, pin, x, y, cell, T_own);
    v[2] = pull<PS, S, 2, W>(K, pin, x, y, cell, T_own);
    v[3] = pull<PS, S, 3, W>(K, pin, x, y, cell, T_own);
    v[4] = pull<PS, S, 4, W>(K, pin, x, y, cell, T_own);
    v[5] = pull<PS, S, 5, W>(K, pin, x, y, cell, T_own);
    v[6] = pull<PS, S, 6, W>(K, pin, x, y, cell, T_own);
    v[7] = pull<PS, S, 7, W>(K, pin, x, y, cell, T_own);
    v[8] = pull<PS, S, 8, W>(K, pin, x, y, cell, T_own);
}

// Lagged field (plane A) of the cell that wrote the population pulled into
// direction I at (x, y) (the own cell at a wall).
template <int A, int I, bool W>
__device__ __forceinline__ real aux_src(const Consts &K, const float *__restrict__ ain, int x, int y, int cell)
{
    constexpr int ys_off = -cy(I);
    const int ys = y + ys_off;
    const float *a = plane_ptr(ain, A, K);
    if (W && ys_off != 0 && (ys < 0 || ys >= K.ny)) return __ldg(a + cell);
    return __ldg(a + (ys * K.pitch + wrapx(x - cx(I), K.nx)));
}

// sum_{i>0} w_i (z^n(source_i) - z^n(x)) of a lagged field: the reference
// offsets of the pulled deviations relative to the own lagged value.
template <int A, bool W = true, int Q = 9>
__device__ __forceinline__ real aux_dev_sum(const Consts &K, const float *__restrict__ ain, int x, int y, int cell,
                                            real own)
{
    if (Q == 5)  // the same order as the strip kernel's phase A (lag_dev_sums)
        return wfl<5>(1) * (((aux_src<A, 1, W>(K, ain, x, y, cell) - own) + (aux_src<A, 2, W>(K, ain, x, y, cell) - own)) +
                            ((aux_src<A, 3, W>(K, ain, x, y, cell) - own) + (aux_src<A, 4, W>(K, ain, x, y, cell) - own)));
    return (wgt(1) * (aux_src<A, 1, W>(K, ain, x, y, cell) - own) + wgt(2) * (aux_src<A, 2, W>(K, ain, x, y, cell) - own) +
            wgt(3) * (aux_src<A, 3, W>(K, ain, x, y, cell) - own) + wgt(4) * (aux_src<A, 4, W>(K, ain, x, y, cell) - own)) +
           (wgt(5) * (aux_src<A, 5, W>(K, ain, x, y, cell) - own) + wgt(6) * (aux_src<A, 6, W>(K, ain, x, y, cell) - own) +
            wgt(7) * (aux_src<A, 7, W>(K, ain, x, y, cell) - own) + wgt(8) * (aux_src<A, 8, W>(K, ain, x, y, cell) - own));
}

// Lagged velocity component (plane A = AUX_UX or AUX_UY) at the stencil
// neighbour (x + dx, y + dy); beyond a no-slip wall the ghost is -u of the
// adjacent row (linear extrapolation through u = 0 at the half-way wall).
template <int A, bool W>
__device__ __forceinline__ real u_nb(const Consts &K, const float *__restrict__ ain, int x, int y, int dx, int dy)
{
    const int yy = y + dy, xx = wrapx(x + dx, K.nx);
    const float *a = plane_ptr(ain, A, K);
    if (W && (yy < 0 || yy >= K.ny)) return -__ldg(a + (y * K.pitch + xx));
    return __ldg(a + (yy * K.pitch + xx));
}

// Isotropic divergence of the lagged velocity (end of Sec. 3.4 stencils):
// 3 sum_i w_i (c_ix u_x + c_iy u_y)(x + c_i), written per component.
template <bool W>
__device__ __forceinline__ real lagged_divu(const Consts &K, const float *__restrict__ ain, int x, int y)
{
    const real dudx = wgt(1) * (u_nb<AUX_UX, W>(K, ain, x, y, 1, 0) - u_nb<AUX_UX, W>(K, ain, x, y, -1, 0)) +
                      wgt(5) * ((u_nb<AUX_UX, W>(K, ain, x, y, 1, 1) - u_nb<AUX_UX, W>(K, ain, x, y, -1, 1)) +
                                (u_nb<AUX_UX, W>(K, ain, x, y, 1, -1) - u_nb<AUX_UX, W>(K, ain, x, y, -1, -1)));
    const real dvdy = wgt(2) * (u_nb<AUX_UY, W>(K, ain, x, y, 0, 1) - u_nb<AUX_UY, W>(K, ain, x, y, 0, -1)) +
                      wgt(5) * ((u_nb<AUX_UY, W>(K, ain, x, y, 1, 1) - u_nb<AUX_UY, W>(K, ain, x, y, 1, -1)) +
                                (u_nb<AUX_UY, W>(K, ain, x, y, -1, 1) - u_nb<AUX_UY, W>(K, ain, x, y, -1, -1)));
    return R(3.0) * (dudx + dvdy);
}

__device__ __forceinline__ real sum9(const real v[9])
{
    return v[0] + ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
}

// Local fields of one cell (Sec. 3.1, 3.3, 3.4, Eq. Hfl, Eq. NS1):
//   sum f = phi_p + delta, rho H = ed + rr T_p + rho_l L (chi_p - fs_p)
//   (ed includes Q^{n-1}/2), chi = clamp((1 + sum f)/2), (T, f_s) from the
//   enthalpy, mdot = (1 - rho_s/rho_l)(f_s - f_s^{n-1}),
//   phi = sum f / (1 - mdot/2) = phi_p + dphi, C = sum l.
struct Local {
    real dT, fs, mdot, divu, dphi, C;
};

// div_lag: the isotropic divergence of the previous step's velocity at the
// cell, used as div u when K.divu = 1 (ignored otherwise).
__device__ __forceinline__ Local local_fields(const Consts &K, real phi_p, real delta, real ed, real T_p, real chi_p,
                                              real fs_p, real sl, real div_lag)
{
    Local o;
    // phi = sum f + phi div u / 2 (Sec. 3.1), solved for phi.  With the lagged
    // velocity divergence phi is known before the enthalpy relation, and the
    // material fraction chi of Eq. Hfl is that of phi; with div u = mdot, which
    // needs f_s first, chi is taken from sum f.
    real dphi = R(0.0);
    if (K.divu) dphi = (delta + R(0.5) * div_lag * phi_p) * rcp(R(1.0) - R(0.5) * div_lag);
    const real dsf = K.divu ? dphi : delta;  // change of the argument of chi
    const real hs = R(0.5) * (R(1.0) + (phi_p + dsf)), hp = R(0.5) * (R(1.0) + phi_p);
    const real chi = clamp01(hs);
    const bool inside = hs >= R(0.0) && hs <= R(1.0) && hp >= R(0.0) && hp <= R(1.0);
    const real dchi = inside ? R(0.5) * dsf : chi - chi_p;
    invert_enthalpy(K, ed, T_p, chi_p, fs_p, chi, dchi, o.dT, o.fs);
    o.mdot = K.phase_change ? K.expand * (o.fs - fs_p) : R(0.0);
    o.divu = K.divu ? div_lag : o.mdot;
    if (!K.divu) dphi = (delta + R(0.5) * o.mdot * phi_p) * rcp(R(1.0) - R(0.5) * o.mdot);
    o.dphi = dphi;
    o.C = sl;
    return o;
}

// Phase-A work for one cell: pull f, h, l and the lagged values it needs.
struct CellA {
    Local L;
    real ed, chi_p, fs_p, phi_p, T_p;
};

template <class PS, bool W = true>
__device__ __forceinline__ CellA cell_a(const Consts &K, const float *__restrict__ pin, const float *__restrict__ ain,
                                        int x, int y, int cell)
{
    CellA c;
    real v[9];
    c.phi_p = __ldg(plane_ptr(ain, AUX_PHI, K) + cell);
    c.T_p = __ldg(plane_ptr(ain, AUX_T, K) + cell);
    c.fs_p = __ldg(plane_ptr(ain, AUX_FS, K) + cell);
    c.chi_p = clamp01(R(0.5) * (R(1.0) + c.phi_p));
    pull9<PS, SET_F, W>(K, pin, x, y, cell, v);
    const real delta = sum9(v) + aux_dev_sum<AUX_PHI, W, PS::QFL>(K, ain, x, y, cell, c.phi_p);
    pull9<PS, SET_H, W>(K, pin, x, y, cell, v, c.T_p);
    const real Q_p = __ldg(plane_ptr(ain, AUX_Q, K) + cell);
    c.ed = sum9(v) + K.rr * aux_dev_sum<AUX_T, W>(K, ain, x, y, cell, c.T_p) + R(0.5) * Q_p;
    pull9<PS, SET_L, W>(K, pin, x, y, cell, v);
    const real sl = sum9(v);
    const real dv = K.divu ? lagged_divu<W>(K, ain, x, y) : R(0.0);
    c.L = local_fields(K, c.phi_p, delta, c.ed, c.T_p, c.chi_p, c.fs_p, sl, dv);
    return c;
}

// Error-free sum (Knuth's TwoSum, round to nearest): a + b = s + e exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// The diagnostics of one cell (sums of phi, rho H, C, f_s and chi over the
// lattice, Sec. 4.2 and 4.4) as seven FP32 addends, chosen so that their sums
// keep the accuracy of an FP64 evaluation: phi as its two FP32 parts phi_p and
// dphi; rho H = (sum h + rr dT + Q/2) + rr T_p + rho_l L (chi_p - f_s,p), whose
// cell terms cancel across the lattice, as an FP32 pair hi + lo from
// error-free products and sums (error of order 2^-48 of the terms); C, f_s and
// chi of the new phi.  FP64 is the scarce pipe on this GPU, so these are
// added in FP32 with compensation where many cells are summed, and in FP64
// elsewhere; both sums agree to about 1e-13.
struct DiagTerms {
    float t[7];
};
__device__ __forceinline__ DiagTerms diag_terms(const Consts &K, real phi_p, real dphi, real ed, real T_p, real chi_p,
                                                real fs_p, real C, real fs)
{
    DiagTerms d;
    float dlo, e1, e2;
    const float dc = two_sum(chi_p, -fs_p, dlo);
    const float p = __fmul_rn(K.rr, T_p), plo = __fmaf_rn(K.rr, T_p, -p);
    const float q = __fmul_rn(K.lat_l, dc), qlo = __fmaf_rn(K.lat_l, dc, -q);
    const float s1 = two_sum(ed, p, e1);
    d.t[0] = phi_p;
    d.t[1] = dphi;
    d.t[2] = two_sum(s1, q, e2);
    d.t[3] = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(plo, qlo)), __fmul_rn(K.lat_l, dlo));
    d.t[4] = C;
    d.t[5] = fs;
    d.t[6] = clamp01(R(0.5) * (R(1.0) + __fadd_rn(phi_p, dphi)));
    return d;
}
// FP64 sums of the diagnostics (acc[5]: f_s on the centre column).
__device__ __forceinline__ void add_diag(const Consts &K, real phi_p, real dphi, real ed, real T_p, real chi_p, real fs_p,
                                         real C, real fs, bool centre, double acc[6])
{
    const DiagTerms d = diag_terms(K, phi_p, dphi, ed, T_p, chi_p, fs_p, C, fs);
    acc[0] += (double)d.t[0] + (double)d.t[1];
    acc[1] += (double)d.t[2] + (double)d.t[3];
    acc[2] += (double)d.t[4];
    acc[3] += (double)d.t[5];
    acc[4] += (double)d.t[6];
    if (centre) acc[5] += (double)fs;
}
// Compensated FP32 sum (TwoSum, the rounding errors gathered in c).
struct CompSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        float e;
        s = two_sum(s, x, e);
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Own-cell lagged values staged for phase B (the accessor's aux(k)).
enum { AX_Q = 0, AX_FS = 1, AX_C = 2, NAX = 3 };

// MODE_STEP collides and streams; MODE_FIELDS stores the macroscopic fields of the
// current state instead; MODE_REDUCE runs phase A only and sums the diagnostics.
enum { MODE_STEP = 0, MODE_FIELDS = 1, MODE_REDUCE = 2 };

// ---------------------------------------------------------------------------------------
// Phase B of one interior cell: gradients, forces, velocity, pressure and the
// collision of the four sets (or, in MODE_FIELDS, the macroscopic fields).  The
// accessor A supplies the step's local fields of the cell and its neighbours
// (offsets dy, dx in {-1, 0, 1}, already mirrored at walls) and the cell's
// pulled f, h, l and g, and its own lagged Q, f_s, u and C.
// ---------------------------------------------------------------------------------------
template <int MODE, bool WALLS, class PS, class Acc>
__device__ __forceinline__ void phase_b(const Consts &K, const Buffers &B, const Acc &A, int x, int y, int cell)
{
    const real rr = K.rr;
    const bool at_bottom = WALLS && (y == 0), at_top = WALLS && (y == K.ny - 1);
    const int ds = at_bottom ? 0 : -1;  // south row offset (mirror ghost at the bottom wall)
    const int dn = at_top ? 0 : 1;      // north row offset
    const bool dir_b = at_bottom && K.bc_bottom == WALL_DIRICHLET;
    const bool dir_t = at_top && K.bc_top == WALL_DIRICHLET;

    // own fields: phi = phi_p + dphi, T = T_p + dT; phi_st, T_st are the values
    // written to the lagged fields, which are also the references of the stored
    // deviations (the parts below the FP32 spacing stay in those deviations)
    const real phi_p = A.phip(0, 0), dphi = A.dphi(0, 0);
    const real phi_st = (real)(float)(phi_p + dphi);
    const real phi_lo = (phi_p - phi_st) + dphi;  // phi - phi_st
    const real phi = phi_st + phi_lo;
    const real T_p = A.Tp(0, 0), dT = A.dT(0, 0);
    const real T_st = (real)(float)(T_p + dT);
    const real T_lo = (T_p - T_st) + dT;          // T - T_st
    const real T = T_st + T_lo;
    const real C = A.C(0, 0), fs = (real)(float)A.fs(0, 0);
    const real mdot = A.mdot(0, 0);
    const real divu = A.divu();  // div u of the phi and h sources (mdot, or the lagged velocity divergence)

    // isotropic gradient and Laplacian over the 8 neighbours (order 1..8), from
    // differences z_i - z_0: grad z = 3 sum w_i c_i (z_i - z_0), lap z = 6 sum w_i (z_i - z_0).
    // phi and T differences are split into lagged-value and change parts.  Wall rows
    // are ghosts: mirror, the wetting ghost for phi, or 2 T_w - T_adjacent for the
    // temperature at a Dirichlet wall.
    real gpx, gpy, lphi, gTx, gTy, gCx, gCy, gfx, gfy, gPx, gPy, gSx, gSy;
    {
        // the six fields run as three packed pairs: (phi, T), (C, f_s), (p, S)
        const int dxv[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        const int dyv[9] = {0, 0, dn, 0, ds, dn, dn, ds, ds};
        const pf2 lag0 = pk2(phi_p, T_p), dd0 = pk2(dphi, dT);
        const pf2 cf0 = pk2(A.cfv(0, 0)), ps0 = pk2(A.psv(0, 0));
        pf2 sx01 = 0, sy01 = 0, sx23 = 0, sy23 = 0, sx45 = 0, sy45 = 0;  // bit pattern of (0, 0)
        real sl = R(0.0);
#pragma unroll
        for (int i = 1; i < 9; i++) {
            const int a = dyv[i], b = dxv[i];
            const float2 lg = A.lagv(a, b), dd = A.ddv(a, b);
            pf2 z01;  // (phi_i - phi_0, T_i - T_0)
            if (!WALLS) {
                z01 = add2(sub2(pk2(lg), lag0), sub2(pk2(dd), dd0));
            } else {
                real zph = (lg.x - phi_p) + (dd.x - dphi);
                if ((at_bottom && cy(i) == -1) || (at_top && cy(i) == 1)) {
                    // wetting ghost: phi_adj + cos(theta) (1 - phi_adj^2) / (sqrt 2 eps)
                    const real wet = cy(i) == -1 ? K.wet_b : K.wet_t;
                    const real pa = lg.x + dd.x;
                    zph += wet * (R(1.0) - pa * pa);
                }
                real zT = (lg.y - T_p) + (dd.y - dT);
                if ((dir_b && cy(i) == -1) || (dir_t && cy(i) == 1)) {
                    const real Tw = cy(i) == -1 ? wall_T_bottom(K, (real)wrapx(x + cx(i), K.nx)) : K.T_top;
                    // ghost - T_0 = 2 T_w - T_adj - T_0 = 2 (T_w - Tp_adj) + (Tp_adj - Tp_0) - dT_adj - dT_0
                    zT = R(2.0) * (Tw - lg.y) + (lg.y - T_p) - (dd.y + dT);
                }
                z01 = pk2(zph, zT);
            }
            const pf2 z23 = sub2(pk2(A.cfv(a, b)), cf0), z45 = sub2(pk2(A.psv(a, b)), ps0);
            if (cx(i) != 0) {
                const pf2 w = splat2(wgt(i) * (real)cx(i));
                sx01 = fma2(w, z01, sx01);
                sx23 = fma2(w, z23, sx23);
                sx45 = fma2(w, z45, sx45);
            }
            if (cy(i) != 0) {
                const pf2 w = splat2(wgt(i) * (real)cy(i));
                sy01 = fma2(w, z01, sy01);
                sy23 = fma2(w, z23, sy23);
                sy45 = fma2(w, z45, sy45);
            }
            sl += R(2.0) * wgt(i) * up2(z01).x;
        }
        const float2 gx01 = up2(sx01), gy01 = up2(sy01), gx23 = up2(sx23), gy23 = up2(sy23);
        const float2 gx45 = up2(sx45), gy45 = up2(sy45);
        gpx = R(3.0) * gx01.x; gpy = R(3.0) * gy01.x; lphi = R(3.0) * sl;
        gTx = R(3.0) * gx01.y; gTy = R(3.0) * gy01.y;
        gCx = R(3.0) * gx23.x; gCy = R(3.0) * gy23.x;
        gfx = R(3.0) * gx23.y; gfy = R(3.0) * gy23.y;
        gPx = R(3.0) * gx45.x; gPy = R(3.0) * gy45.x;
        gSx = R(3.0) * gx45.y; gSy = R(3.0) * gy45.y;
    }

    // properties by the linear rule; the density gradient follows from it exactly
    const real rho = zeta(phi, fs, K.rho_l, K.rho_s, K.rho_g);
    const real mu = zeta(phi, fs, K.mu_l, K.mu_s, K.mu_g);
    const real lam = zeta(phi, fs, K.lam_l, K.lam_s, K.lam_g);
    const real rhocp = zeta(phi, fs, K.rcp_l, K.rcp_s, K.rcp_g);
    const real dr_phi = R(0.5) * (K.rho_l - K.rho_g), dr_fs = K.rho_s - K.rho_l;
    const real grx = dr_phi * gpx + dr_fs * gfx, gry = dr_phi * gpy + dr_fs * gfy;

    // normal, chemical potential, surface tension and its gradient
    const real g2 = gpx * gpx + gpy * gpy;
    const real inv = rsqrt(g2 + R(1e-6));  // regularised normal: smooth away from the interface
    const real nxv = gpx * inv, nyv = gpy * inv;
    // chemical potential (phi^3 - phi)/eps^2 - lap phi: the cubic term as
    // phi (phi - 1)(phi + 1), each factor formed as (phi_st -/+ 1) + phi_lo with
    // phi_st -/+ 1 exact near the bulk values, so that the term keeps its relative
    // precision where it is small (phi near +-1)
    const real phi2m1 = ((phi_st - R(1.0)) + phi_lo) * ((phi_st + R(1.0)) + phi_lo);  // phi^2 - 1
    const real muphi = phi * phi2m1 * K.inv_eps2 - lphi;
    const real sigma = K.sigma0 + K.sigma_T * (T - K.T_ref) + K.sigma_c * (C - K.c_ref);
    const real gsx = K.sigma_T * gTx + K.sigma_c * gCx;
    const real gsy = K.sigma_T * gTy + K.sigma_c * gCy;

    // Eq. Fs: Marangoni part alpha (|grad phi|^2 grad sigma - (grad sigma . grad phi) grad phi)
    // plus capillary part alpha sigma mu_phi grad phi, times (1 - f_s) when modulated
    const real gsgp = gsx * gpx + gsy * gpy;
    real Fsx = K.alpha * (g2 * gsx - gsgp * gpx) + K.alpha * sigma * muphi * gpx;
    real Fsy = K.alpha * (g2 * gsy - gsgp * gpy) + K.alpha * sigma * muphi * gpy;
    if (K.fs_mod) {
        Fsx *= (R(1.0) - fs);
        Fsy *= (R(1.0) - fs);
    }
    const real Fx = Fsx + rho * K.gx, Fy = Fsy + rho * K.gy;

    // flow set: velocity and pressure (Sec. 3.2).  g is stored as deviations from
    // 3 p^n(s) (w_i - [i = 0]); dg_i = g_i - 3 p_p (w_i - [i = 0]) with p_p the own
    // lagged pressure, so that the momentum and the pressure are sums of small terms
    const real p_p = A.p(0, 0);
    real g[9], dg[9];
    A.gpops(K, g);
    real jx = R(0.0), jy = R(0.0), sg = R(0.0);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const int ys = y - cy(i);
        const bool wall = WALLS && cy(i) != 0 && (ys < 0 || ys >= K.ny);
        const real pps = (i == 0 || wall) ? p_p : A.p(-cy(i), -cx(i));
        dg[i] = g[i] + R(3.0) * (wgt(i) - (i == 0 ? R(1.0) : R(0.0))) * (pps - p_p);
        jx += (real)cx(i) * dg[i];
        jy += (real)cy(i) * dg[i];
        if (i) sg += dg[i];
    }
    const real inv_rho = rcp(rho);
    const real usx = (jx + R(0.5) * Fx) * inv_rho, usy = (jy + R(0.5) * Fy) * inv_rho;
    const real ffx = -fs * usx, ffy = -fs * usy;       // f = f_s (0 - u*)
    const real ux = usx + R(0.5) * ffx, uy = usy + R(0.5) * ffy;
    const real rfx = rho * ffx, rfy = rho * ffy;
    const real S = rho * mdot + ux * grx + uy * gry;
    const real Ftx = Fx - gPx + (R(1.0) / R(3.0)) * grx + (R(1.0) / R(3.0)) * gSx;
    const real Fty = Fy - gPy + (R(1.0) / R(3.0)) * gry + (R(1.0) / R(3.0)) * gSy;
    const real tau_g = R(0.5) + R(3.0) * mu * inv_rho;
    const real uu = ux * ux + uy * uy;
    const real uF = ux * Ftx + uy * Fty;
    const real G0 = wgt(0) * (S - R(3.0) * uF);
    const real s0 = wgt(0) * (-R(1.5) * uu);
    // p = c_s^2/(1 - w_0) [sum_{i>0} g_i + S/2 + tau G_0 + rho s_0(u)] = p_p + dp
    const real dp = (R(1.0) / R(3.0)) / (R(1.0) - wgt(0)) * (sg + R(0.5) * S + tau_g * G0 + rho * s0);
    const real p_st = (real)(float)(p_p + dp);
    const real p_lo = (p_p - p_st) + dp;  // p - p_st
    const real pr = p_st + p_lo;

    if (MODE == MODE_FIELDS) {
        float *o = B.fields;
        plane_ptr(o, 0, K)[cell] = phi;
        plane_ptr(o, 1, K)[cell] = T;
        plane_ptr(o, 2, K)[cell] = fs;
        plane_ptr(o, 3, K)[cell] = C;
        plane_ptr(o, 4, K)[cell] = ux;
        plane_ptr(o, 5, K)[cell] = uy;
        plane_ptr(o, 6, K)[cell] = pr;
        return;
    }

    // The collisions run over the rest direction and the four pairs (i, opp(i))
    // with c_opp = -c_i: every equilibrium and source term splits into a part
    // even in c_i, shared by the pair, and an odd part that changes sign.  The
    // pairs go two at a time, (1, 2) and (5, 6) -- each two of equal weight -- as
    // packed f32x2 values: "p" holds directions (a, a + 1), "m" their opposites.
    float *__restrict__ pout = B.pout;
    auto store4 = [&](auto set, int a, const pf2 vp, const pf2 vm) {  // set: integral_constant of the set
        constexpr int S = decltype(set)::value;
        const float2 op = up2(vp), om2 = up2(vm);
        put_pop<PS, S>(K, pout, a, cell, op.x);
        put_pop<PS, S>(K, pout, a + 1, cell, op.y);
        put_pop<PS, S>(K, pout, opp(a), cell, om2.x);
        put_pop<PS, S>(K, pout, opp(a + 1), cell, om2.y);
    };
    // (c_a . v, c_{a+1} . v)
    auto cdot2 = [](int a, real vx, real vy) {
        return pk2((real)cx(a) * vx + (real)cy(a) * vy, (real)cx(a + 1) * vx + (real)cy(a + 1) * vy);
    };
    const pf2 u2 = splat2(R(-1.5) * uu);

    // flow set (Sec. 3.2); d_i = g_i - 3 p_st (w_i - [i = 0]) is formed from the
    // stored deviation, the reference of the stored value being 3 p_st (w_i - [i = 0])
    const real om_g = rcp(tau_g), src_g = R(1.0) - R(0.5) * om_g;
    {
        const real dpp = p_p - p_st;
        const real Fqx = Fx + rfx, Fqy = Fy + rfy;  // F + rho f
        {
            const real wp = R(3.0) * (wgt(0) - R(1.0));
            const real d = dg[0] + wp * dpp;
            const real deq = wp * p_lo + rho * (wgt(0) * (-R(1.5) * uu));
            const real G0 = wgt(0) * (S - R(3.0) * uF);
            put_pop<PS, SET_G>(K, pout, 0, cell, d - (d - deq) * om_g + src_g * G0);
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int a = q == 0 ? 1 : 5;
            const real w = wgt(a), w3 = R(3.0) * w;
            const pf2 cu = cdot2(a, ux, uy), cF = cdot2(a, Ftx, Fty), cG = cdot2(a, Fqx, Fqy);
            const pf2 eq_e = fma2(splat2(rho * w), fma2(splat2(R(4.5)), mul2(cu, cu), u2), splat2(w3 * p_lo));
            const pf2 eq_o = mul2(splat2(rho * w3), cu);
            const pf2 G_e = fma2(splat2(R(9.0) * w), mul2(cu, cF), splat2(w * (S - R(3.0) * uF)));
            const pf2 G_o = mul2(splat2(w3), cG);
            const pf2 sh = splat2(w3 * dpp);
            const pf2 dp = add2(pk2(dg[a], dg[a + 1]), sh), dm = add2(pk2(dg[opp(a)], dg[opp(a + 1)]), sh);
            const pf2 sg = splat2(src_g), og = splat2(om_g);
            store4(std::integral_constant<int, SET_G>{}, a, fma2(sg, add2(G_e, G_o), fma2(sub2(add2(eq_e, eq_o), dp), og, dp)),
                   fma2(sg, sub2(G_e, G_o), fma2(sub2(sub2(eq_e, eq_o), dm), og, dm)));
        }
    }

    // phase-field set (Sec. 3.1): F_i = w c.[d_t(phi u) + cs2 n (1 - phi^2)/(sqrt2 eps)]/cs2 + w phi div u
    {
        const float2 u_p = A.lagu();
        const real ux_p = u_p.x, uy_p = u_p.y;
        const real kf = -(R(1.0) / R(3.0)) * phi2m1 * K.inv_s2eps;
        const real ax = (phi * ux - phi_p * ux_p) + kf * nxv;
        const real ay = (phi * uy - phi_p * uy_p) + kf * nyv;
        const real om = K.om_f, src = K.src_f;
        // d_i = f_i - w_i phi_st: the stored deviation plus w_i (phi^n(source) - phi_st);
        // stored as f_i* - w_i phi_st
        real f[9];
        A.template pops<SET_F>(K, B.pin, x, y, cell, f, R(0.0));
        constexpr int QF = PS::QFL;
        {
            const real d = f[0] + wfl<QF>(0) * (phi_p - phi_st);
            const real deq = wfl<QF>(0) * phi_lo;
            put_pop<PS, SET_F>(K, pout, 0, cell, d - (d - deq) * om + src * (wfl<QF>(0) * phi * divu));
        }
        // lagged phi of the cell that wrote the population pulled into direction i (own cell at a wall)
        auto php = [&](int i) {
            const int ys = y - cy(i);
            return (WALLS && cy(i) != 0 && (ys < 0 || ys >= K.ny)) ? phi_p : A.phip(-cy(i), -cx(i));
        };
#pragma unroll
        for (int q = 0; q < (QF == 9 ? 2 : 1); q++) {
            const int a = q == 0 ? 1 : 5;
            const real w = wfl<QF>(a), w3 = R(3.0) * w;
            const pf2 ws = splat2(w), ps = splat2(phi_st);
            const pf2 dp = fma2(ws, sub2(pk2(php(a), php(a + 1)), ps), pk2(f[a], f[a + 1]));
            const pf2 dm = fma2(ws, sub2(pk2(php(opp(a)), php(opp(a + 1))), ps), pk2(f[opp(a)], f[opp(a + 1)]));
            const pf2 eq_e = splat2(w * phi_lo), eq_o = mul2(splat2(w3 * phi), cdot2(a, ux, uy));  // f_eq - w phi_st
            const pf2 F_e = splat2(w * phi * divu), F_o = mul2(splat2(w3), cdot2(a, ax, ay));
            const pf2 sf = splat2(src), of = splat2(om);
            store4(std::integral_constant<int, SET_F>{}, a, fma2(sf, add2(F_e, F_o), fma2(sub2(add2(eq_e, eq_o), dp), of, dp)),
                   fma2(sf, sub2(F_e, F_o), fma2(sub2(sub2(eq_e, eq_o), dm), of, dm)));
        }

        // solute set (Sec. 3.4): R = (1-phi) C n/(sqrt2 eps) - (k_p - 1) C grad(1 - f_s)/k_eff
        const real C_p = A.aux(AX_C);
        const real keff = R(1.0) - fs * (R(1.0) - K.k_p);
        const real inv_keff = rcp(keff);
        const real De = fs * K.k_p * K.D_s + (R(1.0) - fs) * K.D_l;
        const real tau_l = R(0.5) + R(3.0) * De * inv_keff;
        const real om_l = rcp(tau_l), src_l = R(1.0) - R(0.5) * om_l;
        const real Rx = (R(1.0) - phi) * C * nxv * K.inv_s2eps + (K.k_p - R(1.0)) * C * gfx * inv_keff;
        const real Ry = (R(1.0) - phi) * C * nyv * K.inv_s2eps + (K.k_p - R(1.0)) * C * gfy * inv_keff;
        const real bx = (C * ux - C_p * ux_p) + (R(1.0) / R(3.0)) * Rx;
        const real by = (C * uy - C_p * uy_p) + (R(1.0) / R(3.0)) * Ry;
        real l[9];
        A.template pops<SET_L>(K, B.pin, x, y, cell, l, R(0.0));
        put_pop<PS, SET_L>(K, pout, 0, cell, l[0] - (l[0] - wfl<QF>(0) * C) * om_l);
#pragma unroll
        for (int q = 0; q < (QF == 9 ? 2 : 1); q++) {
            const int a = q == 0 ? 1 : 5;
            const real w = wfl<QF>(a), w3 = R(3.0) * w;
            const pf2 eq_e = splat2(w * C), eq_o = mul2(splat2(w3 * C), cdot2(a, ux, uy));
            const pf2 sL = mul2(splat2(src_l * w3), cdot2(a, bx, by));  // src_l L_i, odd
            const pf2 lp = pk2(l[a], l[a + 1]), lm = pk2(l[opp(a)], l[opp(a + 1)]), ol = splat2(om_l);
            store4(std::integral_constant<int, SET_L>{}, a, add2(fma2(sub2(add2(eq_e, eq_o), lp), ol, lp), sL),
                   sub2(fma2(sub2(sub2(eq_e, eq_o), lm), ol, lm), sL));
        }
    }

    // enthalpy set (Sec. 3.3), two relaxation times: antisymmetric part with
    // tau_bar = 1/2 + lam/(rho_ref Cp_ref cs2), symmetric part with 1/tau_tilde = 2 - 1/tau_bar;
    // isotropic source w_i Q weighted with (1 - 1/(2 tau_tilde)).  Everything is formed as
    // deviations from w_i rr T_st (and the latent reference for i = 0).  For a pair the
    // symmetric and antisymmetric equilibrium parts are the even and odd parts above.
    const real Q = rhocp * T * divu;
    {
        const real tau_hb = R(0.5) + R(3.0) * lam * K.inv_rr;
        const real om_a = rcp(tau_hb), om_s = R(2.0) - om_a;
        const real src_h = R(1.0) - R(0.5) * om_s;
        const real rcT = rhocp * T;
        real h[9];
        A.template pops<SET_H>(K, B.pin, x, y, cell, h, T_p);
        auto Tps = [&](int i) {
            const int ys = y - cy(i);
            return (WALLS && cy(i) != 0 && (ys < 0 || ys >= K.ny)) ? T_p : A.Tp(-cy(i), -cx(i));
        };
        pf2 snz2 = 0;  // sum_{i>0} (h_i - w_i rr T_st), two halves
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int a = q == 0 ? 1 : 5;
            const real w = wgt(a);
            const pf2 wr = splat2(w * rr), ts = splat2(T_st);
            const pf2 dhp = fma2(wr, sub2(pk2(Tps(a), Tps(a + 1)), ts), pk2(h[a], h[a + 1]));
            const pf2 dhm = fma2(wr, sub2(pk2(Tps(opp(a)), Tps(opp(a + 1))), ts), pk2(h[opp(a)], h[opp(a + 1)]));
            const pf2 cu = cdot2(a, ux, uy);
            const pf2 es = fma2(splat2(w * rcT), fma2(splat2(R(4.5)), mul2(cu, cu), u2), splat2(w * rr * T_lo));
            const pf2 ea = mul2(splat2(w * rcT * R(3.0)), cu);
            const pf2 half = splat2(R(0.5));
            const pf2 hs = mul2(half, add2(dhp, dhm)), ha = mul2(half, sub2(dhp, dhm));
            const pf2 rel_s = mul2(sub2(hs, es), splat2(om_s)), rel_a = mul2(sub2(ha, ea), splat2(om_a));
            const pf2 base = sub2(splat2(src_h * w * Q), rel_s);
            store4(std::integral_constant<int, SET_H>{}, a, add2(sub2(dhp, rel_a), base), add2(add2(dhm, rel_a), base));
            snz2 = add2(snz2, add2(dhp, dhm));
        }
        const float2 snzv = up2(snz2);
        const real snz = snzv.x + snzv.y;
        // rest population: h_0 - h_eq_0 = -(sum_{i>0} h_i + Q^{n-1}/2) + (1 - w_0) rr T
        // + w_0 rho Cp T 3 u.u/2 exactly (sum_i h_eq_i = rho H); the stored reference
        // moves from w_0 rr T_p + rho_l L (chi_p - fs_p) to w_0 rr T_st + rho_l L (chi_st - f_s)
        {
            const real Q_p = A.aux(AX_Q);
            const real fs_p = A.aux(AX_FS);
            const real chi_p = clamp01(R(0.5) * (R(1.0) + phi_p));
            const real chi_n = clamp01(R(0.5) * (R(1.0) + phi_st));
            // sum_{i>0} h_i - (1 - w_0) rr T = sum_{i>0} dh_i - (1 - w_0) rr T_lo
            const real dev0 = wgt(0) * rcT * R(1.5) * uu - (snz - (R(1.0) - wgt(0)) * rr * T_lo) - R(0.5) * Q_p;
            const real dref = wgt(0) * rr * (T_p - T_st) + K.lat_l * ((chi_p - chi_n) - (fs_p - fs));
            put_pop<PS, SET_H>(K, pout, 0, cell, h[0] + dref - dev0 * om_s + src_h * wgt(0) * Q);
        }
    }

    // lagged fields for the next step
    float *__restrict__ aout = B.aout;
    plane_ptr(aout, AUX_FS, K)[cell] = fs;
    plane_ptr(aout, AUX_Q, K)[cell] = Q;
    plane_ptr(aout, AUX_UX, K)[cell] = ux;
    plane_ptr(aout, AUX_UY, K)[cell] = uy;
    plane_ptr(aout, AUX_PHI, K)[cell] = (float)phi_st;
    plane_ptr(aout, AUX_C, K)[cell] = C;
    plane_ptr(aout, AUX_P, K)[cell] = (float)p_st;
    plane_ptr(aout, AUX_S, K)[cell] = S;
    plane_ptr(aout, AUX_T, K)[cell] = (float)T_st;

    // a non-finite value anywhere in the cell's new state is reported once
    if (!isfinite(T + phi + C + ux + uy + pr)) atomicOr(B.status, 1u);
}



// ---------------------------------------------------------------------------------------
// Strip form of the step (see the top of this file).  Every global value a
// warp needs is staged into its rings by cp.async one row ahead of its use:
// while the warp computes phase A of row y and phase B of row y - 1, the
// copies for phase A of row y + 1 (and phase B of row y) are in flight.
// Rings per warp (columns x0-2 .. x0+31 for lag and uv, the warp's 32 lanes otherwise;
// WarpRing below, sized per storage form):
//   lag  lagged (phi, T) pairs                             rows y mod 5
//   uv   lagged (u_x, u_y) pairs                           rows y mod 5
//   dd, cf, md, dv  (dphi, dT), (C, f_s), mdot, div u from phase A   rows y mod 3
//   ps   staged lagged (p, S) pairs                        rows y & 3
//   pop  staged pulls of f, h, l (stored form), windows    rows y mod 3
//   ax   staged own-cell Q, f_s, C, windows                rows y mod 3
//   gp   staged pulls of g, windows                        rows y & 1
// One launch covers the lattice.  Per group of LB_SW strips it has two bands with
// the wall rules -- rows 0 .. 1 and rows ny-2 .. ny-1 -- and segments of K.segh
// rows inside 2 .. ny-3, whose rows and pull sources (ys - 2 .. ye + 1) all lie
// inside the lattice and which run without any wall rule.  Blocks are numbered
// strip group fastest, the two bands first.
// ---------------------------------------------------------------------------------------
#ifndef LB_SW
#define LB_SW 2
#endif
// Inner segment height of single-lattice handles, per kernel kind (measured on
// the 4096^2 step): FP32 D2Q9 is fastest at 8-12 rows (32 rows: 5 % slower);
// the half forms and D2Q5 f/l at 32 rows (24 rows: 0.7-1.3 % slower).  The host
// shortens them where a lattice gives the wave too few work items.
#ifndef LB_SEGH
#define LB_SEGH 12
#endif
#ifndef LB_SEGH_ALT
#define LB_SEGH_ALT 32
#endif

constexpr int NRED = 6;  // diagnostics: sums of phi, rho H, C, f_s, chi, and f_s on the column x = nx/2

// Staged planes are windows of WW columns starting at a 16-byte boundary x_lo
// <= x0 - 2; lane l (column x0 - 1 + l) finds the value pulled into direction i
// at index l + off - c_ix, off = x0 - 1 - x_lo (in 1 .. 4).
constexpr int WW = 40;

// Bytes of a staged window slot of set S: 40 FP32 or 48 half columns.
template <class PS>
__host__ __device__ constexpr int win_bytes(int s)
{
    return PS::esize(s) == 2 ? 96 : 160;
}
// Elements of a staged window slot of set S in its storage type.
template <class PS, int S>
__host__ __device__ constexpr int win_elems()
{
    return win_bytes<PS>(S) / PS::esize(S);
}

// The rings of one warp under storage PS (windows of half sets take 96 bytes,
// so a warp's rings are smaller and more warps fit on an SM).  PB = false:
// the rings of a sweep that runs phase A alone (the diagnostics), without the
// phase-A outputs, the staged (p, S) and the g pulls that only phase B reads
// (one placeholder row each, never touched).
template <class PS, bool PB = true>
struct WarpRing {
    static constexpr int OFF_H = 9 * win_bytes<PS>(SET_F);            // h windows in a pop row
    static constexpr int OFF_L = OFF_H + 9 * win_bytes<PS>(SET_H);    // l windows
    static constexpr int POPROW = OFF_L + 9 * win_bytes<PS>(SET_L);   // bytes of one pop row
    float2 lag[5][34];    // (phi, T) lagged           rows y mod 5
    float2 dd[PB ? 3 : 1][32];     // (dphi, dT)                 rows y mod 3
    float2 cf[PB ? 3 : 1][32];     // (C, f_s)                   rows y mod 3
    float2 ps[PB ? 4 : 1][32];     // (p, S) lagged, staged      rows y & 3
    float md[PB ? 3 : 1][32];      // mdot                       rows y mod 3
    float dv[PB ? 3 : 1][32];      // div u of the phi and h sources, rows y mod 3
    float2 uv[5][34];     // lagged (u_x, u_y), staged    rows y mod 5
    float ax[3][NAX][WW];  // staged own-cell Q, f_s, C   rows y mod 3
    alignas(16) unsigned char pop[3][POPROW];       // staged pulls of f, h, l (windows 0..8 of each)
    alignas(16) unsigned char gp[PB ? 2 : 1][PB ? 9 * win_bytes<PS>(SET_G) : 16];  // staged pulls of g
    // first element of window i of set S (f, h or l) in pop row r, or of g in gp row r
    template <int S>
    __device__ SetT<PS, S> *win(int r, int i)
    {
        unsigned char *b = S == SET_G ? &gp[r][0] : &pop[r][S == SET_F ? 0 : (S == SET_H ? OFF_H : OFF_L)];
        return reinterpret_cast<SetT<PS, S> *>(b) + i * win_elems<PS, S>();
    }
    template <int S>
    __device__ const SetT<PS, S> *win(int r, int i) const
    {
        const unsigned char *b = S == SET_G ? &gp[r][0] : &pop[r][S == SET_F ? 0 : (S == SET_H ? OFF_H : OFF_L)];
        return reinterpret_cast<const SetT<PS, S> *>(b) + i * win_elems<PS, S>();
    }
};

template <class PS, bool PB = true>
__host__ __device__ constexpr size_t strip_smem() { return sizeof(WarpRing<PS, PB>) * LB_SW; }

// Blocks (of LB_SW warps) resident per SM: as many as the rings of storage PS
// allow in the 228 KB of shared memory (1 KB reserved per block), at most 6.
template <class PS, bool PB = true>
__host__ __device__ constexpr int strip_min_blocks()
{
    return (int)((228 * 1024) / (strip_smem<PS, PB>() + 1024)) < 6 ? (int)((228 * 1024) / (strip_smem<PS, PB>() + 1024))
                                                                    : 6;
}

// Warps per block of the step kernel under storage PS.  Its warps claim work
// items independently, so the block shape only packs rings into shared memory.
// FP32 rings (24.3 KB a warp) fit nine warps per SM in blocks of three, but at
// the 168 registers the compiler then takes the step is 3 % slower than eight
// warps of two-warp blocks at 250 (measured at 4096^2).
#ifndef LB_STEP_SW32
#define LB_STEP_SW32 2
#endif
template <class PS>
__host__ __device__ constexpr int step_warps() { return PS::kHalf ? LB_SW : LB_STEP_SW32; }
template <class PS>
__host__ __device__ constexpr size_t step_smem() { return sizeof(WarpRing<PS>) * step_warps<PS>(); }
// Resident step blocks per SM: as many as shared memory allows, at most
// LB_STEP_MAXW warps.
#ifndef LB_STEP_MAXW
#define LB_STEP_MAXW 12
#endif
template <class PS>
__host__ __device__ constexpr int step_min_blocks()
{
    return (int)((228 * 1024) / (step_smem<PS>() + 1024)) < LB_STEP_MAXW / step_warps<PS>()
               ? (int)((228 * 1024) / (step_smem<PS>() + 1024))
               : LB_STEP_MAXW / step_warps<PS>();
}

__host__ __device__ inline int strip_groups(int nx) { return ((nx + LB_TX - 1) / LB_TX + LB_SW - 1) / LB_SW; }
__host__ __device__ inline int strip_segments(int ny, int segh) { return 2 + (ny >= 5 ? (ny - 4 + segh - 1) / segh : 0); }

// Rows [ys, ye) of segment s (empty when ys >= ye); inner segments of segh rows.
__device__ __forceinline__ void segment_rows(int ny, int segh, int s, int &ys, int &ye)
{
    if (s == 0) {
        ys = 0;
        ye = min(2, ny);
    } else if (s == 1) {
        ys = max(2, ny - 2);
        ye = ny;
    } else {
        ys = 2 + (s - 2) * segh;
        ye = min(ys + segh, ny - 2);
    }
}

__device__ __forceinline__ int mod3(int v) { return ((v % 3) + 3) % 3; }
__device__ __forceinline__ int mod5(int v) { return ((v % 5) + 5) % 5; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Decoded staged pulls of set S for the lane whose window index is idx.
template <class PS, int S, class RG>
__device__ __forceinline__ void load9(const Consts &K, const RG &w, int slot, int idx, real v[9])
{
    typedef SetT<PS, S> T;
    constexpr int E = win_elems<PS, S>();
    const T *p = w.template win<S>(slot, 0) + idx;
#pragma unroll
    for (int i = 0; i < 9; i++)
        v[i] = ((S == SET_F || S == SET_L) && i >= PS::QFL) ? R(0.0) : dec_pop<PS, S>(K, i, p[i * E - cx(i)]);
}

// The enthalpy wall rule on decoded pulls (W only).
template <bool W>
__device__ __forceinline__ void abb_fix9(const Consts &K, real v[9], int x, int y, real T_own)
{
    if (!W) return;
    v[1] = abb_fix<SET_H, 1, W>(K, v[1], x, y, T_own);
    v[2] = abb_fix<SET_H, 2, W>(K, v[2], x, y, T_own);
    v[3] = abb_fix<SET_H, 3, W>(K, v[3], x, y, T_own);
    v[4] = abb_fix<SET_H, 4, W>(K, v[4], x, y, T_own);
    v[5] = abb_fix<SET_H, 5, W>(K, v[5], x, y, T_own);
    v[6] = abb_fix<SET_H, 6, W>(K, v[6], x, y, T_own);
    v[7] = abb_fix<SET_H, 7, W>(K, v[7], x, y, T_own);
    v[8] = abb_fix<SET_H, 8, W>(K, v[8], x, y, T_own);
}

// Accessor of phase_b for the strip kernel.
template <class PS, bool W>
struct RingAcc {
    const WarpRing<PS> &w;
    int lane, off, off_h;              // window offsets of the staged planes: all but h, and h
    int sl[3], sq[3], sg[3], sp, sgp;  // rows y-1, y, y+1 in the mod-3, mod-4 and lag rings; pop / ax row, gp row
    // pairs read together (one 64-bit shared load each)
    __device__ float2 lagv(int dy, int dx) const { return w.lag[sg[dy + 1]][lane + 1 + dx]; }
    __device__ float2 ddv(int dy, int dx) const { return w.dd[sl[dy + 1]][lane + dx]; }
    __device__ float2 cfv(int dy, int dx) const { return w.cf[sl[dy + 1]][lane + dx]; }
    __device__ float2 psv(int dy, int dx) const { return w.ps[sq[dy + 1]][lane + dx]; }
    __device__ real phip(int dy, int dx) const { return lagv(dy, dx).x; }
    __device__ real Tp(int dy, int dx) const { return lagv(dy, dx).y; }
    __device__ real dphi(int dy, int dx) const { return ddv(dy, dx).x; }
    __device__ real dT(int dy, int dx) const { return ddv(dy, dx).y; }
    __device__ real C(int dy, int dx) const { return cfv(dy, dx).x; }
    __device__ real fs(int dy, int dx) const { return cfv(dy, dx).y; }
    __device__ real p(int dy, int dx) const { return psv(dy, dx).x; }
    __device__ real S(int dy, int dx) const { return psv(dy, dx).y; }
    __device__ real mdot(int dy, int dx) const { return w.md[sl[dy + 1]][lane + dx]; }
    __device__ real divu() const { return w.dv[sl[1]][lane]; }
    __device__ float2 lagu() const { return w.uv[sg[1]][lane + 1]; }  // own lagged (u_x, u_y)
    // pulled f, h (wall rule applied), l of the cell at (x, y)
    template <int S>
    __device__ void pops(const Consts &K, const float *__restrict__, int x, int y, long long, real v[9], real T_own) const
    {
        load9<PS, S>(K, w, sp, lane + (S == SET_H ? off_h : off), v);
        if (S == SET_H) abb_fix9<W>(K, v, x, y, T_own);
    }
    __device__ void gpops(const Consts &K, real v[9]) const
    {
        typedef SetT<PS, SET_G> T;
        constexpr int E = win_elems<PS, SET_G>();
        const T *p = w.template win<SET_G>(sgp, 0) + lane + off;
#pragma unroll
        for (int i = 0; i < 9; i++) v[i] = dec_val(p[i * E - cx(i)]);
    }
    __device__ real aux(int k) const { return w.ax[sp][k][lane + off]; }
};

// Stage the 9 pulls of set S at (x, y) one lane at a time into dst[i E - c_ix]
// (E the window slot size; raw stored values, decoded and given the wall rule
// when read).  FP32 values go by cp.async; half values are loaded and stored.
template <class PS, int S, bool W>
__device__ __forceinline__ void stage9(const Consts &K, const float *__restrict__ pin, int x, int y, int cell,
                                       SetT<PS, S> *dst)
{
    constexpr int E = win_elems<PS, S>();
    if constexpr (PS::esize(S) == 4) {
        cp_async4(dst + 0 * E - cx(0), pull_src<PS, S, 0, W>(K, pin, x, y, cell));
        cp_async4(dst + 1 * E - cx(1), pull_src<PS, S, 1, W>(K, pin, x, y, cell));
        cp_async4(dst + 2 * E - cx(2), pull_src<PS, S, 2, W>(K, pin, x, y, cell));
        cp_async4(dst + 3 * E - cx(3), pull_src<PS, S, 3, W>(K, pin, x, y, cell));
        cp_async4(dst + 4 * E - cx(4), pull_src<PS, S, 4, W>(K, pin, x, y, cell));
        if ((S != SET_F && S != SET_L) || PS::QFL == 9) {  // D2Q5 f and l: directions 0 .. 4 only
            cp_async4(dst + 5 * E - cx(5), pull_src<PS, S, 5, W>(K, pin, x, y, cell));
            cp_async4(dst + 6 * E - cx(6), pull_src<PS, S, 6, W>(K, pin, x, y, cell));
            cp_async4(dst + 7 * E - cx(7), pull_src<PS, S, 7, W>(K, pin, x, y, cell));
            cp_async4(dst + 8 * E - cx(8), pull_src<PS, S, 8, W>(K, pin, x, y, cell));
        }
    } else {
        dst[0 * E - cx(0)] = __ldg(pull_src<PS, S, 0, W>(K, pin, x, y, cell));
        dst[1 * E - cx(1)] = __ldg(pull_src<PS, S, 1, W>(K, pin, x, y, cell));
        dst[2 * E - cx(2)] = __ldg(pull_src<PS, S, 2, W>(K, pin, x, y, cell));
        dst[3 * E - cx(3)] = __ldg(pull_src<PS, S, 3, W>(K, pin, x, y, cell));
        dst[4 * E - cx(4)] = __ldg(pull_src<PS, S, 4, W>(K, pin, x, y, cell));
        dst[5 * E - cx(5)] = __ldg(pull_src<PS, S, 5, W>(K, pin, x, y, cell));
        dst[6 * E - cx(6)] = __ldg(pull_src<PS, S, 6, W>(K, pin, x, y, cell));
        dst[7 * E - cx(7)] = __ldg(pull_src<PS, S, 7, W>(K, pin, x, y, cell));
        dst[8 * E - cx(8)] = __ldg(pull_src<PS, S, 8, W>(K, pin, x, y, cell));
    }
}

// Lagged phi and T of the cell that wrote the population pulled into direction
// I at row y, lane column: from the lag ring (own cell at a wall).
template <int I, bool W, class RG>
__device__ __forceinline__ void lag_src(const Consts &K, const RG &w, int lane, int y, const int lr[3], real &ph, real &tt)
{
    constexpr int ys_off = -cy(I);
    const int ys = y + ys_off;
    const float2 v = (W && ys_off != 0 && (ys < 0 || ys >= K.ny)) ? w.lag[lr[1]][lane + 1] : w.lag[lr[ys_off + 1]][lane + 1 - cx(I)];
    ph = v.x;
    tt = v.y;
}

// lr: lag-ring rows of rows y - 1, y and y + 1.
template <bool W, int QF, class RG>
__device__ __forceinline__ void lag_dev_sums(const Consts &K, const RG &w, int lane, int y, const int lr[3], real phi_own,
                                             real T_own, real &dph, real &dtt)
{
    real ph[9], tt[9];
    lag_src<1, W>(K, w, lane, y, lr, ph[1], tt[1]);
    lag_src<2, W>(K, w, lane, y, lr, ph[2], tt[2]);
    lag_src<3, W>(K, w, lane, y, lr, ph[3], tt[3]);
    lag_src<4, W>(K, w, lane, y, lr, ph[4], tt[4]);
    lag_src<5, W>(K, w, lane, y, lr, ph[5], tt[5]);
    lag_src<6, W>(K, w, lane, y, lr, ph[6], tt[6]);
    lag_src<7, W>(K, w, lane, y, lr, ph[7], tt[7]);
    lag_src<8, W>(K, w, lane, y, lr, ph[8], tt[8]);
    if (QF == 9)
        dph = (wgt(1) * (ph[1] - phi_own) + wgt(2) * (ph[2] - phi_own) + wgt(3) * (ph[3] - phi_own) +
               wgt(4) * (ph[4] - phi_own)) +
              (wgt(5) * (ph[5] - phi_own) + wgt(6) * (ph[6] - phi_own) + wgt(7) * (ph[7] - phi_own) +
               wgt(8) * (ph[8] - phi_own));
    else
        dph = wfl<5>(1) * (((ph[1] - phi_own) + (ph[2] - phi_own)) + ((ph[3] - phi_own) + (ph[4] - phi_own)));
    dtt = (wgt(1) * (tt[1] - T_own) + wgt(2) * (tt[2] - T_own) + wgt(3) * (tt[3] - T_own) + wgt(4) * (tt[4] - T_own)) +
          (wgt(5) * (tt[5] - T_own) + wgt(6) * (tt[6] - T_own) + wgt(7) * (tt[7] - T_own) + wgt(8) * (tt[8] - T_own));
}

// Isotropic divergence of the lagged velocity at row y, lane column, from the
// uv ring (columns x0 - 2 .. x0 + 31 at index lane + 1 + dx; lr the ring rows
// of rows y - 1, y and y + 1, those of the lag ring); a row beyond a wall is
// the ghost -u of row y.  Same stencil and order as lagged_divu.
template <bool W, class RG>
__device__ __forceinline__ real ring_divu(const Consts &K, const RG &w, int lane, int y, const int lr[3])
{
    const int c = lane + 1;
    const bool gs = W && y - 1 < 0, gn = W && y + 1 >= K.ny;
    const float2 *r0 = w.uv[lr[1]];
    const float2 *rs = gs ? r0 : w.uv[lr[0]];
    const float2 *rn = gn ? r0 : w.uv[lr[2]];
    const real ss = gs ? R(-1.0) : R(1.0), sn = gn ? R(-1.0) : R(1.0);
    const real dudx = wgt(1) * (r0[c + 1].x - r0[c - 1].x) +
                      wgt(5) * ((sn * rn[c + 1].x - sn * rn[c - 1].x) + (ss * rs[c + 1].x - ss * rs[c - 1].x));
    const real dvdy = wgt(2) * (sn * rn[c].y - ss * rs[c].y) +
                      wgt(5) * ((sn * rn[c + 1].y - ss * rs[c + 1].y) + (sn * rn[c - 1].y - ss * rs[c - 1].y));
    return R(3.0) * (dudx + dvdy);
}

// Phase A / phase B sweep of one warp over rows [ys, ye) of its strip.  WALLS =
// false: every row ys - 2 .. ye + 1 lies inside the lattice.
template <int MODE, bool WALLS, class PS>
__device__ __forceinline__ void strip_rows(const Consts &K, const Buffers &B, WarpRing<PS, MODE != MODE_REDUCE> &w, int lane,
                                           int x0, int ys, int ye,
                                           double acc[NRED])
{
    typedef SetT<PS, SET_F> TF;  // f and l
    typedef SetT<PS, SET_G> TG;
    typedef SetT<PS, SET_H> TH;
    constexpr bool PB = MODE != MODE_REDUCE;  // phase B follows phase A
    constexpr bool HALF = PS::kHalf;          // f, g and l in half precision
    constexpr bool HMIX = HALF && PS::esize(SET_H) == 4;  // ... and h in FP32
    constexpr int EF = win_elems<PS, SET_F>();  // window slot size in elements of f / l, g
    constexpr int EG = win_elems<PS, SET_G>();
    constexpr int CH = HALF ? 8 : 4;          // elements of a 16-byte chunk of f, g and l
    constexpr int PLEN = HALF ? 48 : 40;      // staged columns of a population window
    const int ex = x0 - 1 + lane;
    const int xg = ((ex % K.nx) + K.nx) % K.nx;
    const bool b_lane = lane >= 1 && lane <= LB_TX && ex < K.nx;
    const float *__restrict__ pin = B.pin;
    const float *__restrict__ ain = B.ain;
    const int xa = (((x0 - 2 + lane) % K.nx) + K.nx) % K.nx;
    const int xb = (((x0 + 30 + (lane & 1)) % K.nx) + K.nx) % K.nx;
    // Staging form.  Inner segments of strips whose windows (from the 16-byte
    // boundary x_lo <= x0 - 2) lie inside the lattice row copy whole windows in
    // 16-byte chunks, a group of lanes per window; the wall bands and the strips
    // at the x ends copy one value per lane (pull rules, periodic wrap) into the
    // same layout.
    const int x_lo = (x0 - 2) & ~(CH - 1);           // windows of f, g, l and the lagged planes
    const int x_lo_h = HMIX ? ((x0 - 2) & ~3) : x_lo;  // windows of h
    const bool win = !WALLS && x0 >= 2 && x_lo + PLEN <= K.nx && x_lo + WW <= K.nx && x_lo_h + WW <= K.nx;
    const int off = win ? x0 - 1 - x_lo : 4;
    const int off_h = win ? x0 - 1 - x_lo_h : 4;
    const int wg = lane / 10, wpart = lane - 10 * wg;  // float windows: 10 chunks, 3 windows per copy
    const int wcol = x_lo + 4 * wpart;
    const int hg = lane / 6, hpart = lane - 6 * hg;    // half windows: 6 chunks, 5 windows per copy

    // lagged (phi, T) of row yl into lag-ring row lr (= yl mod 5)
    auto stage_lag = [&](int yl, int lr) {
        if (WALLS && (yl < 0 || yl >= K.ny)) return;
        const int ro = yl * K.pitch;
        cp_async4(&w.lag[lr][lane].x, plane_ptr(ain, AUX_PHI, K) + (ro + xa));
        cp_async4(&w.lag[lr][lane].y, plane_ptr(ain, AUX_T, K) + (ro + xa));
        if (lane < 2) {
            cp_async4(&w.lag[lr][32 + lane].x, plane_ptr(ain, AUX_PHI, K) + (ro + xb));
            cp_async4(&w.lag[lr][32 + lane].y, plane_ptr(ain, AUX_T, K) + (ro + xb));
        }
    };
    // lagged (u_x, u_y) of row yl with the one-column halo: the own-cell velocity of
    // phase B, and the divergence of phase A (div u the lagged velocity divergence)
    auto stage_u = [&](int yl, int lr) {  // into uv-ring row lr (= yl mod 5)
        if ((!PB && !K.divu) || (WALLS && (yl < 0 || yl >= K.ny))) return;
        const int ro = yl * K.pitch;
        cp_async4(&w.uv[lr][lane].x, plane_ptr(ain, AUX_UX, K) + (ro + xa));
        cp_async4(&w.uv[lr][lane].y, plane_ptr(ain, AUX_UY, K) + (ro + xa));
        if (lane < 2) {
            cp_async4(&w.uv[lr][32 + lane].x, plane_ptr(ain, AUX_UX, K) + (ro + xb));
            cp_async4(&w.uv[lr][32 + lane].y, plane_ptr(ain, AUX_UY, K) + (ro + xb));
        }
    };
    // own-cell lagged values of row y as float windows: Q, f_s and (phase B) C, one copy
    auto stage_ax_win = [&](int y, int s3) {
        if (wg < 3 && (PB || wg < 2))
            cp_async16(&w.ax[s3][wg][4 * wpart],
                       plane_ptr(ain, wg == 0 ? AUX_Q : (wg == 1 ? AUX_FS : AUX_C), K) + (y * K.pitch + wcol));
    };
    // phase-A inputs of row y, and the own-cell lagged values phase B needs
    auto stage_a = [&](int y, int s3) {  // s3 = y mod 3
        if (WALLS && (y < 0 || y >= K.ny)) return;
        const int cell = y * K.pitch + xg;
        if (win) {
            if constexpr (!HALF) {
                if (wg < 3) {
                    // group wg: set f, h or l; one window per direction, rows y - c_iy
                    const float *src = (wg == 0 ? set_plane<PS, SET_F>(pin, 0, K)
                                                : (wg == 1 ? set_plane<PS, SET_H>(pin, 0, K) : set_plane<PS, SET_L>(pin, 0, K))) +
                                       wcol;
                    float *dst = (wg == 0 ? w.template win<SET_F>(s3, 0)
                                          : (wg == 1 ? w.template win<SET_H>(s3, 0) : w.template win<SET_L>(s3, 0))) +
                                 4 * wpart;
                    const int nq = wg == 1 ? 9 : PS::QFL;  // D2Q5 f and l: directions 0 .. 4
#pragma unroll
                    for (int i = 0; i < 9; i++)
                        if (i < nq) cp_async16(dst + i * EF, plane_ptr(src, i, K) + (y - cy(i)) * K.pitch);
                }
            } else {
                // half windows: f and l (and h unless it is FP32), six 16-byte chunks each
                constexpr int NHW = HMIX ? 18 : 27;
                if (hg < 5) {
#pragma unroll
                    for (int q = 0; q < (NHW + 4) / 5; q++) {
                        const int wi = 5 * q + hg;
                        if (wi < NHW) {
                            // HMIX: f 0..8, l 9..17; else f 0..8, h 9..17, l 18..26
                            const int grp = wi >= 9 ? (wi >= 18 ? 2 : 1) : 0;
                            const int set = HMIX ? (grp == 0 ? SET_F : SET_L) : (grp == 0 ? SET_F : (grp == 1 ? SET_H : SET_L));
                            const int i = wi - 9 * grp;
                            __half *dst = set == SET_F ? w.template win<SET_F>(s3, i)
                                                       : (set == SET_H ? reinterpret_cast<__half *>(w.template win<SET_H>(s3, i))
                                                                       : w.template win<SET_L>(s3, i));
                            const int before = set == SET_F ? set_bytes_before<PS>(SET_F)
                                                             : (set == SET_H ? set_bytes_before<PS>(SET_H)
                                                                             : set_bytes_before<PS>(SET_L));
                            const __half *src = reinterpret_cast<const __half *>(
                                                    reinterpret_cast<const char *>(pin) +
                                                    (size_t)(unsigned)K.plane * (unsigned)(before + 2 * i)) +
                                                ((y - cy_rt(i)) * K.pitch + x_lo + CH * hpart);
                            cp_async16(dst + CH * hpart, src);
                        }
                    }
                }
                if constexpr (HMIX) {
                    // FP32 windows of h: ten 16-byte chunks each, three windows per copy
                    if (wg < 3) {
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            const int i = 3 * q + wg;
                            const int cyi = wg == 0 ? cy(3 * q) : (wg == 1 ? cy(3 * q + 1) : cy(3 * q + 2));
                            cp_async16(reinterpret_cast<float *>(w.template win<SET_H>(s3, i)) + 4 * wpart,
                                       set_plane<PS, SET_H>(pin, i, K) + ((y - cyi) * K.pitch + x_lo_h + 4 * wpart));
                        }
                    }
                }
            }
            stage_ax_win(y, s3);
        } else {
            stage9<PS, SET_F, WALLS>(K, pin, xg, y, cell, w.template win<SET_F>(s3, 0) + lane + off);
            stage9<PS, SET_H, WALLS>(K, pin, xg, y, cell, w.template win<SET_H>(s3, 0) + lane + off_h);
            stage9<PS, SET_L, WALLS>(K, pin, xg, y, cell, w.template win<SET_L>(s3, 0) + lane + off);
            float *pa = &w.ax[s3][0][lane + off];
            cp_async4(pa + AX_Q * WW, plane_ptr(ain, AUX_Q, K) + cell);
            cp_async4(pa + AX_FS * WW, plane_ptr(ain, AUX_FS, K) + cell);
            if (PB) cp_async4(pa + AX_C * WW, plane_ptr(ain, AUX_C, K) + cell);
        }
        if (PB) {
            cp_async4(&w.ps[y & 3][lane].x, plane_ptr(ain, AUX_P, K) + cell);
            cp_async4(&w.ps[y & 3][lane].y, plane_ptr(ain, AUX_S, K) + cell);
        }
    };
    // pulled g of row y, for its phase B one iteration later
    auto stage_g = [&](int y) {
        if (!PB || y < ys || y >= ye) return;
        if (win) {
            if constexpr (!HALF) {
                if (wg < 3) {
                    const float *src = set_plane<PS, SET_G>(pin, 0, K) + wcol;
                    float *gw = reinterpret_cast<float *>(w.template win<SET_G>(y & 1, 0));
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        const int i = 3 * q + wg;  // direction of this group's window
                        const int cyi = wg == 0 ? cy(3 * q) : (wg == 1 ? cy(3 * q + 1) : cy(3 * q + 2));
                        cp_async16(gw + i * EG + 4 * wpart, plane_ptr(src, i, K) + (y - cyi) * K.pitch);
                    }
                }
            } else {
                if (hg < 5) {
                    __half *gw = reinterpret_cast<__half *>(w.template win<SET_G>(y & 1, 0));
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const int i = 5 * q + hg;
                        if (i < 9)
                            cp_async16(gw + i * EG + CH * hpart,
                                       reinterpret_cast<const __half *>(set_plane<PS, SET_G>(pin, i, K)) +
                                           ((y - cy_rt(i)) * K.pitch + x_lo + CH * hpart));
                    }
                }
            }
        } else if (b_lane) {
            stage9<PS, SET_G, WALLS>(K, pin, ex, y, y * K.pitch + ex,
                                     w.template win<SET_G>(y & 1, 0) + lane + off);
        }
    };

    CompSum csum[7];  // MODE_REDUCE: this segment's diagnostics addends (diag_terms)
    const int ya0 = PB ? ys - 1 : ys;
    const int ya1 = PB ? ye : ye - 1;
    int s3 = mod3(ya0), l5 = mod5(ya0);  // ya mod 3 and ya mod 5, advanced with the loop
    auto lrow = [&](int k) {             // lag- and uv-ring row of row ya + k, k in -2 .. 3
        const int v = l5 + k;
        return v >= 5 ? v - 5 : (v < 0 ? v + 5 : v);
    };
    // Rows of copies in flight: one with phase B, whose rings hold row ya - 1 for
    // it; two for phase A alone (the diagnostics), in the ring rows phase B
    // would hold.
    constexpr int AHEAD = PB ? 1 : 2;
    stage_lag(ya0 - 1, lrow(-1));
    stage_lag(ya0, lrow(0));
    stage_lag(ya0 + 1, lrow(1));
    stage_u(ya0 - 1, lrow(-1));
    stage_u(ya0, lrow(0));
    stage_u(ya0 + 1, lrow(1));
    stage_a(ya0, s3);
    cp_async_commit();
    if constexpr (AHEAD == 2) {
        if (ya0 < ya1) {
            stage_lag(ya0 + 2, lrow(2));
            stage_u(ya0 + 2, lrow(2));
            stage_a(ya0 + 1, s3 == 2 ? 0 : s3 + 1);
        }
        cp_async_commit();
    }
    for (int ya = ya0; ya <= ya1; ya++, s3 = s3 == 2 ? 0 : s3 + 1, l5 = l5 == 4 ? 0 : l5 + 1) {
        const int s3n = s3 == 2 ? 0 : s3 + 1, s3p = s3 == 0 ? 2 : s3 - 1;  // (ya + 1), (ya - 1) mod 3
        if (ya + AHEAD <= ya1) {
            stage_lag(ya + 1 + AHEAD, lrow(1 + AHEAD));
            stage_u(ya + 1 + AHEAD, lrow(1 + AHEAD));
            stage_a(ya + AHEAD, AHEAD == 1 ? s3n : s3p);  // (ya + 2) mod 3 = (ya - 1) mod 3
        }
        stage_g(ya);
        cp_async_commit();
        cp_async_wait<AHEAD>();  // everything staged for row ya (and g of row ya - 1) has landed
        __syncwarp();
        // ---- phase A, row ya ------------------------------------------------------------
        if (!WALLS || (ya >= 0 && ya < K.ny)) {
            const int lr[3] = {lrow(-1), lrow(0), lrow(1)};
            const float2 lag0 = w.lag[lr[1]][lane + 1];
            const real phi_p = lag0.x, T_p = lag0.y;
            real dph, dtt, v[9];
            lag_dev_sums<WALLS, PS::QFL>(K, w, lane, ya, lr, phi_p, T_p, dph, dtt);
            load9<PS, SET_F>(K, w, s3, lane + off, v);
            const real delta = sum9(v) + dph;
            load9<PS, SET_H>(K, w, s3, lane + off_h, v);
            abb_fix9<WALLS>(K, v, xg, ya, T_p);
            const real Q_p = w.ax[s3][AX_Q][lane + off];
            const real ed = sum9(v) + K.rr * dtt + R(0.5) * Q_p;
            load9<PS, SET_L>(K, w, s3, lane + off, v);
            const real sl = sum9(v);
            const real fs_p = w.ax[s3][AX_FS][lane + off];
            const real chi_p = clamp01(R(0.5) * (R(1.0) + phi_p));
            const real dv = K.divu ? ring_divu<WALLS>(K, w, lane, ya, lr) : R(0.0);
            const Local L = local_fields(K, phi_p, delta, ed, T_p, chi_p, fs_p, sl, dv);
            if (MODE == MODE_REDUCE) {
                if (b_lane) {
                    const DiagTerms d = diag_terms(K, phi_p, L.dphi, ed, T_p, chi_p, fs_p, L.C, L.fs);
#pragma unroll
                    for (int q = 0; q < 7; q++) csum[q].add(d.t[q]);
                    if (ex == K.nx / 2) acc[5] += (double)L.fs;
                }
            } else {
                w.dd[s3][lane] = make_float2(L.dphi, L.dT);
                w.cf[s3][lane] = make_float2(L.C, L.fs);
                w.md[s3][lane] = L.mdot;
                w.dv[s3][lane] = L.divu;
            }
        }
        __syncwarp();
        // ---- phase B, row ya - 1 ----------------------------------------------------------
        if constexpr (PB) {
            const int yb = ya - 1;
            if (yb >= ys && yb < ye && b_lane) {
                // rows yb - 1 = ya - 2, yb = ya - 1 and yb + 1 = ya are s3n, s3p and s3 mod 3
                const RingAcc<PS, WALLS> A{w, lane, off, off_h, {s3n, s3p, s3}, {(yb - 1) & 3, yb & 3, (yb + 1) & 3},
                                           {lrow(-2), lrow(-1), lrow(0)}, s3p, yb & 1};
                phase_b<MODE, WALLS, PS>(K, B, A, ex, yb, yb * K.pitch + ex);
            }
        }
        __syncwarp();
    }
    cp_async_wait<0>();
    __syncwarp();
    if constexpr (MODE == MODE_REDUCE) {
        acc[0] += csum[0].value() + csum[1].value();
        acc[1] += csum[2].value() + csum[3].value();
        acc[2] += csum[4].value();
        acc[3] += csum[5].value();
        acc[4] += csum[6].value();
    }
}

#ifdef LB_MAXNREG
#define LB_STRIP_BOUNDS __maxnreg__(LB_MAXNREG)
#else
#define LB_STRIP_BOUNDS __launch_bounds__(32 * LB_SW, (strip_min_blocks<PS, MODE != MODE_REDUCE>()))
#endif

template <int MODE, class PS>
__global__ void LB_STRIP_BOUNDS lb_strip_kernel(const Consts K, const Buffers B, double *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char lb_smem[];
    typedef WarpRing<PS, MODE != MODE_REDUCE> Ring;
    Ring &w = reinterpret_cast<Ring *>(lb_smem)[threadIdx.y];
    const int lane = threadIdx.x;
    const int ngroups = strip_groups(K.nx);
    const int nblocks = ngroups * strip_segments(K.ny, K.segh);
    double acc[NRED] = {0, 0, 0, 0, 0, 0};
    // a block may own several (group, segment) pairs when the grid is capped
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int group = b % ngroups, seg = b / ngroups;
        const int x0 = (group * LB_SW + (int)threadIdx.y) * LB_TX;
        int ys, ye;
        segment_rows(K.ny, K.segh, seg, ys, ye);
        if ((seg == 0 && K.ghost_lo) || (seg == 1 && K.ghost_hi)) continue;  // ghost rows of a slab
        if (x0 >= K.nx || ys >= ye) continue;  // the whole warp: warps never synchronise with one another
        if (seg < 2)
            strip_rows<MODE, true, PS>(K, B, w, lane, x0, ys, ye, acc);
        else
            strip_rows<MODE, false, PS>(K, B, w, lane, x0, ys, ye, acc);
        __syncwarp();
    }
    if (MODE == MODE_REDUCE) {
        // one partial per warp, in a fixed place: the final pass adds them in order
#pragma unroll
        for (int q = 0; q < NRED; q++) {
            const double s = warp_sum(acc[q]);
            if (lane == 0) partials[((long long)blockIdx.x * LB_SW + threadIdx.y) * NRED + q] = s;
        }
    }
}

// ---------------------------------------------------------------------------------------
// The step: one persistent launch advances one lattice or a batch of many
// independent lattices (instances) by one time step.  The work items are
// (instance, warp strip, row segment), numbered instance by instance from
// item0; warps claim them from an atomic counter, so uneven instance sizes
// balance dynamically.  counter[0] counts claimed items and counter[1] the
// warps that found the list empty; the last of those resets both, so every
// launch starts from zero without a separate reset.  The constants of an instance are
// read from its read-only record in global memory (cached; no shared-memory
// aliasing with the rings to hold the compiler back).  Each item computes
// exactly what the single-lattice launch computes for that strip and segment,
// so the result does not depend on which warp takes which item.
// ---------------------------------------------------------------------------------------
struct StepRec {
    Consts K;
    Buffers B[2];     // [0]: first buffer -> second, [1]: the reverse
    int nstrip;       // warp strips of the instance
    long long item0;  // first work item of the instance
};


template <class PS>
__global__ void __launch_bounds__(32 * step_warps<PS>(), step_min_blocks<PS>()) lb_step_kernel(const StepRec *__restrict__ inst, int ninst, long long nitems,
                                                int parity, unsigned long long *__restrict__ counter)
{
    const unsigned long long nwarps = (unsigned long long)gridDim.x * blockDim.y;
    extern __shared__ __align__(16) unsigned char lb_smem[];
    WarpRing<PS> &w = reinterpret_cast<WarpRing<PS> *>(lb_smem)[threadIdx.y];
    const int lane = threadIdx.x;
    double acc[NRED];  // unused in MODE_STEP
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= (unsigned long long)nitems) {
            if (lane == 0 && atomicAdd(counter + 1, 1ULL) == nwarps - 1) {
                counter[0] = 0;  // every warp is done claiming: ready for the next launch
                counter[1] = 0;
            }
            break;
        }
        int lo = 0, hi = ninst - 1;  // last instance with item0 <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst[mid].item0 <= (long long)item)
                lo = mid;
            else
                hi = mid - 1;
        }
        const Consts K = inst[lo].K;  // by value: the fields the sweep uses stay in registers
        const Buffers B = inst[lo].B[parity];
        const long long local = (long long)item - inst[lo].item0;
        const int nstrip = inst[lo].nstrip;
        const int strip = (int)(local % nstrip), seg = (int)(local / nstrip);
        int ys, ye;
        segment_rows(K.ny, K.segh, seg, ys, ye);
        if (ys >= ye || (seg == 0 && K.ghost_lo) || (seg == 1 && K.ghost_hi)) continue;
        if (seg < 2)
            strip_rows<MODE_STEP, true, PS>(K, B, w, lane, strip * LB_TX, ys, ye, acc);
        else
            strip_rows<MODE_STEP, false, PS>(K, B, w, lane, strip * LB_TX, ys, ye, acc);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------
// Initialisation: equilibria of the initial fields (p = 0), written in natural
// (post-streaming) layout to `eq`, h as deviations from w_i rr T (with the
// latent reference for i = 0), and the lagged fields of a state at rest in time.
// ---------------------------------------------------------------------------------------
// Velocity component v (dense nx * ny input) at (x + dx, y + dy), with the
// ghost -u of row y beyond a no-slip wall.
__device__ __forceinline__ real dense_u_nb(const Consts &K, const float *__restrict__ v, int x, int y, int dx, int dy)
{
    const int yy = y + dy, xx = wrapx(x + dx, K.nx);
    if (yy < 0 || yy >= K.ny) return -v[(long long)y * K.nx + xx];
    return v[(long long)yy * K.nx + xx];
}

// match_moment (re-initialisation from fields): when div u is the lagged
// velocity divergence, the next step reads phi = sum f / (1 - div u / 2) with
// div u the divergence of the installed velocity; the rest population is then
// lowered by phi div u / 2 so that this reading returns the given phi.
__global__ void lb_init_eq_kernel(const Consts K, const float *__restrict__ phi0, const float *__restrict__ T0,
                                  const float *__restrict__ C0, const float *__restrict__ ux0,
                                  const float *__restrict__ uy0, const float *__restrict__ fs0,
                                  const float *__restrict__ p0, float *__restrict__ eq, float *__restrict__ aux,
                                  int match_moment)
{
    const long long n = (long long)K.nx * K.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / K.nx), x = (int)(k % K.nx);
        const long long cell = (long long)y * K.pitch + x;
        const real phi = phi0[k], T = T0[k], C = C0[k];
        const real ux = ux0 ? ux0[k] : R(0.0), uy = uy0 ? uy0[k] : R(0.0);
        real f0_shift = R(0.0);
        if (match_moment && K.divu && ux0 && uy0) {
            const real dudx = wgt(1) * (dense_u_nb(K, ux0, x, y, 1, 0) - dense_u_nb(K, ux0, x, y, -1, 0)) +
                              wgt(5) * ((dense_u_nb(K, ux0, x, y, 1, 1) - dense_u_nb(K, ux0, x, y, -1, 1)) +
                                        (dense_u_nb(K, ux0, x, y, 1, -1) - dense_u_nb(K, ux0, x, y, -1, -1)));
            const real dvdy = wgt(2) * (dense_u_nb(K, uy0, x, y, 0, 1) - dense_u_nb(K, uy0, x, y, 0, -1)) +
                              wgt(5) * ((dense_u_nb(K, uy0, x, y, 1, 1) - dense_u_nb(K, uy0, x, y, 1, -1)) +
                                        (dense_u_nb(K, uy0, x, y, -1, 1) - dense_u_nb(K, uy0, x, y, -1, -1)));
            f0_shift = -R(0.5) * phi * R(3.0) * (dudx + dvdy);
        }
        const real chi = clamp01(R(0.5) * (R(1.0) + phi));
        real fs;
        real e_sens;
        if (fs0) {
            // given solid fraction (clamped to [0, chi]): sensible enthalpy by the
            // mixture rule of the volumetric heat capacities
            fs = K.phase_change ? fminf(fmaxf(fs0[k], R(0.0)), chi) : R(0.0);
            e_sens = T * (fs * K.rcp_s + (chi - fs) * K.rcp_l + (R(1.0) - chi) * K.rcp_g);
        } else {
            e_sens = forward_sensible(K, T, chi, fs);
        }
        const real rho = zeta(phi, fs, K.rho_l, K.rho_s, K.rho_g);
        const real rhocp = zeta(phi, fs, K.rcp_l, K.rcp_s, K.rcp_g);
        const real uu = ux * ux + uy * uy;
        const real rcT = rhocp * T;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const real cu = (real)cx(i) * ux + (real)cy(i) * uy;
            const real si = wgt(i) * (R(3.0) * cu + R(4.5) * cu * cu - R(1.5) * uu);
            eq[(long long)(SET_F * 9 + i) * K.plane + cell] =
                wfl_rt(K.qfl, i) * phi * (R(1.0) + R(3.0) * cu) + (i == 0 ? f0_shift : R(0.0));
            eq[(long long)(SET_G * 9 + i) * K.plane + cell] = rho * si;
            eq[(long long)(SET_L * 9 + i) * K.plane + cell] = wfl_rt(K.qfl, i) * C * (R(1.0) + R(3.0) * cu);
            // h_0 - w_0 rr T - latent = e_sens - rr T - w_0 rho Cp T 3u.u/2;  h_i - w_i rr T = w_i rho Cp T (...)
            eq[(long long)(SET_H * 9 + i) * K.plane + cell] =
                i == 0 ? e_sens - K.rr * T - wgt(0) * rcT * R(1.5) * uu
                       : wgt(i) * rcT * (R(3.0) * cu + R(4.5) * cu * cu - R(1.5) * uu);
        }
        aux[AUX_FS * K.plane + cell] = fs;
        aux[AUX_Q * K.plane + cell] = 0.0f;
        aux[AUX_UX * K.plane + cell] = ux;
        aux[AUX_UY * K.plane + cell] = uy;
        aux[AUX_PHI * K.plane + cell] = phi;
        aux[AUX_C * K.plane + cell] = C;
        aux[AUX_P * K.plane + cell] = p0 ? p0[k] : 0.0f;
        aux[AUX_S * K.plane + cell] = 0.0f;
        aux[AUX_T * K.plane + cell] = T;
    }
}

// Inverse streaming: the stored state is post-collision, so the initial
// post-streaming populations `eq` are placed where the next pull finds them,
// f, g and h as deviations from the references of the cell that holds them.
template <class PS, int S>
__device__ __forceinline__ void unstream_set(const Consts &K, const float *__restrict__ eq,
                                             const float *__restrict__ aux, float *__restrict__ pops, int x, int y,
                                             long long cell, real phi_here, real T_here)
{
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const int yt = y + cy(i);
        real v;
        if (yt < 0 || yt >= K.ny) {
            v = eq[(long long)(S * 9 + opp(i)) * K.plane + cell];
            if (S == SET_H) {
                const bool bottom = yt < 0;
                if ((bottom ? K.bc_bottom : K.bc_top) == WALL_DIRICHLET) {
                    // stored h_i(x) = 2 w rr T_w - h_eq_opp(x), as a deviation from w rr T(x)
                    real Tw = bottom ? wall_T_bottom(K, (real)x) : K.T_top;
                    v = R(2.0) * wgt(i) * K.rr * (Tw - T_here) - v;
                }
            }
        } else {
            const int xt = wrapx(x + cx(i), K.nx);
            const long long ct = (long long)yt * K.pitch + xt;
            v = eq[(long long)(S * 9 + i) * K.plane + ct];
            if (S == SET_H && i != 0) v += wgt(i) * K.rr * ((real)aux[AUX_T * K.plane + ct] - T_here);
            if (S == SET_G && i != 0)
                v += R(3.0) * wgt(i) * ((real)aux[AUX_P * K.plane + ct] - (real)aux[AUX_P * K.plane + cell]);
        }
        if (S == SET_F) v -= wfl_rt(K.qfl, i) * phi_here;
        set_plane<PS, S>(pops, i, K)[cell] = enc_pop<PS, S>(K, i, v);
    }
}

template <class PS>
__global__ void lb_init_unstream_kernel(const Consts K, const float *__restrict__ eq, const float *__restrict__ aux,
                                        float *__restrict__ pops)
{
    const long long n = (long long)K.nx * K.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / K.nx), x = (int)(k % K.nx);
        const long long cell = (long long)y * K.pitch + x;
        const real phi_here = aux[AUX_PHI * K.plane + cell];
        const real T_here = aux[AUX_T * K.plane + cell];
        unstream_set<PS, SET_F>(K, eq, aux, pops, x, y, cell, phi_here, T_here);
        unstream_set<PS, SET_G>(K, eq, aux, pops, x, y, cell, phi_here, T_here);
        unstream_set<PS, SET_H>(K, eq, aux, pops, x, y, cell, phi_here, T_here);
        unstream_set<PS, SET_L>(K, eq, aux, pops, x, y, cell, phi_here, T_here);
    }
}

// ---------------------------------------------------------------------------------------
// Diagnostics, final pass: adds the per-warp partials of MODE_REDUCE in a fixed order.
// ---------------------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) lb_reduce_final_kernel(const double *__restrict__ partials, int nblocks,
                                                                       double *__restrict__ out)
{
    __shared__ double sh[RED_THREADS / 32][NRED];
    double acc[NRED] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < NRED; q++) acc[q] += partials[(long long)b * NRED + q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NRED; q++) {
        double s = warp_sum(acc[q]);
        if (lane == 0) sh[w][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < NRED) {
        double s = 0.0;
        for (int j = 0; j < RED_THREADS / 32; j++) s += sh[j][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------------------
// Halo messages of a slab (y-slab decomposition).  A message holds, for every
// population plane (in its storage type) and then every lagged plane (FP32),
// two lattice rows of nx values: rows [r0, r0 + 2) of the buffer, plane after
// plane, rows consecutive.  pack copies them out of the state (populations
// then lagged planes), unpack writes them into it.
// ---------------------------------------------------------------------------------------
template <class PS>
__device__ __forceinline__ void halo_plane(int k, int &esz, long long &byte_off, const Consts &K)
{
    // population plane k = 9 s + i: element bytes and byte offset in the buffer
    const int s = k / 9, i = k - 9 * s;
    esz = PS::esize(s);
    const int before = s == 0 ? 0 : (s == 1 ? set_bytes_before<PS>(1) : (s == 2 ? set_bytes_before<PS>(2)
                                                                                : set_bytes_before<PS>(3)));
    byte_off = (long long)K.plane * (before + esz * i);
}

// bytes of one halo message: 36 population planes and NAUX lagged planes, 2 rows of nx
template <class PS>
__host__ __device__ constexpr long long halo_message_bytes(int nx)
{
    return 2LL * nx * (pop_cell_bytes<PS>() + 4 * NAUX);
}

template <class PS, bool PACK>
__global__ void lb_halo_kernel(const Consts K, unsigned char *__restrict__ pops, float *__restrict__ aux, int r0,
                               unsigned char *__restrict__ msg)
{
    const long long per_plane = 2LL * K.nx;
    const long long total = per_plane * (36 + NAUX);
    const long long pop_bytes = per_plane * pop_cell_bytes<PS>();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int plane = (int)(k / per_plane);
        const long long in = k - (long long)plane * per_plane;
        const int r = (int)(in / K.nx), x = (int)(in % K.nx);
        const long long at = (long long)(r0 + r) * K.pitch + x;  // element index within a plane
        if (plane < 36) {
            int esz;
            long long off;
            halo_plane<PS>(plane, esz, off, K);
            // message offset: the planes before, each per_plane values of their own size
            const int s = plane / 9, i = plane - 9 * s;
            const long long m = per_plane * ((s == 0 ? 0 : (s == 1 ? set_bytes_before<PS>(1)
                                                     : (s == 2 ? set_bytes_before<PS>(2) : set_bytes_before<PS>(3)))) +
                                             esz * i) + in * esz;
            unsigned char *g = pops + off + at * esz;
            if (esz == 4) {
                if (PACK) *reinterpret_cast<float *>(msg + m) = *reinterpret_cast<const float *>(g);
                else *reinterpret_cast<float *>(g) = *reinterpret_cast<const float *>(msg + m);
            } else {
                if (PACK) *reinterpret_cast<unsigned short *>(msg + m) = *reinterpret_cast<const unsigned short *>(g);
                else *reinterpret_cast<unsigned short *>(g) = *reinterpret_cast<const unsigned short *>(msg + m);
            }
        } else {
            float *a = aux + (long long)(plane - 36) * K.plane + at;
            float *mm = reinterpret_cast<float *>(msg + pop_bytes) + (long long)(plane - 36) * per_plane + in;
            if (PACK) *mm = *a;
            else *a = *mm;
        }
    }
}

}  // namespace lbk
