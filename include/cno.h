/* cno.h -- C ABI of the learned surrogate of the LB freezing step.
 *
 * The surrogate is a convolutional neural operator: a four-level U-shaped
 * network of 3x3 convolutions that maps the macroscopic fields of a lattice
 * (phi, T, f_s, C, u_x, u_y, p of Sec. 2-3, normalised) to their change over
 * the next k LB steps.  The paper has no learned component; the network, its
 * training and the checks that decide when the LB step takes over are this
 * library's.  Every operation runs in CUDA kernels for sm_103a: the
 * convolutions are implicit GEMMs on the tensor cores (tcgen05.mma with BF16
 * operands staged by TMA and FP32 accumulators in tensor memory).
 *
 * Network (the same definition as the FP64 reference used by the tests):
 *   activations NHWC bf16 (channel index fastest), weights W[o][t][i] with
 *   tap t = 3 (dy + 1) + (dx + 1), zero padding,
 *   y[n,h,w,o] = b[o] + sum_{t,i} x[n,h+dy,w+dx,i] W[o,t,i];
 *   lrelu(z) = z for z > 0, z / 16 otherwise (slope 1/16 also at z = 0);
 *   level l has widths[l] channels at resolution (H / 2^l, W / 2^l);
 *   encoder: two convolutions + lrelu per level, 2x2 average pooling between
 *   levels; decoder: nearest 2x upsampling, addition of the encoder output of
 *   the level, one convolution + lrelu; a linear 3x3 head with cout channels.
 *   Twelve convolutions in this order (in -> out):
 *     cin->c0, c0->c0, c0->c1, c1->c1, c1->c2, c2->c2, c2->c3, c3->c3,
 *     c3->c1, c1->c0, c0->c0, c0->cout        (c3 must equal c2).
 *   Parameters, flat FP32: for each layer in that order, W (cout*9*cin values)
 *   then b (cout values).
 *
 * Shapes: every channel count (cin, widths, cout) a multiple of 64 and at
 * most 256; H and W multiples of 8; W >= 128 or a power of two.  Device
 * pointers must be 16-byte aligned (cudaMalloc gives 256).
 *
 * Errors: calls return CNO_OK or an error code; cno_error_string describes
 * the last failure of the calling thread.  Kernels give up a wait on the
 * tensor-core pipeline after 4 s and record it in a device status word (one
 * per network, one per device for the primitives); later launches that see the
 * word set do no work.  The next network call that synchronises returns
 * CNO_ERR_DEVICE_WAIT (destroy and recreate the network); for the primitives,
 * cno_read_status reports and clears the word.
 */
#ifndef CNO_H
#define CNO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cno_status;
#define CNO_OK 0
#define CNO_ERR_INVALID_ARG 1
#define CNO_ERR_CUDA 2
#define CNO_ERR_OOM 3
#define CNO_ERR_DEVICE_WAIT 4
#define CNO_ERR_UNSUPPORTED 5

const char *cno_error_string(void);

/* Device status word of the primitives below (not of networks): 0 when no
 * kernel has given up a wait.  Synchronises the device; clear = 1 resets it. */
cno_status cno_read_status(unsigned *out, int clear);

/* Self-test of the bounded barrier wait that every tensor-core kernel uses:
 * one thread waits on a barrier that nothing arrives at.  It must give up
 * after `seconds` (0 < seconds <= 10): *gave_up = 1 and *elapsed the time it
 * waited.  No data, TMA or tensor core is involved.  Synchronises the device. */
cno_status cno_wait_selftest(double seconds, int *gave_up, double *elapsed);

/* ---- Primitives on device tensors (asynchronous on `stream`, a cudaStream_t
 * or NULL for the legacy default stream) ---- */

/* y = conv3x3(x, W) + b, then lrelu if act = 1.
 * x: bf16 [n][h][w][cin].  wgt: bf16 [cout][9][cin].  bias: FP32 [cout].
 * y: [n][h][w][y_cs], FP32 if y_f32 else bf16; channels 0 .. n_store-1 are
 * written (n_store <= cout, a multiple of 8 for bf16 output; y_cs >= n_store). */
cno_status cno_conv3x3_forward(const void *x, int n, int h, int w, int cin, const void *wgt, const float *bias,
                               int cout, int act, void *y, int y_f32, int y_cs, int n_store, void *stream);

/* Data gradient of a convolution: dx = conv3x3(dz, Wd) with Wd[i][t][o] =
 * W[o][8-t][i] (bf16 [cin][9][cout], see cno_weights_to_bf16), times
 * lrelu'(slope_src) elementwise if slope_src (bf16 [n][h][w][cin]) is not NULL.
 * dz: bf16 [n][h][w][cout]; dx: bf16 [n][h][w][cin]. */
cno_status cno_conv3x3_dgrad(const void *dz, int n, int h, int w, int cout, const void *wd, int cin,
                             const void *slope_src, void *dx, void *stream);

/* Weight and bias gradients: dw[o][t][i] = sum_p dz[p][o] x[p + s_t][i],
 * db[o] = sum_p dz[p][o], FP32, summed per pixel range in FP32 and over the
 * ranges in a fixed order (deterministic).  dz: bf16 [n][h][w][cout];
 * x: bf16 [n][h][w][cin]; db may be NULL.  Uses a scratch buffer that the
 * library keeps per device. */
cno_status cno_conv3x3_wgrad(const void *dz, const void *x, int n, int h, int w, int cin, int cout, float *dw,
                             float *db, void *stream);

/* bf16 copies of FP32 weights w[cout][9][cin]: wf (same layout) and wd (the
 * data-gradient layout [cin][9][cout], taps reversed). */
cno_status cno_weights_to_bf16(const float *w, int cout, int cin, void *wf, void *wd, void *stream);

/* ---- Networks ---- */
typedef struct cno_net cno_net;

/* nf: number of leading output channels the loss compares (nf <= cout). */
cno_status cno_create(int cin, const int widths[4], int cout, int nf, cno_net **out);
cno_status cno_destroy(cno_net *net);
cno_status cno_set_stream(cno_net *net, void *stream);
cno_status cno_num_params(const cno_net *net, long long *out);

/* Copy all parameters from / to host memory (the flat FP32 layout above).
 * cno_set_params also resets the Adam state and step count. */
cno_status cno_set_params(cno_net *net, const float *host);
cno_status cno_get_params(cno_net *net, float *host);

/* Gradients of the last cno_train_step (same layout as the parameters). */
cno_status cno_get_grads(cno_net *net, float *host);

/* Inference: x bf16 [n][h][w][cin] (device) -> out FP32 [n][h][w][out_cs]
 * (device), channels 0 .. nf-1 (out_cs >= nf).  Asynchronous. */
cno_status cno_forward(cno_net *net, const void *x, int n, int h, int w, float *out, int out_cs);

/* One training step on a batch: forward, mean squared error over the first
 * nf channels against target (FP32 [n][h][w][nf], device), backward through
 * every layer, and, if update = 1, one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr) on FP32 master parameters.  If loss is not
 * NULL the call synchronises and stores the batch loss (before the update). */
cno_status cno_train_step(cno_net *net, const void *x, const float *target, int n, int h, int w, float lr,
                          int update, double *loss);

/* FP32 output of the last cno_forward / cno_train_step head, device pointer
 * [n][h][w][8] (first 8 channels) valid until the next call on the network. */
cno_status cno_last_output(cno_net *net, const float **out);

/* ---- Coupling with the LB fields (Sec. 2-3 variables) ---- */

/* Pack nfield device FP32 planes (each nx*ny, row-major, x fastest) into the
 * network input: x[0][y][x][k] = (field_k - offset[k]) * inv_scale[k] for
 * k < nfield, 0 for the other cin channels (bf16 NHWC, one image). */
cno_status cno_pack_fields(const float *const *fields, int nfield, int nx, int ny, const float *offset,
                           const float *inv_scale, void *x, int cin, void *stream);

/* Training target from two snapshots of the same lattice k steps apart:
 * target[y][x][f] = (next_f - cur_f) * inv_scale[f] (FP32 [ny][nx][nfield]). */
cno_status cno_pack_delta(const float *const *cur, const float *const *next, int nfield, int nx, int ny,
                          const float *inv_scale, float *target, void *stream);

/* dst_f = src_f + scale[f] * out[y][x][f] for f < nfield (out FP32
 * [ny][nx][out_cs]), then clamped to [lo[f], hi[f]] if lo and hi are given
 * (host arrays of nfield values); dst may equal src.  A field with
 * scale[f] = 0 is copied unchanged (and not clamped).  If phi_band > 0,
 * field 0 (phi) changes only where |src_0| < phi_band: the order parameter
 * moves only inside the interface band, and is left exactly at its bulk
 * values elsewhere. */
cno_status cno_apply_update(const float *const *src, float *const *dst, int nfield, int nx, int ny,
                            const float *out, int out_cs, const float *scale, const float *lo, const float *hi,
                            float phi_band, void *stream);

/* Acceptance checks of a predicted state, FP64 sums in a fixed order over a
 * lattice with walls at y = 0 and y = ny - 1 and periodic x:
 *   out[0] = sum phi,  out[1] = sum chi, chi = clamp((1 + phi) / 2, 0, 1),
 *   out[2] = sum f_s (0 if fs is NULL),
 *   out[3] = sum (1 - phi^2),  out[4] = sum |grad phi| (central differences,
 *   one-sided next to the walls),
 *   out[5], out[6] = minimum and maximum of T (0 if T is NULL),
 *   out[7] = sum rho H, the enthalpy of Sec. 2.3 with the mixture rule of the
 *   volumetric heat capacities: rho H = T (f_s c_s + (chi - f_s) c_l +
 *   (1 - chi) c_g) + L_l (chi - f_s), f_s clamped to [0, chi], from
 *   hcoef = {c_l, c_s, c_g, L_l} = {(rho Cp)_l, (rho Cp)_s, (rho Cp)_g, rho_l L}
 *   (0 if hcoef, fs or T is NULL).
 * The mass of the phase-change material is rho_s out[2] + rho_l (out[1] - out[2]);
 * for a flat profile phi = tanh(2 d / W) the width is W = 2 out[3] / out[4].
 * Synchronises the stream; out is host memory. */
cno_status cno_field_checks(const float *phi, const float *fs, const float *T, const float *hcoef, int nx, int ny,
                            double out[8], void *stream);

#ifdef __cplusplus
}
#endif
#endif
