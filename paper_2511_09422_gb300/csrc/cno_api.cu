// cno_api.cu -- host side of the C ABI declared in include/cno.h: tensor maps,
// launch configuration, the network object (buffers, forward, backward, Adam)
// and the coupling kernels with the LB fields.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cno.h"
#include "cno_kernels.cuh"

using cnok::bf16;

static thread_local std::string t_error;

static cno_status fail(cno_status code, const std::string &msg)
{
    t_error = msg;
    return code;
}

#define CK(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? CNO_ERR_OOM : CNO_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

#define CS(call)                      \
    do {                              \
        cno_status s_ = (call);       \
        if (s_ != CNO_OK)             \
            return s_;                \
    } while (0)

extern "C" const char *cno_error_string(void) { return t_error.c_str(); }

// ---------------------------------------------------------------------------
// Tensor maps
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// NHWC bf16 tensor [n][h][w][c] as a 4-D map (c, w, h, n) with a box of
// 64 channels x bw x bh pixels x 1 image, 128-byte swizzle, zero fill.
static cno_status map_nhwc(CUtensorMap *m, const void *p, int n, int h, int w, int c, int bw, int bh)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(CNO_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
    cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)w * c * 2, (cuuint64_t)h * w * c * 2};
    cuuint32_t box[4] = {64, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(p), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(CNO_ERR_INVALID_ARG, "tensor map of an NHWC tensor rejected (error " + std::to_string(r) + ")");
    return CNO_OK;
}

// Row-major bf16 matrix [rows][k] as a 2-D map (k, rows), box 64 x brows.
static cno_status map_matrix(CUtensorMap *m, const void *p, int rows, int k, int brows)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(CNO_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)k * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)brows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(p), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(CNO_ERR_INVALID_ARG, "tensor map of a weight matrix rejected (error " + std::to_string(r) + ")");
    return CNO_OK;
}

// ---------------------------------------------------------------------------
// Per-device scratch of the primitives
// ---------------------------------------------------------------------------
struct DevScratch {
    unsigned *status = nullptr;
    float *partial = nullptr;
    size_t partial_floats = 0;
};
static std::mutex g_mu;
static DevScratch g_scratch[64];

static cno_status scratch(DevScratch **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64)
        return fail(CNO_ERR_UNSUPPORTED, "device index out of range");
    DevScratch &s = g_scratch[dev];
    if (!s.status) {
        CK(cudaMalloc(&s.status, sizeof(unsigned)));
        CK(cudaMemset(s.status, 0, sizeof(unsigned)));
    }
    *out = &s;
    return CNO_OK;
}

static cno_status grow(float **buf, size_t *have, size_t need)
{
    if (need <= *have)
        return CNO_OK;
    if (*buf)
        CK(cudaFree(*buf));
    *buf = nullptr;
    *have = 0;
    CK(cudaMalloc(buf, need * sizeof(float)));
    *have = need;
    return CNO_OK;
}

static int g_sms = 0;
static int num_sms()
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0)
            g_sms = 148;
    }
    return g_sms;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static bool chan_ok(int c) { return c >= 64 && c % 64 == 0 && c <= 4096; }

static cno_status check_image(int n, int h, int w)
{
    if (n < 1 || h < 1 || w < 1)
        return fail(CNO_ERR_INVALID_ARG, "n, h, w must be positive");
    if (w < 128 && (w & (w - 1)) != 0)
        return fail(CNO_ERR_INVALID_ARG, "w must be at least 128 or a power of two");
    if ((long long)n * h * w > (1LL << 31))
        return fail(CNO_ERR_INVALID_ARG, "too many pixels");
    return CNO_OK;
}

static int pick_bn(int cout)
{
    if (cout % 256 == 0)
        return 256;
    if (cout % 128 == 0)
        return 128;
    return 64;
}

template <int BN>
static cno_status launch_fprop_bn(const CUtensorMap &mx, const CUtensorMap &mw, const cnok::ConvArgs &a, int tiles,
                                  cudaStream_t st)
{
    using S = cnok::ConvShape<BN>;
    static bool attr = false;
    if (!attr) {
        CK(cudaFuncSetAttribute(cnok::conv_fprop_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
        attr = true;
    }
    // persistent: at most the CTAs that fit on the SMs at once
    const int ctas = std::min(tiles, S::CTAS_PER_SM * num_sms());
    dim3 grid(ctas, a.cout / BN);
    cnok::conv_fprop_kernel<BN><<<grid, 192, S::SMEM, st>>>(mx, mw, a);
    CK(cudaGetLastError());
    return CNO_OK;
}

// Common launcher of forward (epi = BIAS / BIAS_LRELU) and data-gradient
// (epi = SLOPE / PLAIN) convolutions: out[p][o] = sum_{t,i} in[p + s_t][i] wmat[o][t][i].
static cno_status conv_launch(const void *in, int n, int h, int w, int cin, const void *wmat, int cout, int epi,
                              const float *bias, const void *slope_src, void *out, int out_f32, int out_cs,
                              int n_store, unsigned *status, cudaStream_t st)
{
    CS(check_image(n, h, w));
    if (!chan_ok(cin) || !chan_ok(cout))
        return fail(CNO_ERR_INVALID_ARG, "channel counts must be positive multiples of 64");
    if (!in || !wmat || !out || n_store < 1 || n_store > cout || out_cs < n_store)
        return fail(CNO_ERR_INVALID_ARG, "null pointer or bad output channel layout");
    if (!out_f32 && (n_store % 8 != 0 || out_cs % 8 != 0))
        return fail(CNO_ERR_INVALID_ARG, "bf16 output needs n_store and out_cs multiples of 8");
    if (((uintptr_t)in | (uintptr_t)wmat | (uintptr_t)out) & 15)
        return fail(CNO_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    const int wt = w >= 128 ? 128 : w;
    const int ht = 128 / wt;
    CUtensorMap mx, mw;
    const int bn = pick_bn(cout);
    CS(map_nhwc(&mx, in, n, h, w, cin, wt, ht));
    CS(map_matrix(&mw, wmat, cout, 9 * cin, bn));
    cnok::ConvArgs a;
    a.n = n;
    a.h = h;
    a.w = w;
    a.cin = cin;
    a.cout = cout;
    a.wt = wt;
    a.ht = ht;
    a.tiles_w = (w + wt - 1) / wt;
    a.tiles_h = (h + ht - 1) / ht;
    a.cblocks = cin / 64;
    a.kblocks = 9 * a.cblocks;
    a.tiles = (int)std::min<long long>((long long)n * a.tiles_w * a.tiles_h, 0x7fffffffLL);
    a.epi = epi;
    a.bias = bias;
    a.slope_src = (const bf16 *)slope_src;
    a.out = out;
    a.out_cs = out_cs;
    a.n_store = n_store;
    a.out_f32 = out_f32;
    a.status = status;
    const long long tiles = (long long)n * a.tiles_w * a.tiles_h;
    if (tiles > 0x7fffffffLL)
        return fail(CNO_ERR_INVALID_ARG, "too many tiles");
    switch (bn) {
    case 256: return launch_fprop_bn<256>(mx, mw, a, (int)tiles, st);
    case 128: return launch_fprop_bn<128>(mx, mw, a, (int)tiles, st);
    default: return launch_fprop_bn<64>(mx, mw, a, (int)tiles, st);
    }
}

template <int BN>
static cno_status launch_wgrad_bn(const CUtensorMap &mdz, const CUtensorMap &mx, const cnok::WgradArgs &a,
                                  cudaStream_t st)
{
    using S = cnok::WgradShape<BN>;
    static bool attr = false;
    if (!attr) {
        CK(cudaFuncSetAttribute(cnok::conv_wgrad_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
        attr = true;
    }
    dim3 grid(9 * a.mtiles * a.ntiles, a.splits);
    cnok::conv_wgrad_kernel<BN><<<grid, 192, S::SMEM, st>>>(mdz, mx, a);
    CK(cudaGetLastError());
    return CNO_OK;
}

static unsigned grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    const long long cap = (long long)num_sms() * 8;
    return (unsigned)std::max(1LL, std::min(g, cap));
}

// Tiling of a weight gradient: 64-pixel K blocks (wt x ht pixels of one
// image), 9 taps x output-channel tiles x input-channel tiles, and as many
// pixel ranges ("splits") as fill one wave of two CTAs per SM, with at least
// 8 K blocks each.
static void wgrad_plan(int n, int h, int w, int cin, int cout, cnok::WgradArgs *a, int *bn)
{
    *bn = pick_bn(cin);
    a->n = n;
    a->h = h;
    a->w = w;
    a->cin = cin;
    a->cout = cout;
    a->wt = w >= 64 ? 64 : w;
    a->ht = 64 / a->wt;
    a->tiles_w = (w + a->wt - 1) / a->wt;
    a->tiles_h = (h + a->ht - 1) / a->ht;
    a->kb_total = n * a->tiles_w * a->tiles_h;
    a->mtiles = (cout + 127) / 128;
    a->ntiles = cin / *bn;
    // one wave: at most two CTAs per SM in total
    const int base = 9 * a->mtiles * a->ntiles;
    int splits = (2 * num_sms()) / base;
    splits = std::max(1, std::min(splits, a->kb_total / 8));
    a->kb_per_split = (a->kb_total + splits - 1) / splits;
    a->splits = (a->kb_total + a->kb_per_split - 1) / a->kb_per_split;
}

// Blocks of the bias-gradient first pass: two per SM, at least 256 pixels each.
static int bias_blocks(int n, int h, int w)
{
    const long long npix = (long long)n * h * w;
    return (int)std::max(1LL, std::min((long long)2 * num_sms(), (npix + 255) / 256));
}

// FP32 scratch of a weight gradient: the per-range partials of dW, reused for
// the per-block partials of db.
static size_t wgrad_scratch_floats(int n, int h, int w, int cin, int cout)
{
    cnok::WgradArgs a;
    int bn;
    wgrad_plan(n, h, w, cin, cout, &a, &bn);
    return (size_t)std::max((long long)a.splits * cout * 9 * cin, (long long)bias_blocks(n, h, w) * cout);
}

// Weight gradient into dw (FP32 [cout][9][cin]) and optionally db; `partial`
// must hold wgrad_scratch_floats() floats.
static cno_status wgrad_launch(const void *dz, const void *x, int n, int h, int w, int cin, int cout, float *dw,
                               float *db, float *partial, size_t partial_floats, unsigned *status, cudaStream_t st)
{
    CS(check_image(n, h, w));
    if (!chan_ok(cin) || !chan_ok(cout) || !dz || !x || !dw)
        return fail(CNO_ERR_INVALID_ARG, "bad weight-gradient arguments");
    if (((uintptr_t)dz | (uintptr_t)x) & 15)
        return fail(CNO_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    if (!partial || partial_floats < wgrad_scratch_floats(n, h, w, cin, cout))
        return fail(CNO_ERR_INVALID_ARG, "internal: weight-gradient scratch too small");
    cnok::WgradArgs a;
    int bn;
    wgrad_plan(n, h, w, cin, cout, &a, &bn);
    CUtensorMap mdz, mx;
    CS(map_nhwc(&mdz, dz, n, h, w, cout, a.wt, a.ht));
    CS(map_nhwc(&mx, x, n, h, w, cin, a.wt, a.ht));
    a.partial = partial;
    a.status = status;
    switch (bn) {
    case 256: CS(launch_wgrad_bn<256>(mdz, mx, a, st)); break;
    case 128: CS(launch_wgrad_bn<128>(mdz, mx, a, st)); break;
    default: CS(launch_wgrad_bn<64>(mdz, mx, a, st)); break;
    }
    const long long count = (long long)cout * 9 * cin;
    cnok::sum_partials_kernel<<<grid_for(count, 256), 256, 0, st>>>(partial, a.splits, count, dw);
    CK(cudaGetLastError());
    if (db) {
        // bias gradient: per-block channel sums, then the blocks in order (the
        // same stream orders this after the weight sum above)
        const long long npix = (long long)n * h * w;
        const int blocks = bias_blocks(n, h, w);
        const long long ppb = (npix + blocks - 1) / blocks;
        cnok::channel_sum_kernel<<<blocks, 256, 0, st>>>((const bf16 *)dz, npix, cout, ppb, partial);
        CK(cudaGetLastError());
        cnok::sum_partials_kernel<<<grid_for(cout, 256), 256, 0, st>>>(partial, blocks, cout, db);
        CK(cudaGetLastError());
    }
    return CNO_OK;
}

// ---------------------------------------------------------------------------
// Primitives
// ---------------------------------------------------------------------------
extern "C" cno_status cno_read_status(unsigned *out, int clear)
{
    DevScratch *s;
    CS(scratch(&s));
    CK(cudaDeviceSynchronize());
    unsigned v = 0;
    CK(cudaMemcpy(&v, s->status, sizeof(v), cudaMemcpyDeviceToHost));
    if (out)
        *out = v;
    if (clear)
        CK(cudaMemset(s->status, 0, sizeof(unsigned)));
    return CNO_OK;
}

extern "C" cno_status cno_conv3x3_forward(const void *x, int n, int h, int w, int cin, const void *wgt,
                                          const float *bias, int cout, int act, void *y, int y_f32, int y_cs,
                                          int n_store, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DevScratch *s;
    CS(scratch(&s));
    if (!bias)
        return fail(CNO_ERR_INVALID_ARG, "bias is required");
    return conv_launch(x, n, h, w, cin, wgt, cout, act ? cnok::EPI_BIAS_LRELU : cnok::EPI_BIAS, bias, nullptr, y,
                       y_f32, y_cs, n_store, s->status, (cudaStream_t)stream);
}

extern "C" cno_status cno_conv3x3_dgrad(const void *dz, int n, int h, int w, int cout, const void *wd, int cin,
                                        const void *slope_src, void *dx, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DevScratch *s;
    CS(scratch(&s));
    return conv_launch(dz, n, h, w, cout, wd, cin, slope_src ? cnok::EPI_SLOPE : cnok::EPI_PLAIN, nullptr, slope_src,
                       dx, 0, cin, cin, s->status, (cudaStream_t)stream);
}

extern "C" cno_status cno_conv3x3_wgrad(const void *dz, const void *x, int n, int h, int w, int cin, int cout,
                                        float *dw, float *db, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DevScratch *s;
    CS(scratch(&s));
    if (chan_ok(cin) && chan_ok(cout) && check_image(n, h, w) == CNO_OK) {
        const size_t need = wgrad_scratch_floats(n, h, w, cin, cout);
        if (need > s->partial_floats) {
            CK(cudaDeviceSynchronize());  // earlier launches may still read the old scratch
            CS(grow(&s->partial, &s->partial_floats, need));
        }
    }
    return wgrad_launch(dz, x, n, h, w, cin, cout, dw, db, s->partial, s->partial_floats, s->status,
                        (cudaStream_t)stream);
}

extern "C" cno_status cno_wait_selftest(double seconds, int *gave_up, double *elapsed)
{
    if (!gave_up || !elapsed || !(seconds > 0.0) || seconds > 10.0)
        return fail(CNO_ERR_INVALID_ARG, "seconds must lie in (0, 10]");
    DevScratch *s;
    CS(scratch(&s));
    unsigned long long *d = nullptr, h[2] = {0, 0};
    CK(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    cnok::wait_selftest_kernel<<<1, 1>>>((unsigned long long)(seconds * 1e9), s->status, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess)
        return fail(CNO_ERR_CUDA, cudaGetErrorString(e));
    *gave_up = (int)h[0];
    *elapsed = (double)h[1] * 1e-9;
    return CNO_OK;
}

extern "C" cno_status cno_weights_to_bf16(const float *w, int cout, int cin, void *wf, void *wd, void *stream)
{
    if (!w || !wf || !wd || cout < 1 || cin < 1)
        return fail(CNO_ERR_INVALID_ARG, "bad weight conversion arguments");
    const long long total = (long long)cout * 9 * cin;
    cnok::weights_to_bf16_kernel<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(w, cout, cin, (bf16 *)wf,
                                                                                         (bf16 *)wd);
    CK(cudaGetLastError());
    return CNO_OK;
}

// ---------------------------------------------------------------------------
// Network
// ---------------------------------------------------------------------------
struct Layer {
    int cin, cout, act;
    long long w_off, b_off;  // offsets into the flat parameter vector
};

struct cno_net {
    int cin, cout, nf;
    int widths[4];
    std::vector<Layer> layers;
    long long nparams = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, gradient, Adam moments
    std::vector<bf16 *> wf, wd;                                       // bf16 forward / data-gradient weights
    long long step = 0;
    cudaStream_t st = nullptr;
    unsigned *status = nullptr;
    double *loss_partial = nullptr;
    double loss_host = 0.0;
    // activation and gradient buffers for the current shape
    int an = 0, ah = 0, aw = 0;
    std::vector<bf16 *> act;      // named activations (see enum below)
    std::vector<bf16 *> grad;     // named gradients
    float *out = nullptr;         // head output FP32 [pix][8]
    bf16 *dout = nullptr;         // loss gradient bf16 [pix][cout]
    float *partial = nullptr;
    size_t partial_floats = 0;
};

enum {
    A_X0, A_A0, A_E0, A_U0, A_D0,       // level 0
    A_P1, A_A1, A_E1, A_U1, A_D1,       // level 1
    A_P2, A_A2, A_E2, A_U2, A_D2,       // level 2
    A_P3, A_A3, A_E3,                   // level 3
    A_COUNT
};
static const int k_act_level[A_COUNT] = {0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3};

enum {
    G_DZ10, G_DU0, G_DZ1, G_DZ0,        // level 0
    G_DZ9, G_DU1, G_DZ3, G_DZ2, G_DP1,  // level 1 (dp1 is at level 1)
    G_DZ8, G_DU2, G_DZ5, G_DZ4, G_DP2,  // level 2
    G_DZ7, G_DZ6, G_DP3,                // level 3
    G_COUNT
};
static const int k_grad_level[G_COUNT] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3};

static int act_channels(const cno_net *net, int a)
{
    switch (a) {
    case A_X0: return net->cin;
    case A_P1: return net->widths[0];   // pooled level-0 output
    case A_P2: return net->widths[1];
    case A_P3: return net->widths[2];
    case A_D2: return net->widths[1];
    case A_D1: return net->widths[0];
    default: return net->widths[k_act_level[a]];
    }
}

static int grad_channels(const cno_net *net, int g)
{
    switch (g) {
    case G_DZ9: return net->widths[0];  // gradient of d1 (c0 channels, level 1)
    case G_DZ8: return net->widths[1];  // gradient of d2 (c1 channels, level 2)
    case G_DZ7: return net->widths[3];
    case G_DZ6: return net->widths[3];
    case G_DP3: return net->widths[2];
    case G_DP2: return net->widths[1];
    case G_DP1: return net->widths[0];
    case G_DZ2: return net->widths[1];
    case G_DZ3: return net->widths[1];
    case G_DU1: return net->widths[1];
    case G_DZ4: return net->widths[2];
    case G_DZ5: return net->widths[2];
    case G_DU2: return net->widths[2];
    default: return net->widths[0];     // level 0: dz10, du0, dz1, dz0
    }
}

static void free_buffers(cno_net *net)
{
    for (auto *p : net->act)
        if (p)
            cudaFree(p);
    for (auto *p : net->grad)
        if (p)
            cudaFree(p);
    net->act.clear();
    net->grad.clear();
    if (net->out)
        cudaFree(net->out);
    if (net->dout)
        cudaFree(net->dout);
    net->out = nullptr;
    net->dout = nullptr;
    net->an = net->ah = net->aw = 0;
}

static cno_status ensure_buffers(cno_net *net, int n, int h, int w, bool training)
{
    if (h % 8 || w % 8)
        return fail(CNO_ERR_INVALID_ARG, "h and w must be multiples of 8");
    CS(check_image(n, h, w));
    const bool have_grads = !net->grad.empty();
    if (net->an == n && net->ah == h && net->aw == w && (!training || have_grads))
        return CNO_OK;
    CK(cudaStreamSynchronize(net->st));
    free_buffers(net);
    net->act.assign(A_COUNT, nullptr);
    for (int a = 1; a < A_COUNT; a++) {  // A_X0 is the caller's input, read in place
        const int l = k_act_level[a];
        const size_t pix = (size_t)n * (h >> l) * (w >> l);
        CK(cudaMalloc(&net->act[a], pix * act_channels(net, a) * sizeof(bf16)));
    }
    const size_t pix0 = (size_t)n * h * w;
    CK(cudaMalloc(&net->out, pix0 * 8 * sizeof(float)));
    if (training) {
        net->grad.assign(G_COUNT, nullptr);
        for (int g = 0; g < G_COUNT; g++) {
            const int l = k_grad_level[g];
            const size_t pix = (size_t)n * (h >> l) * (w >> l);
            CK(cudaMalloc(&net->grad[g], pix * grad_channels(net, g) * sizeof(bf16)));
        }
        CK(cudaMalloc(&net->dout, pix0 * net->cout * sizeof(bf16)));
        size_t need = 0;
        for (int k = 0; k < 12; k++) {
            const Layer &L = net->layers[k];
            const int lv = k <= 1 ? 0 : k <= 3 ? 1 : k <= 5 ? 2 : k <= 7 ? 3 : k == 8 ? 2 : k == 9 ? 1 : 0;
            need = std::max(need, wgrad_scratch_floats(n, h >> lv, w >> lv, L.cin, L.cout));
        }
        CS(grow(&net->partial, &net->partial_floats, need));
    }
    net->an = n;
    net->ah = h;
    net->aw = w;
    return CNO_OK;
}

extern "C" cno_status cno_create(int cin, const int widths[4], int cout, int nf, cno_net **out)
{
    if (!widths || !out)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    for (int l = 0; l < 4; l++)
        if (!chan_ok(widths[l]) || widths[l] > 256)
            return fail(CNO_ERR_INVALID_ARG, "widths must be multiples of 64 up to 256");
    if (widths[3] != widths[2])
        return fail(CNO_ERR_INVALID_ARG, "the level-3 width must equal the level-2 width");
    if (!chan_ok(cin) || cin > 256 || !chan_ok(cout) || cout > 256 || nf < 1 || nf > 8 || nf > cout)
        return fail(CNO_ERR_INVALID_ARG, "cin, cout must be multiples of 64 up to 256; 1 <= nf <= 8");
    cno_net *net = new cno_net();
    net->cin = cin;
    net->cout = cout;
    net->nf = nf;
    memcpy(net->widths, widths, sizeof(net->widths));
    const int c0 = widths[0], c1 = widths[1], c2 = widths[2], c3 = widths[3];
    const int tab[12][3] = {{cin, c0, 1}, {c0, c0, 1}, {c0, c1, 1}, {c1, c1, 1}, {c1, c2, 1}, {c2, c2, 1},
                            {c2, c3, 1},  {c3, c3, 1}, {c3, c1, 1}, {c1, c0, 1}, {c0, c0, 1}, {c0, cout, 0}};
    long long off = 0;
    for (int k = 0; k < 12; k++) {
        Layer L;
        L.cin = tab[k][0];
        L.cout = tab[k][1];
        L.act = tab[k][2];
        L.w_off = off;
        off += (long long)L.cout * 9 * L.cin;
        L.b_off = off;
        off += L.cout;
        net->layers.push_back(L);
    }
    net->nparams = off;
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess)
            return false;
        fail(e == cudaErrorMemoryAllocation ? CNO_ERR_OOM : CNO_ERR_CUDA, cudaGetErrorString(e));
        return true;
    };
    if (bad(cudaMalloc(&net->p, off * sizeof(float))) || bad(cudaMalloc(&net->g, off * sizeof(float))) ||
        bad(cudaMalloc(&net->m, off * sizeof(float))) || bad(cudaMalloc(&net->v, off * sizeof(float))) ||
        bad(cudaMalloc(&net->status, sizeof(unsigned))) || bad(cudaMalloc(&net->loss_partial, 4096 * sizeof(double))) ||
        bad(cudaMemset(net->p, 0, off * sizeof(float))) || bad(cudaMemset(net->g, 0, off * sizeof(float))) ||
        bad(cudaMemset(net->m, 0, off * sizeof(float))) || bad(cudaMemset(net->v, 0, off * sizeof(float))) ||
        bad(cudaMemset(net->status, 0, sizeof(unsigned)))) {
        cno_destroy(net);
        return t_error.find("memory") != std::string::npos ? CNO_ERR_OOM : CNO_ERR_CUDA;
    }
    for (int k = 0; k < 12; k++) {
        bf16 *a = nullptr, *b = nullptr;
        const size_t cnt = (size_t)net->layers[k].cout * 9 * net->layers[k].cin;
        if (bad(cudaMalloc(&a, cnt * sizeof(bf16))) || bad(cudaMalloc(&b, cnt * sizeof(bf16)))) {
            if (a)
                cudaFree(a);
            cno_destroy(net);
            return CNO_ERR_OOM;
        }
        net->wf.push_back(a);
        net->wd.push_back(b);
    }
    *out = net;
    return CNO_OK;
}

extern "C" cno_status cno_destroy(cno_net *net)
{
    if (!net)
        return CNO_OK;
    cudaStreamSynchronize(net->st);
    free_buffers(net);
    for (auto *p : net->wf)
        cudaFree(p);
    for (auto *p : net->wd)
        cudaFree(p);
    for (void *p : {(void *)net->p, (void *)net->g, (void *)net->m, (void *)net->v, (void *)net->status,
                    (void *)net->loss_partial, (void *)net->partial})
        if (p)
            cudaFree(p);
    delete net;
    return CNO_OK;
}

extern "C" cno_status cno_set_stream(cno_net *net, void *stream)
{
    if (!net)
        return fail(CNO_ERR_INVALID_ARG, "null network");
    net->st = (cudaStream_t)stream;
    return CNO_OK;
}

extern "C" cno_status cno_num_params(const cno_net *net, long long *out)
{
    if (!net || !out)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    *out = net->nparams;
    return CNO_OK;
}

static cno_status refresh_bf16(cno_net *net)
{
    for (int k = 0; k < 12; k++) {
        const Layer &L = net->layers[k];
        CS(cno_weights_to_bf16(net->p + L.w_off, L.cout, L.cin, net->wf[k], net->wd[k], net->st));
    }
    return CNO_OK;
}

static cno_status check_status(cno_net *net)
{
    unsigned v = 0;
    CK(cudaMemcpyAsync(&v, net->status, sizeof(v), cudaMemcpyDeviceToHost, net->st));
    CK(cudaStreamSynchronize(net->st));
    if (v)
        return fail(CNO_ERR_DEVICE_WAIT, "a tensor-core kernel gave up waiting (status " + std::to_string(v) + ")");
    return CNO_OK;
}

extern "C" cno_status cno_set_params(cno_net *net, const float *host)
{
    if (!net || !host)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    CK(cudaMemcpyAsync(net->p, host, net->nparams * sizeof(float), cudaMemcpyHostToDevice, net->st));
    CK(cudaMemsetAsync(net->m, 0, net->nparams * sizeof(float), net->st));
    CK(cudaMemsetAsync(net->v, 0, net->nparams * sizeof(float), net->st));
    net->step = 0;
    CS(refresh_bf16(net));
    CK(cudaStreamSynchronize(net->st));
    return CNO_OK;
}

extern "C" cno_status cno_get_params(cno_net *net, float *host)
{
    if (!net || !host)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    CK(cudaMemcpyAsync(host, net->p, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, net->st));
    CK(cudaStreamSynchronize(net->st));
    return CNO_OK;
}

extern "C" cno_status cno_get_grads(cno_net *net, float *host)
{
    if (!net || !host)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    CK(cudaMemcpyAsync(host, net->g, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, net->st));
    CK(cudaStreamSynchronize(net->st));
    return CNO_OK;
}

static cno_status fwd_conv(cno_net *net, int k, const bf16 *in, int lv, bf16 *out_bf)
{
    const Layer &L = net->layers[k];
    const int h = net->ah >> lv, w = net->aw >> lv;
    if (k == 11)
        return conv_launch(in, net->an, h, w, L.cin, net->wf[k], L.cout, cnok::EPI_BIAS, net->p + L.b_off, nullptr,
                           net->out, 1, 8, 8, net->status, net->st);
    return conv_launch(in, net->an, h, w, L.cin, net->wf[k], L.cout, cnok::EPI_BIAS_LRELU, net->p + L.b_off, nullptr,
                       out_bf, 0, L.cout, L.cout, net->status, net->st);
}

static cno_status pool(cno_net *net, const bf16 *x, int lv_out, int c, bf16 *y)
{
    const int ho = net->ah >> lv_out, wo = net->aw >> lv_out;
    const long long total = (long long)net->an * ho * wo * (c / 8);
    cnok::pool2_kernel<<<grid_for(total, 256), 256, 0, net->st>>>(x, net->an, ho, wo, c, y);
    CK(cudaGetLastError());
    return CNO_OK;
}

static cno_status up_add(cno_net *net, const bf16 *x, const bf16 *skip, int lv_out, int c, bf16 *u)
{
    const int h = net->ah >> lv_out, w = net->aw >> lv_out;
    const long long total = (long long)net->an * h * w * (c / 8);
    cnok::up_add_kernel<<<grid_for(total, 256), 256, 0, net->st>>>(x, skip, net->an, h, w, c, u);
    CK(cudaGetLastError());
    return CNO_OK;
}

static cno_status forward_all(cno_net *net, const bf16 *x)
{
    auto &A = net->act;
    const int c0 = net->widths[0], c1 = net->widths[1], c2 = net->widths[2];
    const bf16 *x0 = x;
    CS(fwd_conv(net, 0, x0, 0, A[A_A0]));
    CS(fwd_conv(net, 1, A[A_A0], 0, A[A_E0]));
    CS(pool(net, A[A_E0], 1, c0, A[A_P1]));
    CS(fwd_conv(net, 2, A[A_P1], 1, A[A_A1]));
    CS(fwd_conv(net, 3, A[A_A1], 1, A[A_E1]));
    CS(pool(net, A[A_E1], 2, c1, A[A_P2]));
    CS(fwd_conv(net, 4, A[A_P2], 2, A[A_A2]));
    CS(fwd_conv(net, 5, A[A_A2], 2, A[A_E2]));
    CS(pool(net, A[A_E2], 3, c2, A[A_P3]));
    CS(fwd_conv(net, 6, A[A_P3], 3, A[A_A3]));
    CS(fwd_conv(net, 7, A[A_A3], 3, A[A_E3]));
    CS(up_add(net, A[A_E3], A[A_E2], 2, c2, A[A_U2]));
    CS(fwd_conv(net, 8, A[A_U2], 2, A[A_D2]));
    CS(up_add(net, A[A_D2], A[A_E1], 1, c1, A[A_U1]));
    CS(fwd_conv(net, 9, A[A_U1], 1, A[A_D1]));
    CS(up_add(net, A[A_D1], A[A_E0], 0, c0, A[A_U0]));
    CS(fwd_conv(net, 10, A[A_U0], 0, A[A_D0]));
    CS(fwd_conv(net, 11, A[A_D0], 0, nullptr));
    return CNO_OK;
}

extern "C" cno_status cno_forward(cno_net *net, const void *x, int n, int h, int w, float *out, int out_cs)
{
    if (!net || !x)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    if (out && out_cs < net->nf)
        return fail(CNO_ERR_INVALID_ARG, "out_cs must be at least nf");
    CS(ensure_buffers(net, n, h, w, false));
    CS(forward_all(net, (const bf16 *)x));
    if (out) {
        CK(cudaMemcpy2DAsync(out, (size_t)out_cs * sizeof(float), net->out, 8 * sizeof(float),
                             net->nf * sizeof(float), (size_t)n * h * w, cudaMemcpyDeviceToDevice, net->st));
    }
    return CNO_OK;
}

extern "C" cno_status cno_last_output(cno_net *net, const float **out)
{
    if (!net || !out)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    *out = net->out;
    return CNO_OK;
}

static cno_status dgrad(cno_net *net, int k, const bf16 *dz, int lv, const bf16 *slope_src, bf16 *dx)
{
    const Layer &L = net->layers[k];
    return conv_launch(dz, net->an, net->ah >> lv, net->aw >> lv, L.cout, net->wd[k], L.cin,
                       slope_src ? cnok::EPI_SLOPE : cnok::EPI_PLAIN, nullptr, slope_src, dx, 0, L.cin, L.cin,
                       net->status, net->st);
}

static cno_status wgrad(cno_net *net, int k, const bf16 *dz, const bf16 *x, int lv)
{
    const Layer &L = net->layers[k];
    return wgrad_launch(dz, x, net->an, net->ah >> lv, net->aw >> lv, L.cin, L.cout, net->g + L.w_off,
                        net->g + L.b_off, net->partial, net->partial_floats, net->status, net->st);
}

static cno_status up_bwd(cno_net *net, const bf16 *du, const bf16 *y, int lv_out, int c, bf16 *dz)
{
    const int ho = net->ah >> lv_out, wo = net->aw >> lv_out;
    const long long total = (long long)net->an * ho * wo * (c / 8);
    cnok::up_bwd_kernel<<<grid_for(total, 256), 256, 0, net->st>>>(du, y, net->an, ho, wo, c, dz);
    CK(cudaGetLastError());
    return CNO_OK;
}

static cno_status pool_bwd(cno_net *net, const bf16 *du, const bf16 *dp, const bf16 *e, int lv, int c, bf16 *dz)
{
    const int h = net->ah >> lv, w = net->aw >> lv;
    const long long total = (long long)net->an * h * w * (c / 8);
    cnok::pool_bwd_kernel<<<grid_for(total, 256), 256, 0, net->st>>>(du, dp, e, net->an, h, w, c, dz);
    CK(cudaGetLastError());
    return CNO_OK;
}

static cno_status backward_all(cno_net *net, const bf16 *x0)
{
    auto &A = net->act;
    auto &G = net->grad;
    const int c0 = net->widths[0], c1 = net->widths[1], c2 = net->widths[2], c3 = net->widths[3];
    const bf16 *dout = net->dout;
    // level 0 decoder and head
    CS(wgrad(net, 11, dout, A[A_D0], 0));
    CS(dgrad(net, 11, dout, 0, A[A_D0], G[G_DZ10]));
    CS(wgrad(net, 10, G[G_DZ10], A[A_U0], 0));
    CS(dgrad(net, 10, G[G_DZ10], 0, nullptr, G[G_DU0]));
    CS(up_bwd(net, G[G_DU0], A[A_D1], 1, c0, G[G_DZ9]));
    // level 1 decoder
    CS(wgrad(net, 9, G[G_DZ9], A[A_U1], 1));
    CS(dgrad(net, 9, G[G_DZ9], 1, nullptr, G[G_DU1]));
    CS(up_bwd(net, G[G_DU1], A[A_D2], 2, c1, G[G_DZ8]));
    // level 2 decoder
    CS(wgrad(net, 8, G[G_DZ8], A[A_U2], 2));
    CS(dgrad(net, 8, G[G_DZ8], 2, nullptr, G[G_DU2]));
    CS(up_bwd(net, G[G_DU2], A[A_E3], 3, c3, G[G_DZ7]));
    // level 3
    CS(wgrad(net, 7, G[G_DZ7], A[A_A3], 3));
    CS(dgrad(net, 7, G[G_DZ7], 3, A[A_A3], G[G_DZ6]));
    CS(wgrad(net, 6, G[G_DZ6], A[A_P3], 3));
    CS(dgrad(net, 6, G[G_DZ6], 3, nullptr, G[G_DP3]));
    // level 2 encoder
    CS(pool_bwd(net, G[G_DU2], G[G_DP3], A[A_E2], 2, c2, G[G_DZ5]));
    CS(wgrad(net, 5, G[G_DZ5], A[A_A2], 2));
    CS(dgrad(net, 5, G[G_DZ5], 2, A[A_A2], G[G_DZ4]));
    CS(wgrad(net, 4, G[G_DZ4], A[A_P2], 2));
    CS(dgrad(net, 4, G[G_DZ4], 2, nullptr, G[G_DP2]));
    // level 1 encoder
    CS(pool_bwd(net, G[G_DU1], G[G_DP2], A[A_E1], 1, c1, G[G_DZ3]));
    CS(wgrad(net, 3, G[G_DZ3], A[A_A1], 1));
    CS(dgrad(net, 3, G[G_DZ3], 1, A[A_A1], G[G_DZ2]));
    CS(wgrad(net, 2, G[G_DZ2], A[A_P1], 1));
    CS(dgrad(net, 2, G[G_DZ2], 1, nullptr, G[G_DP1]));
    // level 0 encoder
    CS(pool_bwd(net, G[G_DU0], G[G_DP1], A[A_E0], 0, c0, G[G_DZ1]));
    CS(wgrad(net, 1, G[G_DZ1], A[A_A0], 0));
    CS(dgrad(net, 1, G[G_DZ1], 0, A[A_A0], G[G_DZ0]));
    CS(wgrad(net, 0, G[G_DZ0], x0, 0));
    return CNO_OK;
}

extern "C" cno_status cno_train_step(cno_net *net, const void *x, const float *target, int n, int h, int w,
                                     float lr, int update, double *loss)
{
    if (!net || !x || !target)
        return fail(CNO_ERR_INVALID_ARG, "null pointer");
    CS(ensure_buffers(net, n, h, w, true));
    CS(forward_all(net, (const bf16 *)x));
    const long long npix = (long long)n * h * w;
    const unsigned blocks = std::min<unsigned>(4096u, grid_for(npix, 256));
    cnok::mse_kernel<<<blocks, 256, 0, net->st>>>(net->out, 8, target, net->nf, npix, net->cout,
                                                  1.0 / ((double)npix * net->nf), net->dout, net->loss_partial);
    CK(cudaGetLastError());
    CS(backward_all(net, (const bf16 *)x));
    if (update) {
        net->step++;
        const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
        const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
        cnok::adam_kernel<<<grid_for(net->nparams, 256), 256, 0, net->st>>>(net->p, net->g, net->m, net->v,
                                                                            net->nparams, lr, 0.9f, 0.999f,
                                                                            (float)(1.0 - 0.9), (float)(1.0 - 0.999),
                                                                            1e-8f, c1, c2);
        CK(cudaGetLastError());
        CS(refresh_bf16(net));
    }
    if (loss) {
        std::vector<double> part(blocks);
        CK(cudaMemcpyAsync(part.data(), net->loss_partial, blocks * sizeof(double), cudaMemcpyDeviceToHost, net->st));
        CS(check_status(net));
        double s = 0.0;
        for (double v : part)
            s += v;
        *loss = s / ((double)npix * net->nf);
    }
    return CNO_OK;
}

// ---------------------------------------------------------------------------
// Coupling with the LB fields
// ---------------------------------------------------------------------------
namespace {
constexpr int MAXF = 8;
struct FieldPtrs {
    const float *f[MAXF];
    float off[MAXF], sc[MAXF];
};
struct FieldOut {
    float *f[MAXF];
    float sc[MAXF], lo[MAXF], hi[MAXF];
};

__global__ void pack_fields_kernel(FieldPtrs fp, int nfield, long long npix, int cin, bf16 *__restrict__ x)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < cin; c += 8) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int k = c + e;
                v[e] = k < nfield ? (fp.f[k][p] - fp.off[k]) * fp.sc[k] : 0.0f;
            }
            *(uint4 *)(x + p * cin + c) = cnok::pack8(v);
        }
    }
}

__global__ void pack_delta_kernel(FieldPtrs cur, FieldPtrs next, int nfield, long long npix, float *__restrict__ t)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < nfield; k++)
            t[p * nfield + k] = (next.f[k][p] - cur.f[k][p]) * cur.sc[k];
    }
}

__global__ void apply_update_kernel(FieldPtrs src, FieldOut dst, int nfield, long long npix,
                                    const float *__restrict__ out, int out_cs, float phi_band)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < nfield; k++) {
            const float v = src.f[k][p];
            const bool frozen = dst.sc[k] == 0.0f || (k == 0 && phi_band > 0.0f && fabsf(v) >= phi_band);
            dst.f[k][p] = frozen ? v : fminf(fmaxf(v + dst.sc[k] * out[p * out_cs + k], dst.lo[k]), dst.hi[k]);
        }
    }
}

// per-row sums of phi, chi, f_s, 1 - phi^2, |grad phi|, the row's minimum and
// maximum of T, and the sum of rho H (FP64), one block per row
constexpr int NCHK = 8;
struct HCoef {
    double cl, cs, cg, lat;
    int on;
};
__global__ void field_rows_kernel(const float *__restrict__ phi, const float *__restrict__ fs,
                                  const float *__restrict__ T, HCoef hc, int nx, int ny, double *__restrict__ rows)
{
    __shared__ double red[NCHK][256];
    const int y = blockIdx.x;
    double s[NCHK] = {0, 0, 0, 0, 0, INFINITY, -INFINITY, 0};
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const long long c = (long long)y * nx + x;
        const double f = phi[c];
        const double fe = phi[(long long)y * nx + (x + 1) % nx], fw = phi[(long long)y * nx + (x + nx - 1) % nx];
        double gy;
        if (ny == 1)
            gy = 0.0;
        else if (y == 0)
            gy = phi[c + nx] - f;
        else if (y == ny - 1)
            gy = f - phi[c - nx];
        else
            gy = 0.5 * (phi[c + nx] - phi[c - nx]);
        const double gx = 0.5 * (fe - fw);
        s[0] += f;
        s[1] += fmin(fmax(0.5 * (1.0 + f), 0.0), 1.0);
        s[2] += fs ? (double)fs[c] : 0.0;
        s[3] += 1.0 - f * f;
        s[4] += sqrt(gx * gx + gy * gy);
        const double t = T ? (double)T[c] : 0.0;
        s[5] = fmin(s[5], t);
        s[6] = fmax(s[6], t);
        if (hc.on) {
            const double chi = fmin(fmax(0.5 * (1.0 + f), 0.0), 1.0);
            const double sol = fmin(fmax((double)fs[c], 0.0), chi);
            s[7] += t * (sol * hc.cs + (chi - sol) * hc.cl + (1.0 - chi) * hc.cg) + hc.lat * (chi - sol);
        }
    }
    for (int k = 0; k < NCHK; k++)
        red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            for (int k = 0; k < 5; k++)
                red[k][threadIdx.x] += red[k][threadIdx.x + st];
            red[5][threadIdx.x] = fmin(red[5][threadIdx.x], red[5][threadIdx.x + st]);
            red[6][threadIdx.x] = fmax(red[6][threadIdx.x], red[6][threadIdx.x + st]);
            red[7][threadIdx.x] += red[7][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NCHK; k++)
            rows[NCHK * y + k] = red[k][0];
}
}  // namespace

extern "C" cno_status cno_pack_fields(const float *const *fields, int nfield, int nx, int ny, const float *offset,
                                      const float *inv_scale, void *x, int cin, void *stream)
{
    if (!fields || !x || !offset || !inv_scale || nfield < 1 || nfield > MAXF || nfield > cin || cin % 8 ||
        nx < 1 || ny < 1)
        return fail(CNO_ERR_INVALID_ARG, "bad pack arguments");
    FieldPtrs fp;
    for (int k = 0; k < MAXF; k++) {
        fp.f[k] = k < nfield ? fields[k] : nullptr;
        fp.off[k] = k < nfield ? offset[k] : 0.0f;
        fp.sc[k] = k < nfield ? inv_scale[k] : 0.0f;
        if (k < nfield && !fields[k])
            return fail(CNO_ERR_INVALID_ARG, "null field");
    }
    const long long npix = (long long)nx * ny;
    pack_fields_kernel<<<grid_for(npix, 256), 256, 0, (cudaStream_t)stream>>>(fp, nfield, npix, cin, (bf16 *)x);
    CK(cudaGetLastError());
    return CNO_OK;
}

static cno_status field_ptrs(const float *const *f, int nfield, const float *sc, FieldPtrs *fp)
{
    for (int k = 0; k < MAXF; k++) {
        fp->f[k] = k < nfield ? f[k] : nullptr;
        fp->off[k] = 0.0f;
        fp->sc[k] = (k < nfield && sc) ? sc[k] : 0.0f;
        if (k < nfield && !f[k])
            return fail(CNO_ERR_INVALID_ARG, "null field");
    }
    return CNO_OK;
}

extern "C" cno_status cno_pack_delta(const float *const *cur, const float *const *next, int nfield, int nx, int ny,
                                     const float *inv_scale, float *target, void *stream)
{
    if (!cur || !next || !inv_scale || !target || nfield < 1 || nfield > MAXF || nx < 1 || ny < 1)
        return fail(CNO_ERR_INVALID_ARG, "bad target arguments");
    FieldPtrs a, b;
    CS(field_ptrs(cur, nfield, inv_scale, &a));
    CS(field_ptrs(next, nfield, inv_scale, &b));
    const long long npix = (long long)nx * ny;
    pack_delta_kernel<<<grid_for(npix, 256), 256, 0, (cudaStream_t)stream>>>(a, b, nfield, npix, target);
    CK(cudaGetLastError());
    return CNO_OK;
}

extern "C" cno_status cno_apply_update(const float *const *src, float *const *dst, int nfield, int nx, int ny,
                                       const float *out, int out_cs, const float *scale, const float *lo,
                                       const float *hi, float phi_band, void *stream)
{
    if (!src || !dst || !out || !scale || nfield < 1 || nfield > MAXF || out_cs < nfield || nx < 1 || ny < 1)
        return fail(CNO_ERR_INVALID_ARG, "bad update arguments");
    FieldPtrs a;
    CS(field_ptrs(src, nfield, nullptr, &a));
    FieldOut o;
    for (int k = 0; k < MAXF; k++) {
        o.f[k] = k < nfield ? dst[k] : nullptr;
        o.sc[k] = k < nfield ? scale[k] : 0.0f;
        o.lo[k] = (k < nfield && lo) ? lo[k] : -INFINITY;
        o.hi[k] = (k < nfield && hi) ? hi[k] : INFINITY;
        if (k < nfield && !dst[k])
            return fail(CNO_ERR_INVALID_ARG, "null field");
    }
    const long long npix = (long long)nx * ny;
    apply_update_kernel<<<grid_for(npix, 256), 256, 0, (cudaStream_t)stream>>>(a, o, nfield, npix, out, out_cs,
                                                                                 phi_band);
    CK(cudaGetLastError());
    return CNO_OK;
}

extern "C" cno_status cno_field_checks(const float *phi, const float *fs, const float *T, const float *hcoef,
                                       int nx, int ny, double out[8], void *stream)
{
    if (!phi || !out || nx < 1 || ny < 1)
        return fail(CNO_ERR_INVALID_ARG, "bad check arguments");
    double *rows = nullptr;
    CK(cudaMallocAsync(&rows, (size_t)ny * NCHK * sizeof(double), (cudaStream_t)stream));
    HCoef hc = {0, 0, 0, 0, 0};
    if (hcoef && fs && T)
        hc = {hcoef[0], hcoef[1], hcoef[2], hcoef[3], 1};
    field_rows_kernel<<<ny, 256, 0, (cudaStream_t)stream>>>(phi, fs, T, hc, nx, ny, rows);
    CK(cudaGetLastError());
    std::vector<double> h((size_t)ny * NCHK);
    CK(cudaMemcpyAsync(h.data(), rows, h.size() * sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaFreeAsync(rows, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    for (int k = 0; k < 5; k++)
        out[k] = 0.0;
    out[5] = INFINITY;
    out[6] = -INFINITY;
    out[7] = 0.0;
    for (int y = 0; y < ny; y++) {
        for (int k = 0; k < 5; k++)
            out[k] += h[(size_t)NCHK * y + k];
        out[5] = std::min(out[5], h[(size_t)NCHK * y + 5]);
        out[6] = std::max(out[6], h[(size_t)NCHK * y + 6]);
        out[7] += h[(size_t)NCHK * y + 7];
    }
    if (!T)
        out[5] = out[6] = 0.0;
    return CNO_OK;
}
