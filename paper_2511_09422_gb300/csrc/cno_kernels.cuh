// Kernels of the convolutional neural operator used as the learned surrogate
// of the LB step: 3x3 convolutions as implicit GEMMs on the sm_100-family
// tensor cores (tcgen05.mma, BF16 operands, FP32 accumulators in tensor
// memory, operands staged by TMA), plus the elementwise, reduction and
// optimiser kernels of training.
//
// Conventions (the same as the FP64 reference of the network):
//   activations NHWC bf16, channels a multiple of 64 (one 128-byte row);
//   weights W[o][t][i] bf16, tap t = 3 (dy + 1) + (dx + 1), zero padding;
//   y[n,h,w,o] = b[o] + sum_{t,i} x[n,h+dy,w+dx,i] W[o,t,i];
//   lrelu(z) = z (z > 0), z / 16 otherwise.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace cnok {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128;             // tile rows of a GEMM (pixels, or output channels in wgrad)
constexpr int KB = 64;              // K elements per stage: 64 bf16 = one 128-byte swizzle row
constexpr int ROW_BYTES = 128;
constexpr int SUB_BYTES = 64 * ROW_BYTES;   // one 64-row x 128-byte TMA box
constexpr float LRELU_SLOPE = 0.0625f;
constexpr unsigned long long WAIT_NS = 4000000000ull;  // bound of every barrier wait

// status bits
constexpr unsigned ST_TIMEOUT_PRODUCER = 1u, ST_TIMEOUT_MMA = 2u, ST_TIMEOUT_EPILOGUE = 4u;

// --------------------------------------------------------------------------
// PTX wrappers
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase `parity` of a barrier to complete, for at most limit_ns;
// gives up early when another CTA has already reported a failure.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const unsigned *status,
                                          unsigned long long limit_ns = WAIT_NS)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; it++) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 63u) == 0u) {
            if (*(volatile const unsigned *)status != 0u)
                return false;
            if (global_ns() - t0 > limit_ns)
                return false;
        }
    }
}


__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Self-test of the bounded wait: one thread waits on a barrier that nothing
// arrives at; the wait must give up after limit_ns and report it in out[0]
// (1: gave up), with the elapsed time in out[1] (ns).
__global__ void wait_selftest_kernel(unsigned long long limit_ns, const unsigned *status,
                                     unsigned long long *out)
{
    __shared__ uint64_t bar;
    mbar_init(&bar, 1);
    fence_barrier_init();
    const unsigned long long t0 = global_ns();
    const bool ok = mbar_wait(&bar, 0, status, limit_ns);
    out[0] = ok ? 0ull : 1ull;
    out[1] = global_ns() - t0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tensor memory, FP32) = A * B^T (+ D if accumulate): BF16 operands from
// shared memory descriptors, shape and majors in idesc.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on a barrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of the warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++)
        v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a tcgen05 operand in the 128-byte
// swizzled layout: start address, leading- and stride-dimension byte offsets,
// descriptor version 1 (bits 46-48), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, M x N; a_mn /
// b_mn select the MN-major form of an operand (0: K-major).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float lrelu(float z) { return z > 0.0f ? z : LRELU_SLOPE * z; }
__device__ __forceinline__ float lrelu_slope(float y) { return y > 0.0f ? 1.0f : LRELU_SLOPE; }

// --------------------------------------------------------------------------
// Convolution forward and data gradient: D[pixel][o] = sum_k A[pixel][k] B[o][k]
// with k = (tap, input channel), A gathered by TMA from the shifted input
// (zero fill outside the image), B the weight matrix.  A tile is 128 pixels
// (wt x ht of one image) by BN output channels.
//
// Persistent: each CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// Warp roles (6 warps): warp 0 lane 0 issues the TMA loads into a ring of
// stages, warp 1 owns the tensor memory and its lane 0 issues the MMAs, warps
// 2-5 run the epilogue, warp w reading tensor-memory lanes 32 (w % 4) ...
// 32 (w % 4) + 31.  Two accumulators in tensor memory alternate between tiles,
// so the epilogue of one tile overlaps the main loop of the next.
// --------------------------------------------------------------------------
enum { EPI_BIAS = 0, EPI_BIAS_LRELU = 1, EPI_SLOPE = 2, EPI_PLAIN = 3 };

struct ConvArgs {
    int n, h, w, cin, cout;
    int wt, ht, tiles_w, tiles_h, tiles;
    int kblocks, cblocks;
    int epi;
    const float *bias;          // EPI_BIAS*
    const bf16 *slope_src;      // EPI_SLOPE: y whose lrelu slope multiplies the result (NHWC, cout channels)
    void *out;                  // NHWC, out_cs channels per pixel
    int out_cs, n_store, out_f32;
    unsigned *status;
};

template <int BN>
struct ConvShape {
    static constexpr int A_BYTES = BM * ROW_BYTES;
    static constexpr int B_BYTES = BN * ROW_BYTES;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // BN = 64: three CTAs per SM with 3 stages of 24 KB each (measured 4 % faster
    // over the whole forward pass than two CTAs with 4 stages); BN = 128: two
    // CTAs per SM, 96 KB of stages each (their accumulators fill the 512
    // tensor-memory columns); BN = 256: one CTA per SM, 4 stages
    static constexpr int CTAS_PER_SM = BN >= 256 ? 1 : (BN == 64 ? 3 : 2);
    static constexpr int STAGES = BN >= 256 ? 4 : (BN == 64 ? 3 : ((96 * 1024 / STAGE) < 2 ? 2 : (96 * 1024 / STAGE)));
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM = STAGES * STAGE + 1024 /* alignment */ + BAR_BYTES + BN * 4 /* bias */;
    static constexpr int TMEM_COLS = 2 * BN;  // two FP32 accumulators
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    conv_fprop_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                      const ConvArgs a)
{
    using S = ConvShape<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + S::STAGES * S::STAGE);
    uint64_t *empty = full + S::STAGES;
    uint64_t *acc_full = empty + S::STAGES;  // [2]: the MMAs of a tile are done
    uint64_t *acc_empty = acc_full + 2;      // [2]: the epilogue has read the accumulator
    uint32_t *tmem_holder = (uint32_t *)(acc_empty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_holder + 1);
    float *sbias = (float *)(smem + S::STAGES * S::STAGE + S::BAR_BYTES);

    if (*(volatile unsigned *)a.status != 0u)
        return;  // an earlier launch failed: leave the output untouched

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.y * BN;
    const bool has_bias = a.epi == EPI_BIAS || a.epi == EPI_BIAS_LRELU;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S::STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp >= 2 && has_bias)
        for (int c = threadIdx.x - 64; c < BN; c += 128)
            sbias[c] = a.bias[n0 + c];
    if (warp == 1)
        tmem_alloc(tmem_holder, S::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0 && lane == 0) {
        // producer: the stage ring runs on across tiles
        uint32_t kc = 0;
        for (int tile = blockIdx.x; tile < a.tiles && !*abort_flag; tile += gridDim.x) {
            int t = tile;
            const int tw = t % a.tiles_w;
            t /= a.tiles_w;
            const int th = t % a.tiles_h;
            const int img = t / a.tiles_h;
            const int w0 = tw * a.wt, h0 = th * a.ht;
            for (int kb = 0; kb < a.kblocks; kb++, kc++) {
                const int s = kc % S::STAGES;
                const uint32_t use = kc / S::STAGES;
                if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, a.status)) {
                    atomicOr(a.status, ST_TIMEOUT_PRODUCER);
                    *abort_flag = 1;
                    break;
                }
                const int tap = kb / a.cblocks, cb = kb - tap * a.cblocks;
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                uint8_t *sa = smem + s * S::STAGE;
                mbar_expect_tx(&full[s], S::STAGE);
                tma_load_4d(sa, &map_x, &full[s], cb * KB, w0 + dx, h0 + dy, img);
                tma_load_2d(sa + S::A_BYTES, &map_w, &full[s], kb * KB, n0);
            }
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(BM, BN, 0, 0);
        uint32_t kc = 0;
        int it = 0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, it++) {
            const int acc = it & 1, use = it >> 1;
            if (*abort_flag || (use > 0 && !mbar_wait(&acc_empty[acc], (use - 1) & 1, a.status))) {
                atomicOr(a.status, ST_TIMEOUT_MMA);
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + (uint32_t)(acc * BN);
            bool ok = true;
            for (int kb = 0; kb < a.kblocks; kb++, kc++) {
                const int s = kc % S::STAGES;
                if (*abort_flag || !mbar_wait(&full[s], (kc / S::STAGES) & 1, a.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * S::STAGE);
                const uint32_t sb = sa + S::A_BYTES;
#pragma unroll
                for (int k = 0; k < KB / 16; k++) {
                    // K-major, 128-byte swizzle: rows 128 B apart, 8-row groups 1024 B
                    // apart; the k-th 16-element slice starts 32 B further in.
                    const uint64_t ad = sw128_desc(sa + 32 * k, 16, 1024);
                    const uint64_t bd = sw128_desc(sb + 32 * k, 16, 1024);
                    umma_bf16(dt, ad, bd, idesc, (kb | k) != 0);
                }
                umma_commit(&empty[s]);
            }
            if (!ok) {
                atomicOr(a.status, ST_TIMEOUT_MMA);
                *abort_flag = 1;
                break;
            }
            umma_commit(&acc_full[acc]);
        }
    } else if (warp >= 2) {
        const int q = warp & 3;
        const int r = 32 * q + lane;
        int it = 0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, it++) {
            const int acc = it & 1, use = it >> 1;
            // the tensor-memory loads are warp-collective: take the decision per warp
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], use & 1, a.status));
            if (!ok) {
                if (lane == 0)
                    atomicOr(a.status, ST_TIMEOUT_EPILOGUE);
                break;
            }
            tc_fence_after();
            int t = tile;
            const int tw = t % a.tiles_w;
            t /= a.tiles_w;
            const int th = t % a.tiles_h;
            const int img = t / a.tiles_h;
            const int px = tw * a.wt + r % a.wt, py = th * a.ht + r / a.wt;
            const bool valid = px < a.w && py < a.h;
            const long long pix = ((long long)img * a.h + py) * a.w + px;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + c0), v);
                const int oc = n0 + c0;
                if (!valid || oc >= a.n_store)
                    continue;
                if (has_bias) {
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const float z = v[i] + sbias[c0 + i];
                        v[i] = a.epi == EPI_BIAS_LRELU ? lrelu(z) : z;
                    }
                } else if (a.epi == EPI_SLOPE) {
                    const uint4 *ys = (const uint4 *)(a.slope_src + pix * a.cout + oc);
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        uint4 u = __ldg(&ys[j]);
                        const bf16 *yb = (const bf16 *)&u;
#pragma unroll
                        for (int e = 0; e < 8; e++)
                            v[8 * j + e] *= lrelu_slope(__bfloat162float(yb[e]));
                    }
                }
                const int nst = min(32, a.n_store - oc);
                if (a.out_f32) {
                    float *o = (float *)a.out + pix * a.out_cs + oc;
                    if (nst == 32 && (a.out_cs & 3) == 0) {
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            ((float4 *)o)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; i++)
                            if (i < nst)
                                o[i] = v[i];
                    }
                } else {
                    bf16 *o = (bf16 *)a.out + pix * a.out_cs + oc;
                    if (nst == 32 && (a.out_cs & 7) == 0) {
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            uint4 u;
                            __nv_bfloat162 *p2 = (__nv_bfloat162 *)&u;
#pragma unroll
                            for (int e = 0; e < 4; e++)
                                p2[e] = __floats2bfloat162_rn(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]);
                            ((uint4 *)o)[j] = u;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; i++)
                            if (i < nst)
                                o[i] = __float2bfloat16_rn(v[i]);
                    }
                }
            }
            // the accumulator is read: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&acc_empty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

// --------------------------------------------------------------------------
// Weight gradient of one tap: D[o][i] = sum_p dz[p][o] x[p + s_tap][i] over a
// range of 64-pixel K blocks.  Both operands are loaded from the NHWC tensors
// as they are, so they are MN-major (the 64 channels of one pixel form one
// 128-byte row, consecutive pixels are consecutive K).  M = 128 output
// channels (two 64-channel boxes; a missing second box stays zero), N = BN
// input channels (BN / 64 boxes).  Each CTA writes its FP32 partial sum; a
// second kernel adds the partials of all pixel ranges in a fixed order.
// --------------------------------------------------------------------------
struct WgradArgs {
    int n, h, w, cin, cout;
    int wt, ht, tiles_w, tiles_h;   // 64-pixel K blocks: wt x ht pixels of one image
    int kb_total, kb_per_split, splits;
    int mtiles, ntiles;
    float *partial;                 // [splits][cout][9 cin]
    unsigned *status;
};

template <int BN>
struct WgradShape {
    static constexpr int A_BYTES = 2 * SUB_BYTES;
    static constexpr int B_BYTES = (BN / 64) * SUB_BYTES;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = (96 * 1024 / STAGE) < 2 ? 2 : (96 * 1024 / STAGE);
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
};

template <int BN>
__global__ void __launch_bounds__(192, 1)
    conv_wgrad_kernel(const __grid_constant__ CUtensorMap map_dz, const __grid_constant__ CUtensorMap map_x,
                      const WgradArgs a)
{
    using S = WgradShape<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + S::STAGES * S::STAGE);
    uint64_t *empty = full + S::STAGES;
    uint64_t *done = empty + S::STAGES;
    uint32_t *tmem_holder = (uint32_t *)(done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_holder + 1);

    if (*(volatile unsigned *)a.status != 0u)
        return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int b = blockIdx.x;
    const int tap = b % 9;
    b /= 9;
    const int mt = b % a.mtiles;
    const int nt = b / a.mtiles;
    const int m0 = mt * BM, n0 = nt * BN;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int split = blockIdx.y;
    const int kb_lo = split * a.kb_per_split;
    const int kb_hi = min(a.kb_total, kb_lo + a.kb_per_split);
    const bool two_m = m0 + 64 < a.cout;       // second 64-channel box of A present

    if (!two_m) {
        // the second half of every A stage stays zero (no TMA writes it)
        for (int s = 0; s < S::STAGES; s++) {
            uint4 *z = (uint4 *)(smem + s * S::STAGE + SUB_BYTES);
            for (int i = threadIdx.x; i < SUB_BYTES / 16; i += blockDim.x)
                z[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        fence_proxy_async_smem();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S::STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1)
        tmem_alloc(tmem_holder, S::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const int nk = kb_hi - kb_lo;

    if (warp == 0 && lane == 0) {
        const uint32_t bytes = (two_m ? 2 : 1) * SUB_BYTES + S::B_BYTES;
        for (int j = 0; j < nk && !*abort_flag; j++) {
            const int s = j % S::STAGES, it = j / S::STAGES;
            if (j >= S::STAGES && !mbar_wait(&empty[s], (it - 1) & 1, a.status)) {
                atomicOr(a.status, ST_TIMEOUT_PRODUCER);
                *abort_flag = 1;
                break;
            }
            int kb = kb_lo + j;
            const int tw = kb % a.tiles_w;
            kb /= a.tiles_w;
            const int th = kb % a.tiles_h;
            const int img = kb / a.tiles_h;
            const int pw = tw * a.wt, ph = th * a.ht;
            uint8_t *st = smem + s * S::STAGE;
            mbar_expect_tx(&full[s], bytes);
            tma_load_4d(st, &map_dz, &full[s], m0, pw, ph, img);
            if (two_m)
                tma_load_4d(st + SUB_BYTES, &map_dz, &full[s], m0 + 64, pw, ph, img);
#pragma unroll
            for (int q = 0; q < BN / 64; q++)
                tma_load_4d(st + S::A_BYTES + q * SUB_BYTES, &map_x, &full[s], n0 + 64 * q, pw + dx, ph + dy, img);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(BM, BN, 1, 1);
        bool ok = true;
        for (int j = 0; j < nk; j++) {
            const int s = j % S::STAGES, it = j / S::STAGES;
            if (*abort_flag || !mbar_wait(&full[s], it & 1, a.status)) {
                atomicOr(a.status, ST_TIMEOUT_MMA);
                *abort_flag = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * S::STAGE);
            const uint32_t sb = sa + S::A_BYTES;
#pragma unroll
            for (int k = 0; k < KB / 16; k++) {
                // MN-major, 128-byte swizzle: 64 channels per 128-byte row, the
                // next 64 channels one box (8 KB) further (LBO); 8 pixel rows per
                // 1024-byte group (SBO); 16 pixels (2 KB) per MMA.
                const uint64_t ad = sw128_desc(sa + 2048 * k, SUB_BYTES, 1024);
                const uint64_t bd = sw128_desc(sb + 2048 * k, SUB_BYTES, 1024);
                umma_bf16(tmem, ad, bd, idesc, (j | k) != 0);
            }
            umma_commit(&empty[s]);
        }
        if (ok && nk > 0)
            umma_commit(done);
    } else if (warp >= 2) {
        const int q = warp & 3;
        const int o = m0 + 32 * q + lane;
        const int ldk = 9 * a.cin;
        float *dst = a.partial + ((long long)split * a.cout + o) * ldk + tap * a.cin + n0;
        if (nk == 0) {
            if (o < a.cout)
                for (int c = 0; c < BN; c++)
                    dst[c] = 0.0f;
        } else if (!__all_sync(0xffffffffu, mbar_wait(done, 0, a.status))) {
            if (lane == 0)
                atomicOr(a.status, ST_TIMEOUT_EPILOGUE);
        } else {
            tc_fence_after();
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                if (o < a.cout) {
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        ((float4 *)(dst + c0))[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

__device__ __forceinline__ void unpack8(uint4 u, float (&f)[8])
{
    const __nv_bfloat162 *p = (const __nv_bfloat162 *)&u;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        float2 t = __bfloat1622float2(p[e]);
        f[2 * e] = t.x;
        f[2 * e + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8])
{
    uint4 u;
    __nv_bfloat162 *p = (__nv_bfloat162 *)&u;
#pragma unroll
    for (int e = 0; e < 4; e++)
        p[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
    return u;
}

// dW[i] = sum over splits s (in order) of partial[s][i]
__global__ void sum_partials_kernel(const float *__restrict__ partial, int splits, long long count,
                                    float *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < splits; k++)
            s += partial[k * count + i];
        out[i] = s;
    }
}

// Bias gradient, first pass: block b adds dz (npix x c, bf16) over its pixel
// range [b * ppb, (b + 1) * ppb) per channel into partial[b][c].  Thread t reads
// 8 channels (16 bytes) of pixel p0 + t / (c / 8) + k * (256 / (c / 8)), so a
// warp's loads are contiguous; the threads of one channel group are then added
// in shared memory in a fixed order.
__global__ void __launch_bounds__(256) channel_sum_kernel(const bf16 *__restrict__ dz, long long npix, int c,
                                                          long long ppb, float *__restrict__ partial)
{
    __shared__ float red[256][9];
    const int groups = c / 8;                 // 16-byte channel groups (c <= 2048)
    const int lanes_per_pix = groups;
    const int pix_step = 256 / lanes_per_pix; // pixels per sweep of the block (>= 1)
    const int g = threadIdx.x % lanes_per_pix, r = threadIdx.x / lanes_per_pix;
    const long long p0 = (long long)blockIdx.x * ppb;
    const long long p1 = min(npix, p0 + ppb);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (r < pix_step) {
        for (long long p = p0 + r; p < p1; p += pix_step) {
            float f[8];
            unpack8(*(const uint4 *)(dz + p * c + 8 * g), f);
#pragma unroll
            for (int e = 0; e < 8; e++)
                acc[e] += f[e];
        }
    }
#pragma unroll
    for (int e = 0; e < 8; e++)
        red[threadIdx.x][e] = acc[e];
    __syncthreads();
    for (int ch = threadIdx.x; ch < c; ch += 256) {
        const int gg = ch / 8, e = ch % 8;
        float sum = 0.0f;
        for (int rr = 0; rr < pix_step; rr++)
            sum += red[rr * lanes_per_pix + gg][e];
        partial[(long long)blockIdx.x * c + ch] = sum;
    }
}

// --------------------------------------------------------------------------
// Elementwise kernels on NHWC bf16 tensors, 8 channels (16 bytes) per thread.
// --------------------------------------------------------------------------
// y[n][h][w] = mean of x[n][2h..2h+1][2w..2w+1]; x is n x 2ho x 2wo
__global__ void pool2_kernel(const bf16 *__restrict__ x, int n, int ho, int wo, int c, bf16 *__restrict__ y)
{
    const int cv = c / 8;
    const long long total = (long long)n * ho * wo * cv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % cv);
        long long p = i / cv;
        const int ww = (int)(p % wo);
        p /= wo;
        const int hh = (int)(p % ho);
        const int nn = (int)(p / ho);
        const int wi = 2 * wo;
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dxx = 0; dxx < 2; dxx++) {
                const long long q = (((long long)nn * 2 * ho + 2 * hh + dy) * wi + 2 * ww + dxx) * c + 8 * k;
                float f[8];
                unpack8(*(const uint4 *)(x + q), f);
#pragma unroll
                for (int e = 0; e < 8; e++)
                    s[e] += f[e];
            }
#pragma unroll
        for (int e = 0; e < 8; e++)
            s[e] *= 0.25f;
        *(uint4 *)(y + i * 8) = pack8(s);
    }
}

// u = up2(x) + skip; x is n x h/2 x w/2, skip and u n x h x w
__global__ void up_add_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ skip, int n, int h, int w, int c,
                              bf16 *__restrict__ u)
{
    const int cv = c / 8;
    const long long total = (long long)n * h * w * cv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % cv);
        long long p = i / cv;
        const int ww = (int)(p % w);
        p /= w;
        const int hh = (int)(p % h);
        const int nn = (int)(p / h);
        const long long q = (((long long)nn * (h / 2) + hh / 2) * (w / 2) + ww / 2) * c + 8 * k;
        float a[8], b[8];
        unpack8(*(const uint4 *)(x + q), a);
        unpack8(*(const uint4 *)(skip + i * 8), b);
#pragma unroll
        for (int e = 0; e < 8; e++)
            a[e] += b[e];
        *(uint4 *)(u + i * 8) = pack8(a);
    }
}

// Backward of u = up2(x) + skip followed by x = lrelu(.): dz[p] = slope(y[p]) *
// sum of du over the 2x2 block of p (y = x, the coarse activation)
__global__ void up_bwd_kernel(const bf16 *__restrict__ du, const bf16 *__restrict__ y, int n, int ho, int wo, int c,
                              bf16 *__restrict__ dz)
{
    const int cv = c / 8;
    const long long total = (long long)n * ho * wo * cv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % cv);
        long long p = i / cv;
        const int ww = (int)(p % wo);
        p /= wo;
        const int hh = (int)(p % ho);
        const int nn = (int)(p / ho);
        const int wi = 2 * wo;
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dxx = 0; dxx < 2; dxx++) {
                const long long q = (((long long)nn * 2 * ho + 2 * hh + dy) * wi + 2 * ww + dxx) * c + 8 * k;
                float f[8];
                unpack8(*(const uint4 *)(du + q), f);
#pragma unroll
                for (int e = 0; e < 8; e++)
                    s[e] += f[e];
            }
        float yy[8];
        unpack8(*(const uint4 *)(y + i * 8), yy);
#pragma unroll
        for (int e = 0; e < 8; e++)
            s[e] *= lrelu_slope(yy[e]);
        *(uint4 *)(dz + i * 8) = pack8(s);
    }
}

// Backward at an encoder output e that feeds both a skip addition (gradient
// du) and pooling (gradient dp, at half resolution), followed by e = lrelu(.):
// dz[p] = slope(e[p]) * (du[p] + dp[p / 2] / 4)
__global__ void pool_bwd_kernel(const bf16 *__restrict__ du, const bf16 *__restrict__ dp, const bf16 *__restrict__ e,
                                int n, int h, int w, int c, bf16 *__restrict__ dz)
{
    const int cv = c / 8;
    const long long total = (long long)n * h * w * cv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % cv);
        long long p = i / cv;
        const int ww = (int)(p % w);
        p /= w;
        const int hh = (int)(p % h);
        const int nn = (int)(p / h);
        const long long q = (((long long)nn * (h / 2) + hh / 2) * (w / 2) + ww / 2) * c + 8 * k;
        float a[8], b[8], ee[8];
        unpack8(*(const uint4 *)(du + i * 8), a);
        unpack8(*(const uint4 *)(dp + q), b);
        unpack8(*(const uint4 *)(e + i * 8), ee);
#pragma unroll
        for (int j = 0; j < 8; j++)
            a[j] = lrelu_slope(ee[j]) * (a[j] + 0.25f * b[j]);
        *(uint4 *)(dz + i * 8) = pack8(a);
    }
}

// Mean squared error over the first nf channels of out (FP32, out_cs per
// pixel) against target (FP32, nf per pixel).  dout (bf16, c per pixel) gets
// 2 (out - target) / count on those channels and 0 elsewhere; each block adds
// its squared errors in FP64 into partial[block].
__global__ void mse_kernel(const float *__restrict__ out, int out_cs, const float *__restrict__ target, int nf,
                           long long npix, int c, double inv_count, bf16 *__restrict__ dout,
                           double *__restrict__ partial)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        for (int ch = 0; ch < c; ch += 8) {
            float g[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int k = ch + e;
                if (k < nf) {
                    const float d = out[p * out_cs + k] - target[p * nf + k];
                    acc += (double)d * (double)d;
                    g[e] = (float)(2.0 * inv_count) * d;
                } else {
                    g[e] = 0.0f;
                }
            }
            *(uint4 *)(dout + p * c + ch) = pack8(g);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        partial[blockIdx.x] = red[0];
}

// Adam (Kingma and Ba, Algorithm 1) on FP32 master parameters; omb1 = 1 - beta1,
// omb2 = 1 - beta2, c1 = 1 - beta1^t, c2 = 1 - beta2^t, all rounded from FP64 on
// the host so that omb1 / c1 = omb2 / c2 = 1 exactly at t = 1.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long count, float lr, float beta1, float beta2, float omb1,
                            float omb2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + omb1 * gi;
        const float vi = beta2 * v[i] + omb2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bf16 copies of one layer's FP32 weights W[o][t][i]: the forward matrix
// (same layout) and the data-gradient matrix Wd[i][t][o] = W[o][8 - t][i].
__global__ void weights_to_bf16_kernel(const float *__restrict__ w, int cout, int cin, bf16 *__restrict__ wf,
                                       bf16 *__restrict__ wd)
{
    const long long total = (long long)cout * 9 * cin;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % cin);
        const int t = (int)((idx / cin) % 9);
        const int o = (int)(idx / (9LL * cin));
        const bf16 b = __float2bfloat16_rn(w[idx]);
        wf[idx] = b;
        wd[((long long)i * 9 + (8 - t)) * cout + o] = b;
    }
}

}  // namespace cnok
