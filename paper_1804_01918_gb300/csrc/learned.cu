// learned.cu -- learned collide: an MLP trained on the GPU to replace the plain collide, with an
// exact projection onto the conserved moments and a per-tile fallback to the plain collide.
//
// Training data are (pre, post) pairs of FP32 deviations produced by the plain collide of this
// library (pairs_kernel). The network (mlp_core.cuh) predicts the normalised collision change
// (post - pre); its forward and backward passes run as tcgen05 BF16 x BF16 -> FP32 products with
// hand-written epilogues (bias, GELU, GELU derivative, loss gradient), one 128-sample tile per CTA
// and batch, and Adam updates FP32 master weights and re-packs the BF16 operand images; a training
// run takes one cooperative launch per epoch (mlp_train_kernel<true>).
//
// The learned LB step (step_learned_kernel) is persistent over 32 x 32-site tiles: per tile it
// pulls the populations, runs the MLP on 8 sub-tiles of 128 sites, adds the predicted change,
// projects onto the exact post-collision moments, stores, and on check steps also evaluates the
// plain collide of the same sites: if max |f_learned - f_plain| exceeds bound x max |f_plain| over
// the tile, the plain result (kept in a scratch tile) is copied over the tile, which stays on the
// plain collide until the next check.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lb_learned.h"
#include "d2q37_gpu.cuh"
#include "kernels.cuh"
#include "mlp_core.cuh"
#include "site_fp32dev.cuh"

using namespace lbg;
using namespace lbg::mlp;

namespace lbg {
namespace learn {

constexpr uint64_t WAIT_LIMIT = tc::WAIT_LIMIT_NS;  // bounded mbarrier waits (time)
constexpr int ERR_TIMEOUT = 8;             // status-word bit: a tensor-core wait gave up

// Device view of a network: FP32 master parameters (for biases), BF16 operand images of the
// weights, normalisation (mu_x, sd_x, mu_t, sd_t; 37 each).
struct NetDev {
    const float* params;
    const char* w1img;   // [128][48]
    const char* w2img;   // [128][128]
    const char* w3img;   // [48][128]
    const char* w3timg;  // [128][48]
    const char* w2timg;  // [128][128]
    const float* norm;   // [4][37]
};

struct LearnedStats {
    unsigned long long checked, fallback;
    unsigned int max_res_bits;  // non-negative float as bits (atomicMax)
    unsigned int pad;
};

// ------------------------------------------------------------------------------------------------
// training pairs: pre = pulled deviations, post = plain (exact-split) collide of them
// ------------------------------------------------------------------------------------------------
__global__ void pairs_kernel(const float* __restrict__ src, const StepParams P, const int* __restrict__ sites,
                             int n, float* __restrict__ pre, float* __restrict__ post, int* __restrict__ flag) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int site = sites[k];
    if (site < 0 || site >= P.Lx * P.Ly) {
        atomicOr(flag, 1);
        return;
    }
    const int y = site / P.Lx, x = site - y * P.Lx;
    float d[NPOP];
    Pull32<NPOP - 1>::run(src, d, x, y, P.Lx, P.Ly, P.y_periodic, P.plane);
#pragma unroll
    for (int i = 0; i < NPOP; ++i) pre[(size_t)k * NPOP + i] = d[i];
    SplitPre s;
    split_pre(d, P, s, flag);
    split_collide(d, P, P, s);
    split_project(d, P, P, s);
#pragma unroll
    for (int i = 0; i < NPOP; ++i) post[(size_t)k * NPOP + i] = d[i];
}

// Per-population sums (FP64) of pre and of post - pre for the normalisation statistics, as
// per-block partials part[block][4][37] (sum x, sum x^2, sum t, sum t^2) that the host adds in
// block order. Each block reduces its threads' sums with a fixed tree, so the result does not
// depend on scheduling.
constexpr int STATS_THREADS = 256;
__global__ void __launch_bounds__(STATS_THREADS)
stats_kernel(const float* __restrict__ pre, const float* __restrict__ post, long long n,
             double* __restrict__ part) {
    __shared__ double red[STATS_THREADS];
    double lx[NIN], lx2[NIN], lt[NIN], lt2[NIN];
    for (int i = 0; i < NIN; ++i) lx[i] = lx2[i] = lt[i] = lt2[i] = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        for (int i = 0; i < NIN; ++i) {
            const double a = pre[r * NIN + i], t = (double)post[r * NIN + i] - (double)pre[r * NIN + i];
            lx[i] += a;
            lx2[i] += a * a;
            lt[i] += t;
            lt2[i] += t * t;
        }
    for (int k = 0; k < 4 * NIN; ++k) {
        const int i = k % NIN, q = k / NIN;
        red[threadIdx.x] = q == 0 ? lx[i] : q == 1 ? lx2[i] : q == 2 ? lt[i] : lt2[i];
        __syncthreads();
        for (int w = STATS_THREADS / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * 4 * NIN + k] = red[0];
        __syncthreads();
    }
}

// Column sums over a warp: on return lane L holds the sum over the warp's 32 lanes of their v[L]
// (v is overwritten). Butterfly transpose-reduce: at the stage of width s, lanes with bit s set
// keep the upper half of their columns and exchange the lower half, so 31 shuffles suffice.
__device__ __forceinline__ float warp_column_sums(float* v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int k = 0; k < s; ++k) {
            const float send = upper ? v[k] : v[k + s];
            const float keep = upper ? v[k + s] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// ------------------------------------------------------------------------------------------------
// shared-memory plan of the training kernel
// ------------------------------------------------------------------------------------------------
constexpr int TR_X = 0;
constexpr int TR_H1 = TR_X + BYTES_X;      // H1, later dZ1
constexpr int TR_H2 = TR_H1 + BYTES_H;     // H2, later dZ2
constexpr int TR_DY = TR_H2 + BYTES_H;
constexpr int TR_W1 = TR_DY + BYTES_DY;
constexpr int TR_W2 = TR_W1 + BYTES_W1;
constexpr int TR_W3 = TR_W2 + BYTES_W2;
constexpr int TR_W3T = TR_W3 + BYTES_W3;
constexpr int TR_W2T = TR_W3T + BYTES_W3T;
constexpr int TR_GBN = HID + HID + NOUTP;  // bias-gradient columns db1[128] db2[128] db3[48]
constexpr int TR_WARPS = 8;                 // two warpgroups: each epilogue's columns split in halves
constexpr int TR_GB = TR_W2T + BYTES_W2T;  // per-warp column sums [8][TR_GBN], added in warp order
constexpr int TR_BIAS = TR_GB + TR_WARPS * TR_GBN * 4;  // b1[128] b2[128] b3[48] of this batch
constexpr int TR_MISC = TR_BIAS + TR_GBN * 4;
constexpr int TR_BYTES = TR_MISC + 64;

// Parameter p: the sum of the per-tile gradient partials, then (apply) an Adam step on the FP32
// master parameter and its BF16 entries in the operand images. The arithmetic is written with
// explicit roundings, so that it is the same wherever it is inlined.
__device__ __forceinline__ void adam_param(int p, float* __restrict__ params, float* __restrict__ m,
                                           float* __restrict__ vv, const float* partial, int nparts, float lr,
                                           float bc1, float bc2, int apply, float* __restrict__ grad_out,
                                           char* __restrict__ w1img, char* __restrict__ w2img,
                                           char* __restrict__ w3img, char* __restrict__ w3timg,
                                           char* __restrict__ w2timg) {
    // (from L2: in a training loop the partials were written by other CTAs of the same launch)
    float g = 0.0f;
    for (int c = 0; c < nparts; ++c) g += __ldcg(partial + (size_t)c * PART_STRIDE + p);
    if (grad_out) grad_out[p] = g;
    if (!apply) return;
    const float b1c = 0.9f, b2c = 0.999f;
    const float mm = __fmaf_rn(b1c, m[p], __fmul_rn(1.0f - b1c, g));
    const float vn = __fmaf_rn(b2c, vv[p], __fmul_rn(__fmul_rn(1.0f - b2c, g), g));
    m[p] = mm;
    vv[p] = vn;
    const float step = __fdiv_rn(__fdiv_rn(mm, bc1), __fadd_rn(__fsqrt_rn(__fdiv_rn(vn, bc2)), 1e-8f));
    const float w = __fsub_rn(params[p], __fmul_rn(lr, step));
    params[p] = w;
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    if (p < OFF_B1) {
        const int o = (p - OFF_W1) / NIN, i = (p - OFF_W1) % NIN;
        *reinterpret_cast<__nv_bfloat16*>(w1img + elem_off(o, i, KIN)) = wb;
    } else if (p >= OFF_W2 && p < OFF_B2) {
        const int o = (p - OFF_W2) / HID, i = (p - OFF_W2) % HID;
        *reinterpret_cast<__nv_bfloat16*>(w2img + elem_off(o, i, HID)) = wb;
        *reinterpret_cast<__nv_bfloat16*>(w2timg + elem_off(i, o, HID)) = wb;
    } else if (p >= OFF_W3 && p < OFF_B3) {
        const int j = (p - OFF_W3) / HID, h = (p - OFF_W3) % HID;
        *reinterpret_cast<__nv_bfloat16*>(w3img + elem_off(j, h, HID)) = wb;
        *reinterpret_cast<__nv_bfloat16*>(w3timg + elem_off(h, j, NOUTP)) = wb;
    }
}

// One epoch's training data in permutation order, ready for mlp_train_kernel (raw = 2): sample p
// (p < count) is pair perm[p], normalised -- x = (pre - mu_x) / sd_x, t = (post - pre - mu_t) /
// sd_t, the same arithmetic as the kernel's raw = 1 gather -- with x written as row p mod 128 of
// tile p / 128's BF16 X image (the shared-memory operand layout, so the kernel copies it in one
// bulk copy) and t as t[tile][i][p mod 128]. One thread per sample, all SMs: the random rows of
// pre and post are gathered with the whole GPU's memory parallelism instead of 32 SMs'.
__global__ void prep_epoch_kernel(const float* __restrict__ pre, const float* __restrict__ post,
                                  const int* __restrict__ perm, long long count, const float* __restrict__ norm,
                                  char* __restrict__ ximg, float* __restrict__ timg) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const long long row = perm[p], tile = p / TILE;
    const int r = (int)(p % TILE);
    float xn[KIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        const float av = pre[row * NIN + i], bv = post[row * NIN + i];
        xn[i] = (av - norm[i]) / norm[NIN + i];
        timg[(tile * NIN + i) * TILE + r] = ((bv - av) - norm[2 * NIN + i]) / norm[3 * NIN + i];
    }
#pragma unroll
    for (int i = NIN; i < KIN; ++i) xn[i] = 0.0f;
#pragma unroll
    for (int k0 = 0; k0 < KIN; k0 += 8) store_row8(ximg + tile * BYTES_X, r, k0, KIN, xn + k0);
}

// A bounded barrier of all CTAs of a cooperative launch (bar[0] counts arrivals, bar[1] is the
// generation): false if it was not reached by all within the wait limit.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* shared_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
        __threadfence();  // this CTA's writes before its arrival
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1u) : "memory");
        } else {
            const uint64_t t0 = tc::globaltimer_ns();
            for (;;) {
                unsigned g;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
                if (g != gen) break;
                if (tc::globaltimer_ns() - t0 > WAIT_LIMIT) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *shared_ok = ok;
    }
    __syncthreads();
    return *shared_ok != 0;
}

// Per-batch arguments of an in-kernel training loop (kLoop): the batches' Adam bias corrections
// (bc[2 b], bc[2 b + 1]), the master parameters and moments, the operand images and the grid
// barrier's two words.
struct TrainLoop {
    const float* bc;
    float* params;
    float* m;
    float* v;
    char* img[5];
    float lr;
    unsigned* bar;
    int tiles;  // the batch's tiles: CTAs 0 .. tiles - 1 take one each, the rest join the Adam step
};

// One 128-sample tile per CTA and batch: forward, loss, backward; writes this CTA's
// parameter-gradient partial (packed like the parameters) and adds its loss sum to *loss_acc. Two
// warpgroups: thread q of either owns sample q (TMEM lane q); each epilogue's 128 columns are
// split between them (columns 64 wg .. 64 wg + 63), and the per-sample work (inputs, loss) is
// warpgroup 0's. kLoop: a cooperative launch of one CTA per SM that trains on nbatch consecutive
// batches of the permutation: CTAs 0 .. L.tiles - 1 take a tile each; after each batch a grid
// barrier, the Adam step with the parameters spread over all CTAs' threads, a second barrier, and
// the next batch reloads the weights and biases. Otherwise one batch (nbatch = 1, one CTA per
// tile) whose Adam step is a separate kernel.
//   raw = 1: a = pre deviations, b = post deviations (normalised inside);
//   raw = 0: a = normalised inputs, b = normalised targets;
//   raw = 2: a = the tiles' X images, b = their normalised targets, as prep_epoch_kernel writes
//            them for the permutation's sample order (perm unused).
template <bool kLoop>
__global__ void __launch_bounds__(2 * TILE, 1)
mlp_train_kernel(NetDev net, const float* __restrict__ a, const float* __restrict__ b,
                 const int* __restrict__ perm, long long base, int nbatch, float inv_count, int raw,
                 float* __restrict__ partial, double* __restrict__ loss_acc, int* __restrict__ flag, TrainLoop L) {
    extern __shared__ __align__(1024) char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, q = tid & (TILE - 1), wg = tid >> 7, c0 = 64 * wg;
    float* gb = reinterpret_cast<float*>(sm + TR_GB);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TR_MISC);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + TR_MISC + 8);
    int* shared_ok = reinterpret_cast<int*>(sm + TR_MISC + 12);
    float* loss_sm = reinterpret_cast<float*>(sm + TR_MISC + 16);
    uint64_t* wbar = reinterpret_cast<uint64_t*>(sm + TR_MISC + 24);
    float* bias = reinterpret_cast<float*>(sm + TR_BIAS);
    float* gbw = gb + warp * TR_GBN;  // this warp's slots: each written once per tile, no atomics
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(wbar, 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;
    uint32_t ph = 0;
    bool ok = true, weights_ok = true;
    const int tiles = kLoop ? L.tiles : (int)gridDim.x;
    const int batch = tiles * TILE;
    const bool worker = (int)blockIdx.x < tiles;
    for (int bi = 0; bi < nbatch && ok; ++bi) {
    if (worker) {
    const long long tile0 = base + (long long)bi * batch + (long long)blockIdx.x * TILE;
    if (tid == 0) {
        // the five weight images (100 KB) by bulk copies, arriving on wbar while the threads
        // gather and normalise their samples (a copy loop of 16-byte loads per thread waited for
        // the L2 round trip ~50 times); in a training loop they were just rewritten by the
        // previous batch's Adam step (generic stores): the proxy fence orders those before the
        // asynchronous copy's reads
        if (kLoop) asm volatile("fence.proxy.async.global;" ::: "memory");
        tc::mbar_expect_tx(wbar, BYTES_W1 + BYTES_W2 + BYTES_W3 + BYTES_W3T + BYTES_W2T + (raw == 2 ? BYTES_X : 0));
        if (raw == 2)  // the tile's prepared X image
            tc::bulk_g2s(sm + TR_X, reinterpret_cast<const char*>(a) + (tile0 / TILE) * BYTES_X, BYTES_X, wbar);
        tc::bulk_g2s(sm + TR_W1, net.w1img, BYTES_W1, wbar);
        tc::bulk_g2s(sm + TR_W2, net.w2img, BYTES_W2, wbar);
        tc::bulk_g2s(sm + TR_W3, net.w3img, BYTES_W3, wbar);
        tc::bulk_g2s(sm + TR_W3T, net.w3timg, BYTES_W3T, wbar);
        tc::bulk_g2s(sm + TR_W2T, net.w2timg, BYTES_W2T, wbar);
        *loss_sm = 0.0f;
    }
    for (int k = tid; k < TR_WARPS * TR_GBN; k += blockDim.x) gb[k] = 0.0f;
    // this batch's biases (from L2: in a training loop another CTA's Adam step may have just
    // rewritten them)
    for (int k = tid; k < 2 * HID + NOUT; k += blockDim.x) {
        const int off = k < HID ? OFF_B1 + k : k < 2 * HID ? OFF_B2 + (k - HID) : OFF_B3 + (k - 2 * HID);
        bias[k] = __ldcg(net.params + off);
    }

    // ---- this thread's sample ----
    float xn[KIN], tn[NIN];
    if (raw == 2) {
        // prepared by prep_epoch_kernel: the X image arrives with the weights, the normalised
        // targets are [tile][37][128]
        if (wg == 0)
#pragma unroll
            for (int i = 0; i < NIN; ++i) tn[i] = b[((tile0 / TILE) * NIN + i) * TILE + q];
    } else if (wg == 0) {
        const long long row = perm ? (long long)perm[tile0 + q] : tile0 + q;
        const float* norm = net.norm;
#pragma unroll
        for (int i = 0; i < NIN; ++i) {
            const float av = a[row * NIN + i], bv = b[row * NIN + i];
            if (raw) {
                xn[i] = (av - norm[i]) / norm[NIN + i];
                tn[i] = ((bv - av) - norm[2 * NIN + i]) / norm[3 * NIN + i];
            } else {
                xn[i] = av;
                tn[i] = bv;
            }
        }
#pragma unroll
        for (int i = NIN; i < KIN; ++i) xn[i] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < KIN; k0 += 8) store_row8(sm + TR_X, q, k0, KIN, xn + k0);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // the weights have arrived (the products read them)
    ok = !__syncthreads_or(!tc::mbar_wait_bounded(wbar, (uint32_t)(bi & 1), WAIT_LIMIT));
    weights_ok = ok;

    auto issue_and_wait = [&](int which) {
        if (tid == 0) {
            switch (which) {
                case 0: mma_kmajor(tm + 0, sm + TR_X, sm + TR_W1, KIN, HID); break;
                case 1: mma_kmajor(tm + 128, sm + TR_H1, sm + TR_W2, HID, HID); break;
                case 2: mma_kmajor(tm + 256, sm + TR_H2, sm + TR_W3, HID, NOUTP); break;
                case 3:
                    mma_kmajor(tm + 384, sm + TR_DY, sm + TR_W3T, NOUTP, HID);        // dH2
                    mma_mnmajor(tm + 304, sm + TR_H2, HID, sm + TR_DY, NOUTP, NOUTP);  // dW3^T
                    break;
                case 4:
                    mma_kmajor(tm + 384, sm + TR_H2, sm + TR_W2T, HID, HID);          // dH1 (H2 buf = dZ2)
                    mma_mnmajor(tm + 256, sm + TR_H2, HID, sm + TR_H1, HID, HID);      // dW2
                    break;
                case 5: mma_mnmajor(tm + 128, sm + TR_H1, HID, sm + TR_X, KIN, NOUTP); break;  // dW1 (H1 buf = dZ1)
            }
            tc::mma_commit(bar);
        }
        const bool got = tc::mbar_wait_bounded(bar, ph, WAIT_LIMIT);
        ph ^= 1u;
        if (__syncthreads_or(!got)) {
            ok = false;
            return;
        }
        tc::fence_after_sync();
    };
    auto sync_for_mma = [&]() {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };

    const float* b1 = bias;
    const float* b2 = bias + HID;
    const float* b3 = bias + 2 * HID;
    float v[32];
    do {
        if (!ok) break;
        // ---- forward ----
        issue_and_wait(0);
        if (!ok) break;
        for (int c = c0; c < c0 + 64; c += 32) {
            tc::tmem_ld32(tmem_lane_addr(tm, warp, c), v);
#pragma unroll
            for (int j = 0; j < 32; j += 2) gelu_bias2(v[j], v[j + 1], b1[c + j], b1[c + j + 1]);
#pragma unroll
            for (int j = 0; j < 32; j += 8) store_row8(sm + TR_H1, q, c + j, HID, v + j);
        }
        sync_for_mma();
        issue_and_wait(1);
        if (!ok) break;
        for (int c = c0; c < c0 + 64; c += 32) {
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 128 + c), v);
#pragma unroll
            for (int j = 0; j < 32; j += 2) gelu_bias2(v[j], v[j + 1], b2[c + j], b2[c + j + 1]);
#pragma unroll
            for (int j = 0; j < 32; j += 8) store_row8(sm + TR_H2, q, c + j, HID, v + j);
        }
        sync_for_mma();
        issue_and_wait(2);
        if (!ok) break;
        // ---- output, loss and its gradient ----
        if (wg == 0) {
            float yv[NOUTP];
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 256), yv);
            tc::tmem_ld16(tmem_lane_addr(tm, warp, 288), yv + 32);
            float dy[NOUTP], lsum = 0.0f;
#pragma unroll
            for (int j = 0; j < NOUTP; ++j) {
                if (j < NOUT) {
                    const float e = (yv[j] + b3[j]) - tn[j];
                    lsum += e * e;
                    dy[j] = 2.0f * e * inv_count;
                } else {
                    dy[j] = 0.0f;
                }
            }
#pragma unroll
            for (int j = 0; j < NOUTP; j += 8) store_row8(sm + TR_DY, q, j, NOUTP, dy + j);
            // db3: warp column sums, then one shared atomic per column and warp
            float cs[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) cs[j] = dy[j];
            gbw[2 * HID + (tid & 31)] = warp_column_sums(cs);
#pragma unroll
            for (int j = 0; j < 32; ++j) cs[j] = j < NOUTP - 32 ? dy[32 + j] : 0.0f;
            const float c2 = warp_column_sums(cs);
            if ((tid & 31) < NOUTP - 32) gbw[2 * HID + 32 + (tid & 31)] = c2;
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if ((tid & 31) == 0) atomicAdd(loss_sm, lsum);
        }
        sync_for_mma();
        issue_and_wait(3);
        if (!ok) break;
        // ---- dZ2 = dH2 * gelu'(z2) into the H2 buffer; dW3^T partial ----
        for (int c = c0; c < c0 + 64; c += 32) {
            float z[32];
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 384 + c), v);
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 128 + c), z);
#pragma unroll
            for (int j = 0; j < 32; j += 2) gelu_grad_bias2(v[j], v[j + 1], z[j], z[j + 1], b2[c + j], b2[c + j + 1]);
#pragma unroll
            for (int j = 0; j < 32; j += 8) store_row8(sm + TR_H2, q, c + j, HID, v + j);
            gbw[HID + c + (tid & 31)] = warp_column_sums(v);
        }
        if (wg == 1) {
            float g[NOUTP];
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 304), g);
            tc::tmem_ld16(tmem_lane_addr(tm, warp, 336), g + 32);
            float* out = partial + (size_t)blockIdx.x * PART_STRIDE + OFF_W3;
#pragma unroll
            for (int j = 0; j < NOUT; ++j) out[j * HID + q] = g[j];  // dW3[j][h], h = this lane
        }
        sync_for_mma();
        issue_and_wait(4);
        if (!ok) break;
        // ---- dZ1 = dH1 * gelu'(z1) into the H1 buffer; dW2 partial ----
        for (int c = c0; c < c0 + 64; c += 32) {
            float z[32];
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 384 + c), v);
            tc::tmem_ld32(tmem_lane_addr(tm, warp, c), z);
#pragma unroll
            for (int j = 0; j < 32; j += 2) gelu_grad_bias2(v[j], v[j + 1], z[j], z[j + 1], b1[c + j], b1[c + j + 1]);
#pragma unroll
            for (int j = 0; j < 32; j += 8) store_row8(sm + TR_H1, q, c + j, HID, v + j);
            gbw[c + (tid & 31)] = warp_column_sums(v);
        }
        {
            float* out = partial + (size_t)blockIdx.x * PART_STRIDE + OFF_W2 + (size_t)q * HID;  // row o
            for (int c = c0; c < c0 + 64; c += 32) {
                tc::tmem_ld32(tmem_lane_addr(tm, warp, 256 + c), v);
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4*>(out + c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
        }
        sync_for_mma();
        issue_and_wait(5);
        if (!ok) break;
        if (wg == 0) {
            float g[NOUTP];
            tc::tmem_ld32(tmem_lane_addr(tm, warp, 128), g);
            tc::tmem_ld16(tmem_lane_addr(tm, warp, 160), g + 32);
            float* out = partial + (size_t)blockIdx.x * PART_STRIDE + OFF_W1 + (size_t)q * NIN;  // row o
#pragma unroll
            for (int i = 0; i < NIN; ++i) out[i] = g[i];
        }
    } while (0);

    __syncthreads();
    if (ok) {
        float* out = partial + (size_t)blockIdx.x * PART_STRIDE;
        auto col = [&](int k) {  // the warps' column sums (zero where a warp has none), in warp order
            float a = gb[k];
#pragma unroll
            for (int w = 1; w < TR_WARPS; ++w) a += gb[w * TR_GBN + k];
            return a;
        };
        for (int k = tid; k < HID; k += blockDim.x) {
            out[OFF_B1 + k] = col(k);
            out[OFF_B2 + k] = col(HID + k);
        }
        for (int k = tid; k < NOUT; k += blockDim.x) out[OFF_B3 + k] = col(2 * HID + k);
        if (tid == 0) atomicAdd(loss_acc, (double)*loss_sm);
    }
    }  // worker
    if (kLoop && ok) {
        // all partials written -> the Adam step, the parameters spread over the grid's threads ->
        // the new weights written before any CTA reloads them
        ok = grid_barrier(L.bar, shared_ok);
        if (ok) {
            const float* bcb = L.bc + 2 * bi;
            for (int p = blockIdx.x * blockDim.x + tid; p < NPARAM; p += gridDim.x * blockDim.x)
                adam_param(p, L.params, L.m, L.v, partial, tiles, L.lr, bcb[0], bcb[1], 1, nullptr, L.img[0],
                           L.img[1], L.img[2], L.img[3], L.img[4]);
            asm volatile("fence.proxy.async.global;" ::: "memory");
            ok = grid_barrier(L.bar, shared_ok);
        }
    }
    }  // batches
    if (!ok && tid == 0) atomicOr(flag, ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    // TMEM must be released before the block exits; the barrier is invalidated only when no
    // product can still be pending on it (a wait that gave up leaves it alone)
    if (warp == 0) tc::tmem_dealloc(tm, 512);
    if (tid == 0 && ok) tc::mbar_inval(bar);
    if (tid == 0 && weights_ok) tc::mbar_inval(wbar);
}

// One thread per parameter (the training batches launched one by one).
__global__ void adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ vv,
                            const float* __restrict__ partial, int nparts, float lr, float bc1, float bc2,
                            int apply, float* __restrict__ grad_out, char* __restrict__ w1img,
                            char* __restrict__ w2img, char* __restrict__ w3img, char* __restrict__ w3timg,
                            char* __restrict__ w2timg) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM)
        adam_param(p, params, m, vv, partial, nparts, lr, bc1, bc2, apply, grad_out, w1img, w2img, w3img,
                   w3timg, w2timg);
}

// ------------------------------------------------------------------------------------------------
// forward only (evaluation and the learned step)
// ------------------------------------------------------------------------------------------------
constexpr int FW_X = 0;
constexpr int FW_H = FW_X + BYTES_X;
constexpr int FW_W1 = FW_H + BYTES_H;
constexpr int FW_W2 = FW_W1 + BYTES_W1;
constexpr int FW_W3 = FW_W2 + BYTES_W2;
constexpr int FW_RED = FW_W3 + BYTES_W3;   // block reductions (2 x 4 floats)
constexpr int FW_MISC = FW_RED + 64;
// per-CTA copies of the biases and of the normalisation (input standard deviations as reciprocals)
constexpr int FC_B1 = 0, FC_B2 = FC_B1 + HID, FC_B3 = FC_B2 + HID, FC_MUX = FC_B3 + NOUTP,
              FC_ISDX = FC_MUX + NOUTP, FC_MUT = FC_ISDX + NOUTP, FC_SDT = FC_MUT + NOUTP,
              FC_FLOATS = FC_SDT + NOUTP;
constexpr int FW_CONST = FW_MISC + 64;
constexpr int FW_BYTES = FW_CONST + FC_FLOATS * 4;

struct FwdCtx {
    char* sm;
    const float* cst;  // FC_* constants in shared memory
    uint64_t* bar;
    uint32_t tm;
    uint32_t ph;
    int tid, warp;
};

// Network output (normalised, 37 values) of the inputs this thread stored as row tid of the X
// image (all threads call it together). Returns false if a tensor-core wait gave up.
__device__ __forceinline__ bool mlp_forward_tile(FwdCtx& f, const NetDev& net, float* y) {
    const float* b1 = f.cst + FC_B1;
    const float* b2 = f.cst + FC_B2;
    const float* b3 = f.cst + FC_B3;
    float v[32];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    for (int layer = 0; layer < 3; ++layer) {
        if (f.tid == 0) {
            if (layer == 0) mma_kmajor(f.tm + 0, f.sm + FW_X, f.sm + FW_W1, KIN, HID);
            if (layer == 1) mma_kmajor(f.tm + 128, f.sm + FW_H, f.sm + FW_W2, HID, HID);
            if (layer == 2) mma_kmajor(f.tm + 0, f.sm + FW_H, f.sm + FW_W3, HID, NOUTP);
            tc::mma_commit(f.bar);
        }
        const bool got = tc::mbar_wait_bounded(f.bar, f.ph, WAIT_LIMIT);
        f.ph ^= 1u;
        if (__syncthreads_or(!got)) return false;
        tc::fence_after_sync();
        if (layer < 2) {
            const float* bias = layer == 0 ? b1 : b2;
            for (int c = 0; c < HID; c += 32) {
                tc::tmem_ld32(tmem_lane_addr(f.tm, f.warp, (layer == 0 ? 0 : 128) + c), v);
#pragma unroll
                for (int j = 0; j < 32; j += 2) gelu_bias2(v[j], v[j + 1], bias[c + j], bias[c + j + 1]);
#pragma unroll
                for (int j = 0; j < 32; j += 8) store_row8(f.sm + FW_H, f.tid, c + j, HID, v + j);
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        } else {
            float yv[NOUTP];
            tc::tmem_ld32(tmem_lane_addr(f.tm, f.warp, 0), yv);
            tc::tmem_ld16(tmem_lane_addr(f.tm, f.warp, 32), yv + 32);
#pragma unroll
            for (int j = 0; j < NOUT; ++j) y[j] = yv[j] + b3[j];
            tc::fence_before_sync();
            __syncthreads();  // TMEM columns 0.. are free for the next tile's first layer
            tc::fence_after_sync();
        }
    }
    return true;
}

__device__ __forceinline__ void fwd_setup(FwdCtx& f, const NetDev& net, char* sm) {
    f.sm = sm;
    f.tid = threadIdx.x;
    f.warp = threadIdx.x >> 5;
    f.bar = reinterpret_cast<uint64_t*>(sm + FW_MISC);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + FW_MISC + 8);
    copy_to_smem(sm + FW_W1, net.w1img, BYTES_W1);
    copy_to_smem(sm + FW_W2, net.w2img, BYTES_W2);
    copy_to_smem(sm + FW_W3, net.w3img, BYTES_W3);
    float* cst = reinterpret_cast<float*>(sm + FW_CONST);
    for (int k = f.tid; k < HID; k += blockDim.x) {
        cst[FC_B1 + k] = net.params[OFF_B1 + k];
        cst[FC_B2 + k] = net.params[OFF_B2 + k];
    }
    for (int k = f.tid; k < NOUT; k += blockDim.x) {
        cst[FC_B3 + k] = net.params[OFF_B3 + k];
        cst[FC_MUX + k] = net.norm[k];
        cst[FC_ISDX + k] = 1.0f / net.norm[NIN + k];
        cst[FC_MUT + k] = net.norm[2 * NIN + k];
        cst[FC_SDT + k] = net.norm[3 * NIN + k];
    }
    f.cst = cst;
    if (f.tid == 0) tc::mbar_init(f.bar, 1);
    if (f.warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    f.tm = *tslot;
    f.ph = 0;
}

// ok = false after a wait that gave up: the barrier is then left alone, since a product may still
// be pending on it (TMEM must be released before the block exits either way).
__device__ __forceinline__ void fwd_teardown(FwdCtx& f, bool ok = true) {
    tc::fence_before_sync();
    __syncthreads();
    if (f.warp == 0) tc::tmem_dealloc(f.tm, 256);
    if (f.tid == 0 && ok) tc::mbar_inval(f.bar);
}

// y[n][37] = network(x[n][37]) on normalised inputs; n a multiple of 128; persistent over tiles.
__global__ void __launch_bounds__(128)
mlp_eval_kernel(NetDev net, const float* __restrict__ x, float* __restrict__ y, int ntiles, int* __restrict__ flag) {
    extern __shared__ __align__(1024) char sm[];
    FwdCtx f;
    fwd_setup(f, net, sm);
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long row = (long long)t * TILE + f.tid;
        float xn[KIN];
#pragma unroll
        for (int i = 0; i < NIN; ++i) xn[i] = x[row * NIN + i];
#pragma unroll
        for (int i = NIN; i < KIN; ++i) xn[i] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < KIN; k0 += 8) store_row8(sm + FW_X, f.tid, k0, KIN, xn + k0);
        float out[NOUT];
        if (!mlp_forward_tile(f, net, out)) {
            if (f.tid == 0) atomicOr(flag, ERR_TIMEOUT);
            ok = false;
            break;
        }
#pragma unroll
        for (int j = 0; j < NOUT; ++j) y[row * NOUT + j] = out[j];
    }
    fwd_teardown(f, ok);
}

// ---- the learned LB step ----------------------------------------------------------------------
// One CTA per SM with three independent groups of four warps (a warpgroup each), persistent over
// 32 x 32-site tiles: a group takes a whole tile and steps it in eight sub-tiles of 128 sites (four
// rows of 32, one site per thread): pull, exact-split sums, the network (three tcgen05 products
// issued by one thread of the group, bias + GELU epilogues from the group's 128 TMEM columns into
// its H image), the change added and projected onto the exact moments, stored. On check steps the
// group evaluates the plain collide of the same sites while its first product runs, for the tile
// residual and, in the group's scratch tile, for a fallback, which copies it over the stored tile.
// While one group waits for the tensor cores the other two keep the SM busy. Per group in shared
// memory: the H image (whose first 12 KB hold the X image until the first product has read it) and
// the pulled deviations (staged there during the network, so that a thread holds few registers);
// the BF16 weights are shared by the groups. TMEM: layer 1's accumulator at the group's columns
// 0..127, layer 2's at the same columns once the first epilogue has read them, the output at
// 0..47; the plain result waits for the residual in 37 of the spare columns 384..511. Waits on the
// tensor cores are bounded in time; only named barriers of the group synchronise it.
namespace ws {
constexpr int GROUPS = 3;
constexpr int THREADS = GROUPS * TILE;
constexpr int SLOT_D = NPOP * TILE * 4;     // [37][128] floats
constexpr int SCRATCH_TILE = NPOP * 1024;   // floats: a tile's plain result, [37][32 rows][32]
constexpr int COPY_V4 = NPOP * 32 * 8;      // 16-byte pieces of a tile
constexpr uint64_t START_STAGGER_NS = 5000;  // group g starts g x this late
// TMEM: the groups' networks at columns 0..383, their plain results (37 columns) from 384 on
constexpr int PLAIN_COL = GROUPS * 128, PLAIN_STRIDE = 40;
static_assert(PLAIN_COL + (GROUPS - 1) * PLAIN_STRIDE + NPOP <= 512, "TMEM columns");
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + BYTES_W1;
constexpr int OFF_W3 = OFF_W2 + BYTES_W2;
constexpr int OFF_H = OFF_W3 + BYTES_W3;    // per group
constexpr int OFF_D = OFF_H + GROUPS * BYTES_H;
constexpr int OFF_C = OFF_D + GROUPS * SLOT_D;
constexpr int OFF_RED = OFF_C + FC_FLOATS * 4;  // 8 floats per group
constexpr int OFF_BAR = OFF_RED + GROUPS * 32;
constexpr int OFF_TSLOT = OFF_BAR + GROUPS * 8;
constexpr int BYTES = OFF_TSLOT + 16;
static_assert(BYTES <= 232448, "the learned step needs one SM's shared memory");
static_assert(BYTES_X <= BYTES_H, "the X image lives in the H image");
static_assert(OFF_H % 128 == 0 && BYTES_H % 128 == 0 && OFF_D % 16 == 0 && OFF_BAR % 8 == 0, "alignment");

struct Group {
    char* sm;
    const float* cst;
    char* H;
    float* D;
    float* red;
    uint64_t* bar;
    uint32_t tm;  // the group's TMEM columns (lane 0)
    uint32_t tp;  // this warp's lanes at the group's plain-result columns
    uint32_t ph;  // phase of the group's barrier
    int q, wq, id;
};

// An empty asm the compiler must assume changes the fields of s (no instruction is emitted).
__device__ __forceinline__ void opaque(SplitPre& s) {
    asm volatile("" : "+r"(s.p.n0), "+r"(s.p.nx), "+r"(s.p.ny), "+r"(s.p.ne), "+f"(s.p.r0), "+f"(s.p.rx),
                 "+f"(s.p.ry), "+f"(s.p.re), "+f"(s.s0), "+f"(s.rho), "+f"(s.ux), "+f"(s.uy), "+f"(s.T));
}

// The first product of a sub-tile whose inputs the group has written as the X image: the group
// synchronises and one thread issues it (the threads may work on before mlp_finish).
__device__ __forceinline__ void mlp_begin(Group& g) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    tc::wg_sync(g.id);
    if (g.q == 0) {
        tc::fence_after_sync();
        mma_kmajor(g.tm, g.H, g.sm + OFF_W1, KIN, HID);
        tc::mma_commit(g.bar);
    }
}

// The rest of the network for the sub-tile: the two epilogues and products that follow, and the
// network's output (without b3) for this thread's site in y. False if a wait gave up (the whole
// group then returns false).
__device__ __forceinline__ bool mlp_finish(Group& g, float* y) {
    const float* b1 = g.cst + FC_B1;
    const float* b2 = g.cst + FC_B2;
    float v[32];
    for (int layer = 0; layer < 3; ++layer) {
        const bool ok = tc::mbar_wait_bounded(g.bar, g.ph, WAIT_LIMIT);
        g.ph ^= 1u;
        if (tc::wg_any(g.id, !ok)) return false;
        tc::fence_after_sync();
        if (layer < 2) {
            const float* bias = layer == 0 ? b1 : b2;
            for (int cc = 0; cc < HID; cc += 32) {
                tc::tmem_ld32(tmem_lane_addr(g.tm, g.wq, cc), v);
#pragma unroll
                for (int j = 0; j < 32; j += 2) gelu_bias2(v[j], v[j + 1], bias[cc + j], bias[cc + j + 1]);
#pragma unroll
                for (int j = 0; j < 32; j += 8) store_row8(g.H, g.q, cc + j, HID, v + j);
            }
            tc::fence_async_smem();
        } else {
            tc::tmem_ld32(tmem_lane_addr(g.tm, g.wq, 0), y);
            tc::tmem_ld16(tmem_lane_addr(g.tm, g.wq, 32), y + 32);
        }
        // the group's TMEM columns (and H, for the next sub-tile's X) are free for the next product
        tc::fence_before_sync();
        tc::wg_sync(g.id);
        if (layer < 2 && g.q == 0) {
            tc::fence_after_sync();
            mma_kmajor(g.tm, g.H, g.sm + (layer == 0 ? OFF_W2 : OFF_W3), HID, layer == 0 ? HID : NOUTP);
            tc::mma_commit(g.bar);
        }
    }
    return true;
}

// The plain result of a tile that falls back, from the group's scratch tile over the stored one.
__device__ __forceinline__ void copy_tile(const float* scr, float* __restrict__ dst, const StepParams& P, int x0,
                                          int y0, int q) {
    constexpr int BATCH = 4;
    for (int u0 = 0; u0 < COPY_V4; u0 += TILE * BATCH) {
        float4 v4[BATCH];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int u = u0 + b * TILE + q;
            if (u < COPY_V4) v4[b] = reinterpret_cast<const float4*>(scr)[u];
        }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int u = u0 + b * TILE + q;
            if (u < COPY_V4) {
                // piece u: population u / 256, row (u / 8) mod 32, 16-byte column u mod 8
                const int j = u >> 8, row = (u >> 3) & 31, c4 = u & 7;
                char* base = reinterpret_cast<char*>(dst + (long long)(y0 + row + HALO) * P.Lx + x0);
                reinterpret_cast<float4*>(base + P.plane_b32[j])[c4] = v4[b];
            }
        }
    }
}

// One learned tile stepped by group g. False if a wait gave up.
__device__ __forceinline__ bool learned_tile(Group& g, const float* __restrict__ src, float* __restrict__ dst,
                                             const StepParams& P, int t, int x0, int y0, int check, float bound,
                                             float* scr, unsigned char* __restrict__ tile_mode,
                                             LearnedStats* __restrict__ stats, int* flag) {
    const int q = g.q;
    const float* mu_x = g.cst + FC_MUX;
    const float* isd_x = g.cst + FC_ISDX;
    const float* b3 = g.cst + FC_B3;
    const float* mu_t = g.cst + FC_MUT;
    const float* sd_t = g.cst + FC_SDT;
    float rmax = 0.0f, fmax = 0.0f;
    for (int sub = 0; sub < 8; ++sub) {
        const int x = x0 + (q & 31), yy = 4 * sub + (q >> 5);
        SplitPre sp;
        {
            float d[NPOP];
            pull32(src, d, P, x, y0 + yy);
            split_pre(d, P, sp, flag);
            float xn[KIN];
#pragma unroll
            for (int j = 0; j < NIN; ++j) {
                g.D[j * TILE + q] = d[j];
                xn[j] = (d[j] - mu_x[j]) * isd_x[j];
            }
#pragma unroll
            for (int j = NIN; j < KIN; ++j) xn[j] = 0.0f;
#pragma unroll
            for (int k0 = 0; k0 < KIN; k0 += 8) store_row8(g.H, q, k0, KIN, xn + k0);
            mlp_begin(g);
            if (check) {
                // while the first product runs: the plain result of the same sites (the plain
                // step's arithmetic in the plain step's order), for the residual (parked in the
                // group's spare TMEM columns) and, in the scratch tile, for a fallback
                split_collide(d, P, P, sp);
                split_project(d, P, P, sp);
                const int o = yy * 32 + (q & 31);
#pragma unroll
                for (int j = 0; j < NPOP; ++j) {
                    scr[j * 1024 + o] = d[j];
                    fmax = fmaxf(fmax, fabsf((float)shell_w(shell_of(j)) + d[j]));
                }
                tc::tmem_st32(g.tp, d);
                tc::tmem_st4(g.tp + 32u, d + 32);
                tc::tmem_st1(g.tp + 36u, d[36]);
            }
        }
        // no product of the plain projection above may be shared with the projection below (a
        // shared product is not fused into an FMA, a private one may be, as in the plain step):
        // the site fields pass an empty asm that the compiler must treat as changing them
        opaque(sp);
        float yv[NOUTP];
        if (!mlp_finish(g, yv)) return false;
        float dl[NPOP];
#pragma unroll
        for (int j = 0; j < NPOP; ++j) dl[j] = g.D[j * TILE + q] + fmaf(yv[j] + b3[j], sd_t[j], mu_t[j]);
        split_project(dl, P, P, sp);
        if (check) {
            float pl[NPOP];
            tc::tmem_wait_st();
            tc::tmem_ld32(g.tp, pl);
            tc::tmem_ld4(g.tp + 32u, pl + 32);
            pl[36] = tc::tmem_ld1(g.tp + 36u);
#pragma unroll
            for (int j = 0; j < NPOP; ++j) rmax = fmaxf(rmax, fabsf(dl[j] - pl[j]));
        }
        split_store(dst, P, x, y0 + yy, dl, sp, flag);
    }
    if (!check) return true;
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
    }
    if ((q & 31) == 0) {
        g.red[g.wq] = rmax;
        g.red[4 + g.wq] = fmax;
    }
    tc::wg_sync(g.id);  // also orders the group's stores above before the fallback copy below
    const float R = fmaxf(fmaxf(g.red[0], g.red[1]), fmaxf(g.red[2], g.red[3]));
    const float F = fmaxf(fmaxf(g.red[4], g.red[5]), fmaxf(g.red[6], g.red[7]));
    tc::wg_sync(g.id);  // red is reused by the next tile
    const float res = F > 0.0f ? R / F : R;
    const int fall = !(res <= bound);
    if (q == 0) {
        tile_mode[t] = (unsigned char)fall;
        atomicAdd(&stats->checked, 1ull);
        if (fall) atomicAdd(&stats->fallback, 1ull);
        atomicMax(&stats->max_res_bits, __float_as_uint(res));
    }
    if (fall) {
        copy_tile(scr, dst, P, x0, y0, q);
        tc::wg_sync(g.id);  // the scratch tile is rewritten by the group's next tile
    }
    return true;
}

}  // namespace ws

// The learned LB step (see the file header and above). Lx and Ly are multiples of 32; scratch
// holds one tile per group.
__global__ void __launch_bounds__(ws::THREADS, 1)
step_learned_kernel(const float* __restrict__ src, float* __restrict__ dst, const StepParams P, NetDev net,
                    unsigned char* __restrict__ tile_mode, int check, float bound,
                    LearnedStats* __restrict__ stats, float* scratch, int* __restrict__ flag) {
    using namespace ws;
    extern __shared__ __align__(1024) char sm[];
    const int tid = threadIdx.x, gi = tid >> 7;
    copy_to_smem(sm + OFF_W1, net.w1img, BYTES_W1);
    copy_to_smem(sm + OFF_W2, net.w2img, BYTES_W2);
    copy_to_smem(sm + OFF_W3, net.w3img, BYTES_W3);
    float* cst = reinterpret_cast<float*>(sm + OFF_C);
    for (int k = tid; k < HID; k += THREADS) {
        cst[FC_B1 + k] = net.params[OFF_B1 + k];
        cst[FC_B2 + k] = net.params[OFF_B2 + k];
    }
    for (int k = tid; k < NOUT; k += THREADS) {
        cst[FC_B3 + k] = net.params[OFF_B3 + k];
        cst[FC_MUX + k] = net.norm[k];
        cst[FC_ISDX + k] = 1.0f / net.norm[NIN + k];
        cst[FC_MUT + k] = net.norm[2 * NIN + k];
        cst[FC_SDT + k] = net.norm[3 * NIN + k];
    }
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_TSLOT);
    if (tid < GROUPS) tc::mbar_init(bars + tid, 1);
    if (tid < 32) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    Group g;
    g.sm = sm;
    g.cst = cst;
    g.H = sm + OFF_H + gi * BYTES_H;
    g.D = reinterpret_cast<float*>(sm + OFF_D + gi * SLOT_D);
    g.red = reinterpret_cast<float*>(sm + OFF_RED) + 8 * gi;
    g.bar = bars + gi;
    g.tm = *tslot + 128u * (uint32_t)gi;
    g.tp = tmem_lane_addr(*tslot, (tid >> 5) & 3, PLAIN_COL + PLAIN_STRIDE * gi);
    g.ph = 0;
    g.q = tid & 127;
    g.wq = (tid >> 5) & 3;
    g.id = 1 + gi;
    float* scr = scratch + ((size_t)blockIdx.x * GROUPS + gi) * SCRATCH_TILE;
    // Stagger the groups' start by about a third of a sub-tile's ~13 us each: groups that start
    // together keep epilogues and product waits in step and leave the SM idle together (measured
    // +2.7 %, flat between 4 and 7 us); the delay costs ~10 us of a group's time per launch.
    if (gi > 0) {
        const uint64_t t0 = tc::globaltimer_ns();
        while (tc::globaltimer_ns() - t0 < (uint64_t)gi * START_STAGGER_NS) __nanosleep(256);
    }
    const int ntx = P.Lx / 32, ntiles = ntx * (P.Ly / 32);
    bool alive = true;
    for (int t = blockIdx.x * GROUPS + gi; t < ntiles && alive; t += gridDim.x * GROUPS) {
        const int x0 = (t % ntx) * 32, y0 = (t / ntx) * 32;
        if (!check && tile_mode[t]) {
            for (int sub = 0; sub < 8; ++sub)
                fp32split_site(src, dst, P, P, x0 + (g.q & 31), y0 + 4 * sub + (g.q >> 5), flag);
            continue;
        }
        alive = learned_tile(g, src, dst, P, t, x0, y0, check, bound, scr, tile_mode, stats, flag);
    }
    if (!alive && g.q == 0) atomicOr(flag, ERR_TIMEOUT);
    tc::fence_before_sync();
    const bool gave_up = __syncthreads_or(!alive);
    if (tid < 32) tc::tmem_dealloc(*tslot, 512);
    if (tid < GROUPS && !gave_up) tc::mbar_inval(bars + tid);
}

// ---- FP32 debug mode of the loss and gradient ------------------------------------------------
// The same network, loss and gradient as the tensor-core training kernel, in plain FP32 on the CUDA
// cores without BF16 rounding: GELU from the library erff/expf, one block of HID threads per sample
// (thread j owns hidden unit j; output unit j < NOUT), activations in shared memory, gradients
// accumulated over the samples in FP64 (atomics) so that only the per-sample FP32 arithmetic
// rounds. Slow by design: a tight check of the host logic (packing, normalisation, loss scaling)
// and of the backward formulas against an FP64 reference.
__device__ __forceinline__ float gelu_ref(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_ref(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__global__ void __launch_bounds__(HID)
mlp_loss_grad_fp32_kernel(const float* __restrict__ p, const float* __restrict__ x, const float* __restrict__ t,
                          int n, double* __restrict__ g, double* __restrict__ loss) {
    __shared__ float xs[NIN], h1[HID], h2[HID], dy[NOUT], dz2[HID];
    const float* W1 = p + OFF_W1;
    const float* b1 = p + OFF_B1;
    const float* W2 = p + OFF_W2;
    const float* b2 = p + OFF_B2;
    const float* W3 = p + OFF_W3;
    const float* b3 = p + OFF_B3;
    const int j = threadIdx.x;
    const double scale = 2.0 / ((double)n * NOUT);
    for (int smp = blockIdx.x; smp < n; smp += gridDim.x) {
        if (j < NIN) xs[j] = x[(size_t)smp * NIN + j];
        __syncthreads();
        float z1 = b1[j];
        for (int k = 0; k < NIN; ++k) z1 = fmaf(W1[j * NIN + k], xs[k], z1);
        h1[j] = gelu_ref(z1);
        __syncthreads();
        float z2 = b2[j];
        for (int k = 0; k < HID; ++k) z2 = fmaf(W2[j * HID + k], h1[k], z2);
        h2[j] = gelu_ref(z2);
        __syncthreads();
        if (j < NOUT) {
            float y = b3[j];
            for (int k = 0; k < HID; ++k) y = fmaf(W3[j * HID + k], h2[k], y);
            const float e = y - t[(size_t)smp * NOUT + j];
            atomicAdd(loss, (double)e * (double)e);
            dy[j] = (float)(scale * e);
        }
        __syncthreads();
        // output layer: dW3[i][k] = dy_i h2_k (thread j owns column k = j), db3
        for (int i = 0; i < NOUT; ++i) atomicAdd(&g[OFF_W3 + i * HID + j], (double)dy[i] * h2[j]);
        if (j < NOUT) atomicAdd(&g[OFF_B3 + j], (double)dy[j]);
        float dh2 = 0.0f;
        for (int i = 0; i < NOUT; ++i) dh2 = fmaf(W3[i * HID + j], dy[i], dh2);
        const float d2 = dh2 * gelu_grad_ref(z2);
        dz2[j] = d2;
        __syncthreads();
        for (int i = 0; i < HID; ++i) atomicAdd(&g[OFF_W2 + i * HID + j], (double)dz2[i] * h1[j]);
        atomicAdd(&g[OFF_B2 + j], (double)d2);
        float dh1 = 0.0f;
        for (int i = 0; i < HID; ++i) dh1 = fmaf(W2[i * HID + j], dz2[i], dh1);
        const float d1 = dh1 * gelu_grad_ref(z1);
        for (int k = 0; k < NIN; ++k) atomicAdd(&g[OFF_W1 + j * NIN + k], (double)d1 * xs[k]);
        atomicAdd(&g[OFF_B1 + j], (double)d1);
        __syncthreads();  // xs, h1, h2, dy, dz2 are reused by the next sample
    }
}

__global__ void doubles_to_floats(const double* __restrict__ a, float* __restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

}  // namespace learn
}  // namespace lbg

using namespace lbg::learn;

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
struct lb_mlp {
    char* mem = nullptr;  // one device allocation
    float* params = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* norm = nullptr;
    char* img[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    long long adam_steps = 0;
    NetDev dev() const {
        NetDev n;
        n.params = params;
        n.w1img = img[0];
        n.w2img = img[1];
        n.w3img = img[2];
        n.w3timg = img[3];
        n.w2timg = img[4];
        n.norm = norm;
        return n;
    }
};

namespace {

lb_status fail_l(cudaError_t e, const char* where) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", where, cudaGetErrorString(e));
    set_last_error(msg);
    return LB_ERR_CUDA;
}

#define L_CUDA(call)                                   \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return fail_l(e_, #call); \
    } while (0)

constexpr size_t IMG_BYTES[5] = {BYTES_W1, BYTES_W2, BYTES_W3, BYTES_W3T, BYTES_W2T};

// SplitMix64 (Steele, Lea & Flood 2014): counter-based 64-bit generator.
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

// Pack host FP32 parameters into the BF16 operand images (host copies, then one upload).
void pack_images(const std::vector<float>& p, std::vector<std::vector<uint16_t>>& img) {
    auto bf = [](float x) {
        // round to nearest even on the bit pattern (finite inputs)
        uint32_t u;
        std::memcpy(&u, &x, 4);
        const uint32_t lsb = (u >> 16) & 1u;
        u += 0x7FFFu + lsb;
        return (uint16_t)(u >> 16);
    };
    for (int k = 0; k < 5; ++k) img[k].assign(IMG_BYTES[k] / 2, 0);
    for (int o = 0; o < HID; ++o)
        for (int i = 0; i < NIN; ++i) img[0][elem_off(o, i, KIN) / 2] = bf(p[OFF_W1 + o * NIN + i]);
    for (int o = 0; o < HID; ++o)
        for (int i = 0; i < HID; ++i) {
            img[1][elem_off(o, i, HID) / 2] = bf(p[OFF_W2 + o * HID + i]);
            img[4][elem_off(i, o, HID) / 2] = bf(p[OFF_W2 + o * HID + i]);
        }
    for (int j = 0; j < NOUT; ++j)
        for (int h = 0; h < HID; ++h) {
            img[2][elem_off(j, h, HID) / 2] = bf(p[OFF_W3 + j * HID + h]);
            img[3][elem_off(h, j, NOUTP) / 2] = bf(p[OFF_W3 + j * HID + h]);
        }
}

lb_status upload_params(lb_mlp* net, const float* params, const float* norm, cudaStream_t s) {
    std::vector<float> p(params, params + NPARAM);
    std::vector<std::vector<uint16_t>> img(5);
    pack_images(p, img);
    L_CUDA(cudaMemcpyAsync(net->params, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s));
    if (norm) L_CUDA(cudaMemcpyAsync(net->norm, norm, 4 * NIN * sizeof(float), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < 5; ++k)
        L_CUDA(cudaMemcpyAsync(net->img[k], img[k].data(), IMG_BYTES[k], cudaMemcpyHostToDevice, s));
    L_CUDA(cudaMemsetAsync(net->m, 0, NPARAM * sizeof(float), s));
    L_CUDA(cudaMemsetAsync(net->v, 0, NPARAM * sizeof(float), s));
    L_CUDA(cudaStreamSynchronize(s));
    net->adam_steps = 0;
    return LB_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return std::max(1, n);
}

// The kernels' dynamic shared-memory limits, raised once per device (the attribute is per device).
lb_status set_smem_limits() {
    constexpr int MAXDEV = 64;
    static std::atomic<bool> done[MAXDEV];
    int dev = 0;
    L_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < MAXDEV && done[dev].load()) return LB_OK;
    L_CUDA(cudaFuncSetAttribute(mlp_train_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_BYTES));
    L_CUDA(cudaFuncSetAttribute(mlp_train_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_BYTES));
    L_CUDA(cudaFuncSetAttribute(mlp_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_BYTES));
    L_CUDA(cudaFuncSetAttribute(step_learned_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ws::BYTES));
    if (dev >= 0 && dev < MAXDEV) done[dev].store(true);
    return LB_OK;
}

// Run the training kernel on `ntiles` tiles (rows from perm or contiguous) and reduce gradients;
// apply = take an Adam step. Device scratch: partial [ntiles][NPARAM], loss accumulator, flag.
lb_status train_batch(lb_mlp* net, const float* a, const float* b, const int* perm, long long base,
                      int ntiles, int raw, float lr, int apply, float* partial, double* loss_acc,
                      int* flag, float* grad_out, cudaStream_t s) {
    const float inv_count = 1.0f / ((float)ntiles * TILE * NOUT);
    mlp_train_kernel<false><<<ntiles, 2 * TILE, TR_BYTES, s>>>(net->dev(), a, b, perm, base, 1, inv_count, raw,
                                                               partial, loss_acc, flag, TrainLoop{});
    L_CUDA(cudaGetLastError());
    float bc1 = 1.0f, bc2 = 1.0f;
    if (apply) {
        net->adam_steps += 1;
        bc1 = 1.0f - std::pow(0.9f, (float)net->adam_steps);
        bc2 = 1.0f - std::pow(0.999f, (float)net->adam_steps);
    }
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(net->params, net->m, net->v, partial, ntiles, lr, bc1,
                                                     bc2, apply, grad_out, net->img[0], net->img[1], net->img[2],
                                                     net->img[3], net->img[4]);
    L_CUDA(cudaGetLastError());
    return LB_OK;
}

// The training loop's CTAs that can be resident at once (0 without cooperative launches).
int train_loop_ctas() {
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_train_kernel<true>, 2 * TILE, TR_BYTES) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sm_count();
}

// Whether ntiles training CTAs can all be resident at once (the cooperative launch's condition).
bool train_loop_fits(int ntiles) { return train_loop_ctas() >= ntiles; }

// All batches of one epoch in one cooperative launch (mlp_train_kernel<true>) on the data that
// prep_epoch_kernel laid out (raw = 2: a = X images, b = targets); bc holds the batches' Adam bias
// corrections, gbar two words for the grid barrier (zeroed here).
lb_status train_epoch_loop(lb_mlp* net, const float* a, const float* b, int nbatch, int ntiles, float lr,
                           const float* bc, float* partial, double* loss_acc, int* flag, unsigned* gbar,
                           cudaStream_t s) {
    L_CUDA(cudaMemsetAsync(gbar, 0, 2 * sizeof(unsigned), s));
    NetDev nd = net->dev();
    long long base = 0;
    const int* perm = nullptr;
    int raw = 2;
    float inv_count = 1.0f / ((float)ntiles * TILE * NOUT);
    TrainLoop L{bc, net->params, net->m, net->v, {net->img[0], net->img[1], net->img[2], net->img[3], net->img[4]},
                lr, gbar, ntiles};
    // every SM takes part: the batch's tiles on ntiles of them, the Adam step on all
    const int grid = std::max(ntiles, train_loop_ctas());
    void* args[] = {&nd, (void*)&a, (void*)&b, (void*)&perm, &base, &nbatch, &inv_count, &raw, &partial,
                    &loss_acc, &flag, &L};
    L_CUDA(cudaLaunchCooperativeKernel((const void*)mlp_train_kernel<true>, dim3(grid), dim3(2 * TILE), args,
                                       (size_t)TR_BYTES, s));
    net->adam_steps += nbatch;
    return LB_OK;
}


struct Scratch {
    char* mem = nullptr;
    float* partial = nullptr;
    double* loss = nullptr;
    int* flag = nullptr;
    float* grad = nullptr;
    ~Scratch() {
        if (mem) cudaFree(mem);
    }
    lb_status alloc(int ntiles) {
        const size_t pb = ((size_t)ntiles * PART_STRIDE * sizeof(float) + 255) / 256 * 256;
        const size_t gb = ((size_t)NPARAM * sizeof(float) + 255) / 256 * 256;
        cudaError_t e = cudaMalloc((void**)&mem, pb + gb + 256);
        if (e != cudaSuccess) {
            cudaGetLastError();
            mem = nullptr;
            set_last_error("MLP training scratch allocation failed");
            return LB_ERR_ALLOC;
        }
        partial = (float*)mem;
        grad = (float*)(mem + pb);
        loss = (double*)(mem + pb + gb);
        flag = (int*)(mem + pb + gb + 64);
        return LB_OK;
    }
};

lb_status check_flag(int* dflag, cudaStream_t s) {
    int h = 0;
    L_CUDA(cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    L_CUDA(cudaStreamSynchronize(s));
    if (h & ERR_TIMEOUT) {
        set_last_error("a tensor-core completion wait gave up (MLP kernel)");
        return LB_ERR_CUDA;
    }
    if (h & 2) return LB_ERR_RANGE;
    if (h) return LB_ERR_NONFINITE;
    return LB_OK;
}

}  // namespace

// Host and device permutation buffers of a training run (two of each) and its per-epoch loss sums.
struct TrainBuffers {
    int* hperm[2] = {nullptr, nullptr};
    int* dperm[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    double* loss = nullptr;
    float* bc = nullptr;       // Adam bias corrections of every batch of the run (training loop)
    unsigned* gbar = nullptr;  // grid barrier words (training loop)
    char* ximg = nullptr;      // an epoch's X images and targets in batch order (training loop)
    float* timg = nullptr;
    ~TrainBuffers() {
        for (int b = 0; b < 2; ++b) {
            if (hperm[b]) cudaFreeHost(hperm[b]);
            if (dperm[b]) cudaFree(dperm[b]);
            if (copied[b]) cudaEventDestroy(copied[b]);
        }
        if (loss) cudaFree(loss);
        if (bc) cudaFree(bc);
        if (gbar) cudaFree(gbar);
        if (ximg) cudaFree(ximg);
        if (timg) cudaFree(timg);
    }
    // the training loop's prepared data: count samples (a multiple of 128)
    lb_status alloc_prepared(long long count) {
        if (cudaMalloc((void**)&ximg, (size_t)(count / TILE) * BYTES_X) != cudaSuccess ||
            cudaMalloc((void**)&timg, (size_t)count * NIN * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("MLP training buffers allocation failed");
            return LB_ERR_ALLOC;
        }
        return LB_OK;
    }
    lb_status alloc(long long n, int epochs, long long nbatches) {
        for (int b = 0; b < 2; ++b) {
            cudaError_t e = cudaMallocHost((void**)&hperm[b], (size_t)n * sizeof(int));
            if (e == cudaSuccess) e = cudaMalloc((void**)&dperm[b], (size_t)n * sizeof(int));
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_last_error("MLP training buffers allocation failed");
                return LB_ERR_ALLOC;
            }
        }
        if (cudaMalloc((void**)&loss, (size_t)epochs * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&bc, (size_t)nbatches * 2 * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&gbar, 2 * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("MLP training buffers allocation failed");
            return LB_ERR_ALLOC;
        }
        return LB_OK;
    }
};

extern "C" {

lb_status lb_mlp_create(uint64_t seed, lb_mlp** out) {
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    lb_mlp* net = new (std::nothrow) lb_mlp();
    if (!net) return LB_ERR_ALLOC;
    size_t total = 3 * ((NPARAM * sizeof(float) + 255) / 256 * 256) + 1024;
    for (int k = 0; k < 5; ++k) total += IMG_BYTES[k];
    cudaError_t e = cudaMalloc((void**)&net->mem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete net;
        set_last_error("MLP allocation failed");
        return LB_ERR_ALLOC;
    }
    char* p = net->mem;
    const size_t pbytes = (NPARAM * sizeof(float) + 255) / 256 * 256;
    net->params = (float*)p;
    p += pbytes;
    net->m = (float*)p;
    p += pbytes;
    net->v = (float*)p;
    p += pbytes;
    net->norm = (float*)p;
    p += 1024;
    for (int k = 0; k < 5; ++k) {
        net->img[k] = p;
        p += IMG_BYTES[k];
    }
    // PyTorch-style default initialisation: weights and biases uniform in +-1/sqrt(fan_in)
    std::vector<float> w(NPARAM);
    uint64_t s = seed ^ 0x5D3F2A1B9C8E7F60ull;
    auto fill = [&](int off, int count, int fan_in) {
        const double a = 1.0 / std::sqrt((double)fan_in);
        for (int k = 0; k < count; ++k) w[off + k] = (float)((2.0 * uniform01(s) - 1.0) * a);
    };
    fill(OFF_W1, HID * NIN, NIN);
    fill(OFF_B1, HID, NIN);
    fill(OFF_W2, HID * HID, HID);
    fill(OFF_B2, HID, HID);
    fill(OFF_W3, NOUT * HID, HID);
    fill(OFF_B3, NOUT, HID);
    std::vector<float> norm(4 * NIN, 0.0f);
    for (int i = 0; i < NIN; ++i) norm[NIN + i] = norm[3 * NIN + i] = 1.0f;
    lb_status st = set_smem_limits();
    if (st == LB_OK) st = upload_params(net, w.data(), norm.data(), 0);
    if (st != LB_OK) {
        lb_mlp_free(net);
        return st;
    }
    *out = net;
    return LB_OK;
}

void lb_mlp_free(lb_mlp* net) {
    if (!net) return;
    cudaDeviceSynchronize();
    if (net->mem) cudaFree(net->mem);
    delete net;
}

lb_status lb_mlp_get_params(const lb_mlp* net, float* params, float* norm) {
    if (!net) return LB_ERR_ARG;
    if (params) L_CUDA(cudaMemcpy(params, net->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (norm) L_CUDA(cudaMemcpy(norm, net->norm, 4 * NIN * sizeof(float), cudaMemcpyDeviceToHost));
    return LB_OK;
}

lb_status lb_mlp_set_params(lb_mlp* net, const float* params, const float* norm) {
    if (!net || !params) return LB_ERR_ARG;
    return upload_params(net, params, norm, 0);
}

lb_status lb_mlp_eval(lb_mlp* net, const float* x, float* y, int n, void* stream) {
    if (!net || !x || !y || n <= 0 || n % TILE) return LB_ERR_ARG;
    lb_status st = set_smem_limits();
    if (st != LB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc;
    st = sc.alloc(1);
    if (st != LB_OK) return st;
    L_CUDA(cudaMemsetAsync(sc.flag, 0, sizeof(int), s));
    const int ntiles = n / TILE;
    const int grid = std::min(ntiles, 2 * sm_count());
    mlp_eval_kernel<<<grid, TILE, FW_BYTES, s>>>(net->dev(), x, y, ntiles, sc.flag);
    L_CUDA(cudaGetLastError());
    return check_flag(sc.flag, s);
}

lb_status lb_mlp_loss_grad(lb_mlp* net, const float* x, const float* t, int n, double* loss, float* grad,
                           void* stream) {
    if (!net || !x || !t || n <= 0 || n % TILE) return LB_ERR_ARG;
    lb_status st = set_smem_limits();
    if (st != LB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int ntiles = n / TILE;
    Scratch sc;
    st = sc.alloc(ntiles);
    if (st != LB_OK) return st;
    L_CUDA(cudaMemsetAsync(sc.flag, 0, sizeof(int), s));
    L_CUDA(cudaMemsetAsync(sc.loss, 0, sizeof(double), s));
    st = train_batch(net, x, t, nullptr, 0, ntiles, 0, 0.0f, 0, sc.partial, sc.loss, sc.flag, sc.grad, s);
    if (st != LB_OK) return st;
    st = check_flag(sc.flag, s);
    if (st != LB_OK) return st;
    double l = 0.0;
    L_CUDA(cudaMemcpy(&l, sc.loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (loss) *loss = l / ((double)n * NOUT);
    if (grad) L_CUDA(cudaMemcpy(grad, sc.grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return LB_OK;
}

lb_status lb_mlp_loss_grad_fp32(lb_mlp* net, const float* x, const float* t, int n, double* loss, float* grad,
                                void* stream) {
    if (!net || !x || !t || n <= 0) return LB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double* acc = nullptr;  // NPARAM gradient sums + 1 loss sum (FP64)
    L_CUDA(cudaMalloc((void**)&acc, (NPARAM + 1) * sizeof(double)));
    float* gf = nullptr;
    cudaError_t e = cudaMalloc((void**)&gf, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, (NPARAM + 1) * sizeof(double), s);
    if (e == cudaSuccess) {
        mlp_loss_grad_fp32_kernel<<<std::min(n, 8 * sm_count()), HID, 0, s>>>(net->params, x, t, n, acc,
                                                                              acc + NPARAM);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        doubles_to_floats<<<(NPARAM + 255) / 256, 256, 0, s>>>(acc, gf, NPARAM);
        e = cudaGetLastError();
    }
    double l = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, acc + NPARAM, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, gf, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(gf);
    cudaFree(acc);
    if (e != cudaSuccess) return fail_l(e, "lb_mlp_loss_grad_fp32");
    if (loss) *loss = l / ((double)n * NOUT);
    return LB_OK;
}

lb_status lb_mlp_train(lb_mlp* net, const float* pre, const float* post, long long n, int epochs, int batch,
                       float lr, uint64_t seed, float* epoch_loss, void* stream) {
    lbg::NvtxRange nvtx_("lb_mlp_train");
    if (!net || !pre || !post || n < batch || epochs < 1 || batch < TILE || batch % TILE || !(lr > 0.0f))
        return LB_ERR_ARG;
    if (n > (1ll << 31) - 1) return LB_ERR_ARG;
    lb_status st = set_smem_limits();
    if (st != LB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int ntiles = batch / TILE;
    Scratch sc;
    st = sc.alloc(ntiles);
    if (st != LB_OK) return st;
    // normalisation statistics from the data (FP64 sums on the device)
    {
        const int blocks = 4 * sm_count();
        double* part = nullptr;
        L_CUDA(cudaMalloc((void**)&part, (size_t)blocks * 4 * NIN * sizeof(double)));
        stats_kernel<<<blocks, STATS_THREADS, 0, s>>>(pre, post, n, part);
        std::vector<double> hp((size_t)blocks * 4 * NIN), h(4 * NIN, 0.0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(part);
        if (e != cudaSuccess) return fail_l(e, "normalisation statistics");
        for (int b = 0; b < blocks; ++b)  // block order: the same sums on every run
            for (int k = 0; k < 4 * NIN; ++k) h[k] += hp[(size_t)b * 4 * NIN + k];
        std::vector<float> norm(4 * NIN);
        for (int i = 0; i < NIN; ++i) {
            const double mx = h[i] / n, vx = std::max(0.0, h[NIN + i] / n - mx * mx);
            const double mt = h[2 * NIN + i] / n, vt = std::max(0.0, h[3 * NIN + i] / n - mt * mt);
            norm[i] = (float)mx;
            norm[NIN + i] = (float)(vx > 0.0 ? std::sqrt(vx) : 1.0);
            norm[2 * NIN + i] = (float)mt;
            norm[3 * NIN + i] = (float)(vt > 0.0 ? std::sqrt(vt) : 1.0);
        }
        L_CUDA(cudaMemcpyAsync(net->norm, norm.data(), 4 * NIN * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    // Each epoch's permutation is drawn on the host while the GPU trains on the previous one (two
    // pinned host buffers, two device buffers); the epochs' losses are summed into their own slots
    // and read at the end, so the host waits for the GPU only before reusing a host buffer.
    TrainBuffers tb;
    const long long nb = n / batch;
    st = tb.alloc(n, epochs, (long long)epochs * nb);
    if (st != LB_OK) return st;
    // one cooperative launch per epoch when the batch's CTAs can all be resident, else one launch
    // per batch and one for its Adam step (the same arithmetic)
    const bool loop = train_loop_fits(ntiles);
    if (loop) {
        st = tb.alloc_prepared(nb * batch);
        if (st != LB_OK) return st;
        std::vector<float> bc((size_t)epochs * nb * 2);
        for (long long k = 0; k < (long long)epochs * nb; ++k) {
            const float t = (float)(net->adam_steps + k + 1);
            bc[2 * k] = 1.0f - std::pow(0.9f, t);
            bc[2 * k + 1] = 1.0f - std::pow(0.999f, t);
        }
        L_CUDA(cudaMemcpyAsync(tb.bc, bc.data(), bc.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        L_CUDA(cudaStreamSynchronize(s));  // bc is a local vector
    }
    uint64_t rs = seed;
    auto shuffle = [&](int* perm) {
        for (long long k = 0; k < n; ++k) perm[k] = (int)k;
        for (long long k = n - 1; k > 0; --k) {  // Fisher-Yates
            const long long j = (long long)(splitmix64(rs) % (uint64_t)(k + 1));
            std::swap(perm[k], perm[j]);
        }
    };
    shuffle(tb.hperm[0]);
    L_CUDA(cudaMemsetAsync(sc.flag, 0, sizeof(int), s));
    L_CUDA(cudaMemsetAsync(tb.loss, 0, (size_t)epochs * sizeof(double), s));
    for (int ep = 0; ep < epochs && st == LB_OK; ++ep) {
        const int b = ep & 1;
        cudaError_t e = cudaMemcpyAsync(tb.dperm[b], tb.hperm[b], (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(tb.copied[b], s);
        if (e != cudaSuccess) {
            st = fail_l(e, "epoch setup");
            break;
        }
        if (loop) {
            const long long count = nb * batch;
            prep_epoch_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(pre, post, tb.dperm[b], count, net->norm,
                                                                             tb.ximg, tb.timg);
            e = cudaGetLastError();
            st = e != cudaSuccess ? fail_l(e, "epoch data")
                                  : train_epoch_loop(net, reinterpret_cast<const float*>(tb.ximg), tb.timg, (int)nb,
                                                     ntiles, lr, tb.bc + 2 * (long long)ep * nb, sc.partial,
                                                     tb.loss + ep, sc.flag, tb.gbar, s);
        }
        else
            for (long long bi = 0; bi < nb && st == LB_OK; ++bi)
                st = train_batch(net, pre, post, tb.dperm[b], bi * batch, ntiles, 1, lr, 1, sc.partial,
                                 tb.loss + ep, sc.flag, nullptr, s);
        if (st != LB_OK || ep + 1 == epochs) break;
        // the next epoch's permutation, into the host buffer whose copy (two epochs back) is done
        e = cudaEventSynchronize(tb.copied[b ^ 1]);
        if (e != cudaSuccess) {
            st = fail_l(e, "epoch setup");
            break;
        }
        shuffle(tb.hperm[b ^ 1]);
    }
    if (st == LB_OK) st = check_flag(sc.flag, s);
    if (st == LB_OK) {
        std::vector<double> l((size_t)epochs);
        cudaError_t e = cudaMemcpyAsync(l.data(), tb.loss, (size_t)epochs * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail_l(e, "epoch losses");
        else if (epoch_loss)
            for (int ep = 0; ep < epochs; ++ep) epoch_loss[ep] = (float)(l[ep] / ((double)nb * batch * NOUT));
    }
    cudaStreamSynchronize(s);
    return st;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// integration with lb_ctx (lb_capi.cu): launchers used by the C ABI there
// ------------------------------------------------------------------------------------------------
namespace lbg {

struct LearnedState {
    const lb_mlp* net = nullptr;
    unsigned char* tile_mode = nullptr;
    LearnedStats* stats = nullptr;
    float* scratch = nullptr;  // plain results of the tiles in flight: one tile per group
    int ctas = 1;
    char* mem = nullptr;
    float bound = 1e-4f;
    int check_every = 1;
    long long steps = 0;
};

lb_status learned_create(const lb_mlp* net, int Lx, int Ly, double bound, int check_every, LearnedState** out) {
    if (!net || !out || Lx % 32 || Ly % 32 || check_every < 1 || !(bound >= 0.0)) return LB_ERR_ARG;
    lb_status st = set_smem_limits();
    if (st != LB_OK) return st;
    LearnedState* ls = new (std::nothrow) LearnedState();
    if (!ls) return LB_ERR_ALLOC;
    const size_t ntiles = (size_t)(Lx / 32) * (Ly / 32);
    ls->ctas = sm_count();  // one CTA per SM, a scratch tile per group
    const size_t modes = (ntiles + 255) / 256 * 256;
    cudaError_t e = cudaMalloc((void**)&ls->mem,
                               256 + modes + (size_t)ls->ctas * ws::GROUPS * ws::SCRATCH_TILE * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ls;
        set_last_error("learned-collide state allocation failed");
        return LB_ERR_ALLOC;
    }
    ls->stats = (LearnedStats*)ls->mem;
    ls->tile_mode = (unsigned char*)(ls->mem + 256);
    ls->scratch = (float*)(ls->mem + 256 + modes);
    e = cudaMemset(ls->mem, 0, 256 + ntiles);
    if (e != cudaSuccess) {
        cudaFree(ls->mem);
        delete ls;
        return fail_l(e, "cudaMemset(learned state)");
    }
    ls->net = net;
    ls->bound = (float)bound;
    ls->check_every = check_every;
    *out = ls;
    return LB_OK;
}

lb_status learned_info(const LearnedState* ls, const lb_mlp** net, double* bound, int* check_every) {
    if (!ls) return LB_ERR_STATE;
    if (net) *net = ls->net;
    if (bound) *bound = ls->bound;
    if (check_every) *check_every = ls->check_every;
    return LB_OK;
}

// The caller has synchronised the stream that last used the state (lb_free and the collide
// setters do), so freeing does not need a device-wide synchronisation.
void learned_destroy(LearnedState* ls) {
    if (!ls) return;
    if (ls->mem) cudaFree(ls->mem);
    delete ls;
}

cudaError_t launch_step_learned(const float* src, float* dst, const StepParams& P, LearnedState* ls, int* flag,
                                cudaStream_t s) {
    const int check = (ls->steps % ls->check_every) == 0;
    ls->steps += 1;
    const int ntiles = (P.Lx / 32) * (P.Ly / 32);
    const int grid = std::min((ntiles + ws::GROUPS - 1) / ws::GROUPS, ls->ctas);
    step_learned_kernel<<<grid, ws::THREADS, ws::BYTES, s>>>(src, dst, P, ls->net->dev(), ls->tile_mode, check,
                                                             ls->bound, ls->stats, ls->scratch, flag);
    return cudaGetLastError();
}

cudaError_t launch_pairs(const float* src, const StepParams& P, const int* sites, int n, float* pre, float* post,
                         int* flag, cudaStream_t s) {
    pairs_kernel<<<(n + 127) / 128, 128, 0, s>>>(src, P, sites, n, pre, post, flag);
    return cudaGetLastError();
}

lb_status learned_tiles(LearnedState* ls, int ntiles, unsigned char* modes, cudaStream_t s) {
    L_CUDA(cudaMemcpyAsync(modes, ls->tile_mode, (size_t)ntiles, cudaMemcpyDeviceToHost, s));
    L_CUDA(cudaStreamSynchronize(s));
    return LB_OK;
}

lb_status learned_stats(LearnedState* ls, long long* checked, long long* fallback, double* max_res,
                        cudaStream_t s) {
    LearnedStats h;
    L_CUDA(cudaMemcpyAsync(&h, ls->stats, sizeof h, cudaMemcpyDeviceToHost, s));
    L_CUDA(cudaStreamSynchronize(s));
    if (checked) *checked = (long long)h.checked;
    if (fallback) *fallback = (long long)h.fallback;
    if (max_res) {
        float f;
        std::memcpy(&f, &h.max_res_bits, 4);
        *max_res = f;
    }
    return LB_OK;
}

}  // namespace lbg
