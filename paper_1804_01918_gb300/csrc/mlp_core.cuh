// mlp_core.cuh -- the learned collide's MLP (37 -> 128 -> 128 -> 37, GELU) on tcgen05 tensor cores.
//
// A CTA handles 128 samples (one per TMEM lane / thread). Activations and weights are BF16 in
// shared memory in the no-swizzle core-matrix layout of tc_helpers.cuh, always stored
// "row-major by sample" (rows = samples or output features, 16-byte rows along the reduction
// dimension); accumulators are FP32 in TMEM.
//
//   forward   D1 = X  W1^T  (M 128, N 128, K 48)    z1 = D1 + b1, h1 = gelu(z1)
//             D2 = H1 W2^T  (M 128, N 128, K 128)   z2 = D2 + b2, h2 = gelu(z2)
//             D3 = H2 W3^T  (M 128, N 48,  K 128)   y  = D3 + b3 (first 37 columns)
//   backward  dH2 = dY W3   (B operand W3^T, K 48)  dz2 = dH2 * gelu'(z2)
//             dH1 = dZ2 W2  (B operand W2^T)        dz1 = dH1 * gelu'(z1)
//             dW3^T = H2^T dY, dW2 = dZ2^T H1, dW1 = dZ1^T X  (K = the 128 samples; both operands
//             read MN-major from the same sample-major buffers)
//
// Inputs and targets are normalised per population: x = (d_pre - mu_x) / sd_x and the network
// predicts the collision change t = (d_post - d_pre - mu_t) / sd_t.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "tc_helpers.cuh"

namespace lbg {
namespace mlp {

constexpr int NIN = 37;
constexpr int KIN = 48;    // input features padded to a multiple of 16
constexpr int HID = 128;
constexpr int NOUT = 37;
constexpr int NOUTP = 48;  // outputs padded to a multiple of 16
constexpr int TILE = 128;  // samples per MMA round

// Parameter packing (FP32): W1[128][37] b1[128] W2[128][128] b2[128] W3[37][128] b3[37]
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HID * NIN;
constexpr int OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID;
constexpr int OFF_B3 = OFF_W3 + NOUT * HID;
constexpr int NPARAM = OFF_B3 + NOUT;
// Stride (floats) between per-tile gradient partials: a multiple of 64 so that every row of the
// W2 block (OFF_W2 and HID are multiples of 4) starts 16-byte aligned for vector stores.
constexpr int PART_STRIDE = (NPARAM + 63) / 64 * 64;
static_assert(OFF_W2 % 4 == 0 && HID % 4 == 0, "vector stores of dW2 rows need 16-byte alignment");

// Byte sizes of the BF16 operand images.
constexpr int BYTES_X = TILE * KIN * 2;      // 12 KB
constexpr int BYTES_H = TILE * HID * 2;      // 32 KB
constexpr int BYTES_W1 = HID * KIN * 2;      // [128][48]
constexpr int BYTES_W2 = HID * HID * 2;      // [128][128]
constexpr int BYTES_W3 = NOUTP * HID * 2;    // [48][128]
constexpr int BYTES_W3T = HID * NOUTP * 2;   // [128][48]
constexpr int BYTES_W2T = HID * HID * 2;     // [128][128]
constexpr int BYTES_DY = TILE * NOUTP * 2;   // [128][48]

// Byte offset of element (r, k) in a [rows][K] BF16 operand image (K a multiple of 8).
__host__ __device__ constexpr int elem_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// GELU(z) = z Phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2, with erf from the rational approximation
// of Abramowitz & Stegun, Handbook of Mathematical Functions (1964), eq. 7.1.26:
//   erf(x) = 1 - P(t) exp(-x^2),  P(t) = a1 t + ... + a5 t^5,  t = 1 / (1 + p x),  x >= 0,
// |error| <= 1.5e-7, extended to x < 0 by oddness. With x = |z| / sqrt 2 and E = exp(-z^2 / 2):
//   Phi(z) = [z >= 0] - sign(z) P E / 2,  GELU(z) = max(z, 0) - |z| P E / 2,
//   GELU'(z) = Phi(z) + z phi(z) = [z >= 0] + E (z / sqrt(2 pi) - sign(z) P / 2),
// so the sign handling is a max or a select. The reciprocal and the exponential are the hardware
// approximations (rcp.approx, ex2.approx: relative error ~2^-22); the activations they feed are
// rounded to bfloat16 (relative 4e-3), so neither error is visible.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// P(t) / 2 and E for |z| = a
__device__ __forceinline__ void gelu_parts(float a, float& half_p, float& e) {
    constexpr float kP = (float)(0.3275911 * 0.70710678118654752);  // p / sqrt 2
    constexpr float c1 = 0.5f * 0.254829592f, c2 = 0.5f * -0.284496736f, c3 = 0.5f * 1.421413741f,
                    c4 = 0.5f * -1.453152027f, c5 = 0.5f * 1.061405429f;
    constexpr float kE = (float)(-0.5 * 1.4426950408889634);         // -log2(e) / 2
    const float t = rcp_approx(fmaf(kP, a, 1.0f));                   // argument >= 1
    half_p = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, c5, c4), c3), c2), c1);
    e = ex2_approx(a * a * kE);
}
__device__ __forceinline__ float gelu(float z) {
    const float a = fabsf(z);
    float hp, e;
    gelu_parts(a, hp, e);
    return fmaxf(z, 0.0f) - a * hp * e;
}
__device__ __forceinline__ float gelu_grad(float z) {
    float hp, e;
    gelu_parts(fabsf(z), hp, e);
    const float step = z >= 0.0f ? 1.0f : 0.0f;
    return fmaf(e, fmaf(z, 0.39894228040143268f, -copysignf(hp, z)), step);
}

// ---- pairs of FP32 values in one 64-bit register and the paired FP32 instructions of sm_100+
// (fma/mul/add .rn.f32x2): each rounds both halves exactly as its scalar counterpart does, in one
// instruction. The epilogues evaluate GELU and its derivative two columns at a time with them.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void x2_split(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_splat(float c) { return x2(c, c); }

// P(t) / 2 and E of gelu_parts for a pair |z| = (a0, a1), and the pair itself as A.
__device__ __forceinline__ void gelu_parts2(f32x2 A, float a0, float a1, f32x2& HP, f32x2& E) {
    constexpr float kP = (float)(0.3275911 * 0.70710678118654752);
    constexpr float c1 = 0.5f * 0.254829592f, c2 = 0.5f * -0.284496736f, c3 = 0.5f * 1.421413741f,
                    c4 = 0.5f * -1.453152027f, c5 = 0.5f * 1.061405429f;
    constexpr float kE = (float)(-0.5 * 1.4426950408889634);
    float d0, d1;
    x2_split(x2_fma(x2_splat(kP), A, x2_splat(1.0f)), d0, d1);
    const f32x2 T = x2(rcp_approx(d0), rcp_approx(d1));
    f32x2 P = x2_fma(T, x2_splat(c5), x2_splat(c4));
    P = x2_fma(T, P, x2_splat(c3));
    P = x2_fma(T, P, x2_splat(c2));
    HP = x2_mul(T, x2_fma(T, P, x2_splat(c1)));
    float q0, q1;
    x2_split(x2_mul(x2_mul(A, A), x2_splat(kE)), q0, q1);
    E = x2(ex2_approx(q0), ex2_approx(q1));
}

// GELU of z0 + b0 and z1 + b1 (in place): gelu() two at a time.
__device__ __forceinline__ void gelu_bias2(float& z0, float& z1, float b0, float b1) {
    float y0, y1;
    x2_split(x2_add(x2(z0, z1), x2(b0, b1)), y0, y1);
    const float a0 = fabsf(y0), a1 = fabsf(y1);
    f32x2 HP, E;
    gelu_parts2(x2(a0, a1), a0, a1, HP, E);
    // max(y, 0) - |y| P E / 2
    const f32x2 R = x2_fma(x2_mul(x2(-a0, -a1), HP), E, x2(fmaxf(y0, 0.0f), fmaxf(y1, 0.0f)));
    x2_split(R, z0, z1);
}

// v0 * GELU'(z0 + b0) and v1 * GELU'(z1 + b1) (into v0, v1): gelu_grad() two at a time.
__device__ __forceinline__ void gelu_grad_bias2(float& v0, float& v1, float z0, float z1, float b0, float b1) {
    float y0, y1;
    x2_split(x2_add(x2(z0, z1), x2(b0, b1)), y0, y1);
    const float a0 = fabsf(y0), a1 = fabsf(y1);
    f32x2 HP, E;
    gelu_parts2(x2(a0, a1), a0, a1, HP, E);
    float h0, h1;
    x2_split(HP, h0, h1);
    // [y >= 0] + E (y / sqrt(2 pi) - sign(y) P / 2)
    const f32x2 inner = x2_fma(x2(y0, y1), x2_splat(0.39894228040143268f), x2(-copysignf(h0, y0), -copysignf(h1, y1)));
    const f32x2 G = x2_fma(E, inner, x2(y0 >= 0.0f ? 1.0f : 0.0f, y1 >= 0.0f ? 1.0f : 0.0f));
    x2_split(x2_mul(x2(v0, v1), G), v0, v1);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Store 8 consecutive values (columns k0..k0+7, k0 a multiple of 8) of row r into an image.
__device__ __forceinline__ void store_row8(char* img, int r, int k0, int K, const float* v) {
    uint4 q;
    q.x = pack_bf16x2(v[0], v[1]);
    q.y = pack_bf16x2(v[2], v[3]);
    q.z = pack_bf16x2(v[4], v[5]);
    q.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(img + elem_off(r, k0, K)) = q;
}

// D = A[128][K] x B[N][K]^T, both K-major images; issued by one thread.
__device__ __forceinline__ void mma_kmajor(uint32_t d, const char* A, const char* B, int K, int N) {
    const uint32_t idesc = tc::idesc_bf16(128, N, 0, 0);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    for (int ks = 0; ks < K / 16; ++ks)
        tc::mma_bf16(d, tc::smem_desc(A + ks * 256, 128u, sbo), tc::smem_desc(B + ks * 256, 128u, sbo),
                     idesc, ks > 0 ? 1u : 0u);
}

// D[M=128][N] = sum over the 128 samples s of A[s][m] B[s][n]: A is a [128][FA] sample-major image
// (FA = 128), B a [128][FB] sample-major image (first N of FB features); both read MN-major.
__device__ __forceinline__ void mma_mnmajor(uint32_t d, const char* A, int FA, const char* B, int FB, int N) {
    const uint32_t idesc = tc::idesc_bf16(128, N, 1, 1);
    const uint32_t lboa = (uint32_t)(FA / 8) * 128u, lbob = (uint32_t)(FB / 8) * 128u;
    for (int ks = 0; ks < TILE / 16; ++ks)
        tc::mma_bf16(d, tc::smem_desc(A + ks * 2 * (int)lboa, lboa, 128u),
                     tc::smem_desc(B + ks * 2 * (int)lbob, lbob, 128u), idesc, ks > 0 ? 1u : 0u);
}

// TMEM address of this warp's 32 lanes at column col (warp w of a 4-warp group owns lanes 32w..).
__device__ __forceinline__ uint32_t tmem_lane_addr(uint32_t base, int warp, int col) {
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col;
}

// Copy nbytes (multiple of 16) from global to shared memory with the whole block.
__device__ __forceinline__ void copy_to_smem(char* dst, const char* src, int nbytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int k = threadIdx.x; k < nbytes / 16; k += blockDim.x) d[k] = __ldg(s + k);
}

}  // namespace mlp
}  // namespace lbg
