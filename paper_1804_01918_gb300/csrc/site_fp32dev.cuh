// site_fp32dev.cuh -- per-site device code of the FP32-deviation step, shared by the
// single-lattice kernel (step_fp32dev.cu) and the ensemble kernel (ensemble.cu).
#pragma once

#include <cuda_runtime.h>

#include "d2q37_gpu.cuh"

namespace lbg {

namespace {

__device__ __forceinline__ long long poff(int i, long long plane) { return (long long)i * plane; }

template <int I>
__device__ __forceinline__ int pull_index32(int x, int y, int Lx, int Ly, int y_periodic) {
    constexpr int cx = cx_of(I);
    constexpr int cy = cy_of(I);
    int xs = x - cx;
    if (cx > 0) {
        if (xs < 0) xs += Lx;
    } else if (cx < 0) {
        if (xs >= Lx) xs -= Lx;
    }
    int ys = y - cy;
    if (y_periodic) {
        if (cy > 0) {
            if (ys < 0) ys += Ly;
        } else if (cy < 0) {
            if (ys >= Ly) ys -= Ly;
        }
    }
    return (ys + HALO) * Lx + xs;
}

template <int I>
struct Pull32 {
    __device__ __forceinline__ static void run(const float* __restrict__ src, float* d, int x, int y,
                                               int Lx, int Ly, int yp, long long plane) {
        Pull32<I - 1>::run(src, d, x, y, Lx, Ly, yp, plane);
        d[I] = __ldg(src + poff(I, plane) + pull_index32<I>(x, y, Lx, Ly, yp));
    }
};
template <>
struct Pull32<-1> {
    __device__ __forceinline__ static void run(const float*, float*, int, int, int, int, int, long long) {}
};

__device__ __forceinline__ bool bad_positive64(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b - 1ull) >= 0x7FEFFFFFFFFFFFFFull;
}

// The FP64 value of an FP32 number, assembled on the integer pipe (the conversion instruction
// issues on GB300's narrow FP64 pipe, twice per population and step here): sign kept, exponent
// rebiased by 1023 - 127, significand shifted into place; a subnormal input is normalised by a
// leading-zero count. Exact, as the conversion is (every FP32 value is an FP64 value); infinities
// and NaN map to infinities and NaN.
__device__ __forceinline__ double exact_double(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned m = b & 0x7FFFFFu;
    const unsigned lz = __clz(m | 1u) - 8u;  // brings a subnormal's leading one to bit 23
    const bool sub = e == 0u;
    const unsigned mm = sub ? (m << lz) & 0x7FFFFFu : m;
    const unsigned E = e == 0xFFu ? 0x7FFu : (sub ? (m == 0u ? 0u : 897u - lz) : e + 896u);
    const unsigned hi = (b & 0x80000000u) | (E << 20) | (mm >> 3);
    return __hiloint2double((int)hi, (int)(mm << 29));
}

// FP64 sums of FP32 deviations: s0 = sum d, sx = sum d c_x, sy = sum d c_y, se = sum d |c|^2.
struct DevSums {
    double s0, sx, sy, se;
};

__device__ __forceinline__ DevSums dev_sums(const float* d) {
    double bx[7], by[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        bx[k] = 0.0;
        by[k] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const double v = exact_double(d[i]);
        bx[cx_of(i) + 3] += v;
        by[cy_of(i) + 3] += v;
    }
    const double px1 = bx[4] + bx[2], px2 = bx[5] + bx[1], px3 = bx[6] + bx[0];
    const double py1 = by[4] + by[2], py2 = by[5] + by[1], py3 = by[6] + by[0];
    DevSums s;
    s.s0 = bx[3] + px1 + px2 + px3;
    s.sx = fma(3.0, bx[6] - bx[0], fma(2.0, bx[5] - bx[1], bx[4] - bx[2]));
    s.sy = fma(3.0, by[6] - by[0], fma(2.0, by[5] - by[1], by[4] - by[2]));
    s.se = fma(9.0, px3, fma(4.0, px2, px1)) + fma(9.0, py3, fma(4.0, py2, py1));
    return s;
}

struct Macro {
    double rho, ux, uy, T;
};

__device__ __forceinline__ Macro macro_of(const DevSums& s, double r, double r2) {
    Macro m;
    m.rho = 1.0 + s.s0;
    const double inv = 1.0 / m.rho;
    const double rinv = r * inv;
    m.ux = s.sx * rinv;
    m.uy = s.sy * rinv;
    const double u2 = m.ux * m.ux + m.uy * m.uy;
    // sum f |c|^2 = D / r^2 + se  ->  rho (u^2 + D T) = r^2 sum f |c|^2 = D + r^2 se
    m.T = 0.5 * (fma(r2, s.se, DIM) * inv - u2);
    return m;
}

// FP32 relaxation of deviations d = f - w toward the shifted equilibrium, regrouped as in the
// FP64 step (step_fp64.cu, relax_site_terms): pair variable b = xi.u*/4 from multiples
// U[k] = k r u*_x / 4, V[k] = k r u*_y / 4, and per shell (W = w / tau)
//   (f_eq(+-c) - w) / tau = WA0 + b^2 (WA2 + C b^2) +- b (WB1 + C b^2),
//   WA0 = W (rho (A0 - 1) + rho - 1),  WA2 = 16 W rho A2,  WB1 = 4 W rho B1,  C = (32/3) W rho,
// with A0 - 1, A2, B1 polynomials in xi^2 whose site coefficients are shared by all shells (h =
// theta/2, m = 1/2 - u*^2/4): A0 - 1 = (u*^4/8 - u*^2/2) + 2h (u*^2 - 1 + 2h) + xi^2 2h (m - 2h)
// + xi^4 h^2 / 2, A2 = m - 3h + xi^2 h / 2, B1 = 2 (m - 2h) + xi^2 h. A0 - 1 is formed from its
// small terms, so the deviation form loses nothing to cancellation. Per pair: one multiply and 7
// FMAs; per shell 8 operations.
struct Relax32 {
    float U[4], V[4];
    float WA0[NSHELL], WA2[NSHELL], WB1[NSHELL], C[NSHELL];
};

// rho and s0 = rho - 1 (kept apart for accuracy), omega = 1/tau, (uxs, uys) = u*, h = (T* - 1)/2.
__device__ __forceinline__ void relax_coefficients32(const StepParams& P, float rho, float s0,
                                                     float omega, float uxs, float uys, float h,
                                                     Relax32& R) {
    const float u2 = fmaf(uxs, uxs, uys * uys);
    const float rr = omega * rho, rs = omega * s0;
    const float a00m1 = u2 * fmaf(u2, 0.125f, -0.5f);
    const float R0 = fmaf(h + h, fmaf(2.0f, h, u2 - 1.0f), a00m1);  // A0 - 1 at xi = 0
    const float bq = fmaf(u2, -0.25f, fmaf(h, -2.0f, 0.5f));         // m - 2h
    const float t = rr * h;
    const float Q0 = fmaf(rr, R0, rs);
    const float Q1 = t * bq;
    const float Q2 = t * h;
    const float Rb = rr * bq;
    const float Ra = Rb - t;                                          // rho (m - 3h)
    R.WA0[0] = P.sh32[0].q_a0 * Q0;
#pragma unroll
    for (int q = 1; q < NSHELL; ++q) {
        const ShellCoef32& c = P.sh32[q];
        R.WA0[q] = fmaf(c.q_a2, Q2, fmaf(c.q_a1, Q1, c.q_a0 * Q0));
        R.WA2[q] = fmaf(c.q_e1, t, c.q_e0 * Ra);
        R.WB1[q] = fmaf(c.q_b1, t, c.q_b0 * Rb);
        R.C[q] = c.q_c * rr;
    }
    const float U1 = P.lr_f * uxs, V1 = P.lr_f * uys;
    R.U[0] = R.V[0] = 0.0f;
    R.U[1] = U1;
    R.V[1] = V1;
    R.U[2] = U1 + U1;
    R.V[2] = V1 + V1;
    R.U[3] = R.U[2] + U1;
    R.V[3] = R.V[2] + V1;
}

template <int I>
__device__ __forceinline__ float pair_b32(const float* U, const float* V) {
    constexpr int cx = cxh(I), cy = cyh(I);
    if (cy == 0) return U[cx];
    if (cx == 0) return cy > 0 ? V[cy] : -V[-cy];
    return cy > 0 ? U[cx] + V[cy] : U[cx] - V[-cy];
}

// Relax pair I (populations I and I + NPAIR) in place.
template <int I>
__device__ __forceinline__ void relax_pair32(float* d, const Relax32& R, float omc) {
    constexpr int S = shellh(I);
    const float b = pair_b32<I>(R.U, R.V);
    const float b2 = b * b;
    const float we = fmaf(b2, fmaf(b2, R.C[S], R.WA2[S]), R.WA0[S]);
    const float q = fmaf(b2, R.C[S], R.WB1[S]);
    d[I] = fmaf(omc, d[I], fmaf(b, q, we));
    d[I + NPAIR] = fmaf(omc, d[I + NPAIR], fmaf(-b, q, we));
}

template <int I>
struct Relax32All {
    __device__ __forceinline__ static void run(float* d, const Relax32& R, float omc) {
        Relax32All<I - 1>::run(d, R, omc);
        relax_pair32<I>(d, R, omc);
    }
};
template <>
struct Relax32All<0> {
    __device__ __forceinline__ static void run(float*, const Relax32&, float) {}
};

// All 37 deviations relaxed in place.
__device__ __forceinline__ void relax32(float* d, const Relax32& R, float omc) {
    d[0] = fmaf(omc, d[0], R.WA0[0]);
    Relax32All<NPAIR>::run(d, R, omc);
}

}  // namespace

// Wall halo rows of an FP32-deviation lattice fed by site (x, y), from its post-collision fields.
// Not inlined: the six wall rows' FP64 code then costs the per-site path no registers.
static __device__ __noinline__ void split_wall_rows(float* __restrict__ dst, const StepParams& P, int x, int y,
                                             double rho, double ux, double uy, double T,
                                             int* __restrict__ flag) {
    const long long plane = P.plane;
    write_wall_rows(P, x, y, rho, ux, uy, T, flag, [&](int i, long long o, double v) {
        __stcs(dst + (long long)i * plane + o, (float)(v - shell_w(shell_of(i))));
    });
}

// Rest-closure wall halo rows fed by site (x, y): rho times the rest equilibrium per unit density
// at the wall temperature, stored as FP32 deviations (none on a side cut from a neighbouring slab).
__device__ __forceinline__ void rest_wall_rows32(float* __restrict__ dst, const StepParams& P, int x, int y,
                                                 double rho) {
    const int Lx = P.Lx, Ly = P.Ly;
    const long long plane = P.plane;
    if (y < HALO && !(P.cut & 1)) {
        const long long o = (long long)(HALO - 1 - y) * Lx + x;
#pragma unroll
        for (int i = 0; i < NPOP; ++i)
            __stcs(dst + (long long)i * plane + o, (float)fma(rho, P.wall_bot[i], -shell_w(shell_of(i))));
    }
    if (y >= Ly - HALO && !(P.cut & 2)) {
        const long long o = (long long)(Ly + HALO + (Ly - 1 - y)) * Lx + x;
#pragma unroll
        for (int i = 0; i < NPOP; ++i)
            __stcs(dst + (long long)i * plane + o, (float)fma(rho, P.wall_top[i], -shell_w(shell_of(i))));
    }
}

// Wall halo rows of an FP32-deviation lattice fed by site (x, y) on rows 0..2 / Ly-3..Ly-1, from
// its post-collision fields. kMirror = false compiles the rest closure only (kernels whose
// lattices all use it); otherwise the mirror closure runs out of line, so its FP64 code costs the
// per-site path no registers.
template <bool kMirror>
__device__ __forceinline__ void wall_rows32(float* __restrict__ dst, const StepParams& P, int x, int y,
                                            double rho, double ux, double uy, double T,
                                            int* __restrict__ flag) {
    if (P.y_periodic || (y >= HALO && y < P.Ly - HALO)) return;
    if (kMirror && P.wall_mode == 1)
        split_wall_rows(dst, P, x, y, rho, ux, uy, T, flag);
    else
        rest_wall_rows32(dst, P, x, y, rho);
}

// One fused FP32-deviation step of site (x, y): src/dst are the member's two population copies,
// P its parameters (kernel parameter space or shared memory). Shared with the ensemble kernel.
template <bool kMirror = true>
__device__ __forceinline__ void fp32dev_site(const float* __restrict__ src, float* __restrict__ dst,
                                             const StepParams& P, int x, int y,
                                             int* __restrict__ flag) {
    const int Lx = P.Lx, Ly = P.Ly;
    const long long plane = P.plane;

    float d[NPOP];
    Pull32<NPOP - 1>::run(src, d, x, y, Lx, Ly, P.y_periodic, plane);

    const DevSums pre = dev_sums(d);
    const Macro m = macro_of(pre, P.r, P.r2);
    if (bad_positive64(m.rho) || bad_positive64(m.T)) atomicOr(flag, 1);

    // shifted equilibrium (forcing), coefficients in FP32 from FP64 moments
    Relax32 R;
    relax_coefficients32(P, (float)m.rho, (float)pre.s0, P.omega_f, (float)(m.ux + P.tgx),
                         (float)(m.uy + P.tgy), (float)(0.5 * ((m.T + P.dT_force) - 1.0)), R);
    relax32(d, R, P.omc_f);

    // FP64 projection onto the exact post-collision moments (c units):
    //   sum d' = rho - 1,  sum d' c = sum d c + rho g / r,
    //   sum d' |c|^2 = sum d |c|^2 + rho (2 u.g + |g|^2) / r^2
    const DevSums post = dev_sums(d);
    const double gx = P.gx, gy = P.gy;
    const double rinv = 1.0 / P.r;
    const double R0 = pre.s0 - post.s0;
    const double Rx = fma(m.rho * gx, rinv, pre.sx) - post.sx;
    const double Ry = fma(m.rho * gy, rinv, pre.sy) - post.sy;
    const double de = m.rho * (2.0 * (m.ux * gx + m.uy * gy) + gx * gx + gy * gy) * (rinv * rinv);
    const double Re = (pre.se + de) - post.se;
    // weighted least-norm correction: M diag(w) M^T lambda = R with
    // M diag(w) M^T = [[1, 2/r^2], [2/r^2, 8/r^4]] (mass/energy block), 1/r^2 (momentum)
    const double r2 = P.r2;
    const float l0 = (float)(2.0 * R0 - 0.5 * r2 * Re);
    const float le = (float)(r2 * (0.25 * r2 * Re - 0.5 * R0));
    const float lx = (float)(r2 * Rx);
    const float ly = (float)(r2 * Ry);

    const long long dsto = (long long)(y + HALO) * Lx + x;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const float corr = fmaf(le, (float)shell_c2(shell_of(i)),
                                fmaf(lx, (float)cx_of(i), fmaf(ly, (float)cy_of(i), l0)));
        __stcs(dst + poff(i, plane) + dsto, fmaf((float)shell_w(shell_of(i)), corr, d[i]));
    }

    // wall halo rows from the post-collision fields (rho, u + g, T), stored as FP32 deviations
    if (!P.y_periodic && (y < HALO || y >= Ly - HALO))
        wall_rows32<kMirror>(dst, P, x, y, m.rho, m.ux + gx, m.uy + gy, m.T, flag);
}

}  // namespace lbg

namespace lbg {
namespace split32 {

// Exact accumulation of FP32 deviations by an error-free split at a fixed quantum q = 2^-22:
// for |d| < 1, t = d + 3 lies in [2, 4), where the FP32 spacing is exactly q, so
//   n = bits(t) - bits(3.0f) = rint(d / q)   (an integer, |n| < 2^22)
//   r = d - (t - 3)                          (exact, |r| <= q / 2)
// and d = n q + r exactly (the magic-number split of Rump, Ogita and Oishi's ExtractScalar, read
// through the bit pattern). The n parts are summed as 32-bit integers -- exactly: |c|^2-weighted
// sums stay below 216 x 2^22 < 2^31 -- and only the r parts are summed in FP32 (absolute error
// <= ~6e-11). Pre- and post-collision sums use the same quantum, so their differences (the
// projection residuals) are exact in the integer parts.
constexpr float QB = 3.0f;
constexpr float Q = 2.384185791015625e-07f;  // 2^-22
constexpr float RANGE = 1.0f;                // |d| must stay below this for the split to be exact

struct Part {
    int n0, nx, ny, ne;       // integer parts of sum d, sum c_x d, sum c_y d, sum |c|^2 d (units of q)
    float r0, rx, ry, re;     // rounded sums of the residuals
};

__device__ __forceinline__ void split_sums(const float* d, Part& p) {
    unsigned bx[7], by[7];
    float rx[7], ry[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        bx[k] = by[k] = 0u;
        rx[k] = ry[k] = 0.0f;
    }
    // bins sum the raw bit patterns of t modulo 2^32 (unsigned: well-defined wrap-around); the
    // bias bits(3.0f) per term cancels in the odd (difference) combinations and is removed once per
    // even combination (the number of populations per bin is a constant), and every final
    // combination fits in a signed 32-bit integer, so the modular arithmetic gives it exactly
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const float t = __fadd_rn(d[i], QB);
        const float r = __fsub_rn(d[i], __fsub_rn(t, QB));
        const unsigned n = __float_as_uint(t);
        const int ix = cx_of(i) + 3, iy = cy_of(i) + 3;
        bx[ix] += n;
        by[iy] += n;
        rx[ix] += r;
        ry[iy] += r;
    }
    constexpr unsigned b3 = 0x40400000u;  // bits of 3.0f
    const unsigned px1 = bx[4] + bx[2], px2 = bx[5] + bx[1], px3 = bx[6] + bx[0];
    const unsigned py1 = by[4] + by[2], py2 = by[5] + by[1], py3 = by[6] + by[0];
    // populations per bin: c = 0: 7, |c| = 1: 7 each, 2: 5 each, 3: 3 each (x and y alike)
    p.n0 = (int)((((bx[3] + px1) + px2) + px3) - (unsigned)NPOP * b3);
    p.nx = (int)(3u * (bx[6] - bx[0]) + 2u * (bx[5] - bx[1]) + (bx[4] - bx[2]));
    p.ny = (int)(3u * (by[6] - by[0]) + 2u * (by[5] - by[1]) + (by[4] - by[2]));
    p.ne = (int)(((9u * px3 + 4u * px2 + px1) + (9u * py3 + 4u * py2 + py1)) -
                 2u * (9u * 6u + 4u * 10u + 14u) * b3);
    const float qx1 = rx[4] + rx[2], qx2 = rx[5] + rx[1], qx3 = rx[6] + rx[0];
    const float qy1 = ry[4] + ry[2], qy2 = ry[5] + ry[1], qy3 = ry[6] + ry[0];
    p.r0 = ((rx[3] + qx1) + qx2) + qx3;
    p.rx = fmaf(3.0f, rx[6] - rx[0], fmaf(2.0f, rx[5] - rx[1], rx[4] - rx[2]));
    p.ry = fmaf(3.0f, ry[6] - ry[0], fmaf(2.0f, ry[5] - ry[1], ry[4] - ry[2]));
    p.re = fmaf(9.0f, qx3, fmaf(4.0f, qx2, qx1)) + fmaf(9.0f, qy3, fmaf(4.0f, qy2, qy1));
}

template <int I>
struct MaxAbs {
    __device__ __forceinline__ static float run(const float* d) {
        return fmaxf(MaxAbs<I - 1>::run(d), fabsf(d[I]));
    }
};
template <>
struct MaxAbs<0> {
    __device__ __forceinline__ static float run(const float* d) { return fabsf(d[0]); }
};

__device__ __forceinline__ bool bad_positive32(float v) {
    const unsigned b = __float_as_uint(v);
    return (b - 1u) >= 0x7F7FFFFFu;
}

}  // namespace split32

// Pre-collision state of one site for the exact-split path: exact hi/mid sums, rounded lo sums,
// and the FP32 macroscopic fields derived from them.
struct SplitPre {
    split32::Part p;
    float s0, rho, ux, uy, T;
};

// Sums and fields of the pulled deviations d; sets flag bit 1 (non-finite / non-positive density
// or temperature) or 2 (a deviation outside the exact-split range).
__device__ __forceinline__ void split_pre(const float* d, const StepParams& P, SplitPre& s,
                                          int* __restrict__ flag) {
    using namespace split32;
    const float dmax = MaxAbs<NPOP - 1>::run(d);
    split_sums(d, s.p);
    s.s0 = fmaf((float)s.p.n0, Q, s.p.r0);
    const float sx = fmaf((float)s.p.nx, Q, s.p.rx);
    const float sy = fmaf((float)s.p.ny, Q, s.p.ry);
    const float se = fmaf((float)s.p.ne, Q, s.p.re);
    const float r = P.r_f, r2 = P.r2_f;
    s.rho = 1.0f + s.s0;
    const float inv = 1.0f / s.rho;
    s.ux = r * sx * inv;
    s.uy = r * sy * inv;
    // rho (u^2 + D T) = D + r^2 se  (sum w xi^2 = D)
    s.T = 0.5f * (fmaf(r2, se, 2.0f) * inv - (s.ux * s.ux + s.uy * s.uy));
    if (bad_positive32(s.rho) || bad_positive32(s.T) || !(dmax < RANGE))
        atomicOr(flag, !(dmax < RANGE) ? 2 : 1);
}

// FP32 BGK relaxation of d (in place) toward the shifted Hermite equilibrium of s. C supplies the
// lattice constants (r, shell coefficients: the same for every lattice), M the lattice's own
// relaxation time and gravity; single lattices pass the same parameters twice.
__device__ __forceinline__ void split_collide(float* d, const StepParams& C, const StepParams& M,
                                              const SplitPre& s) {
    Relax32 R;
    relax_coefficients32(C, s.rho, s.s0, M.omega_f, s.ux + M.tgx_f, s.uy + M.tgy_f,
                         0.5f * ((s.T + M.dT_force_f) - 1.0f), R);
    relax32(d, R, M.omc_f);
}

// Project candidate post-collision deviations d (in place) onto the exact post-collision moments:
// sum d' = sum d, sum d' c = sum d c + rho g / r, sum d' |c|^2 = sum d |c|^2 + rho (2 u.g + g^2) / r^2,
// with the weighted least-norm correction d_i += w_i (l0 + lx c_x + ly c_y + le |c|^2). The
// residual is formed from exact hi/mid differences (same quanta before and after).
__device__ __forceinline__ void split_project(float* d, const StepParams& C, const StepParams& M,
                                              const SplitPre& s) {
    using namespace split32;
    Part p1;
    split_sums(d, p1);
    const float r = C.r_f, r2 = C.r2_f;
    const float gx = M.gx_f, gy = M.gy_f;
    const float rinv = 1.0f / r;
    // integer differences are exact; only the residual sums round
    const float R0 = fmaf((float)(s.p.n0 - p1.n0), Q, s.p.r0 - p1.r0);
    const float Rx = fmaf((float)(s.p.nx - p1.nx), Q, s.p.rx - p1.rx) + s.rho * gx * rinv;
    const float Ry = fmaf((float)(s.p.ny - p1.ny), Q, s.p.ry - p1.ry) + s.rho * gy * rinv;
    const float Re = fmaf((float)(s.p.ne - p1.ne), Q, s.p.re - p1.re) +
                     s.rho * (2.0f * (s.ux * gx + s.uy * gy) + gx * gx + gy * gy) * (rinv * rinv);
    const float lam0 = 2.0f * R0 - 0.5f * r2 * Re;
    const float lame = r2 * (0.25f * r2 * Re - 0.5f * R0);
    const float lamx = r2 * Rx, lamy = r2 * Ry;
    // correction w_i (even_s +- odd_i): even part per shell, odd part per opposite pair
    float ev[NSHELL];
#pragma unroll
    for (int k = 0; k < NSHELL; ++k)
        ev[k] = (float)shell_w(k) * fmaf(lame, (float)shell_c2(k), lam0);
    d[0] += ev[0];
#pragma unroll
    for (int i = 1; i <= NPAIR; ++i) {
        const float od = (float)shell_w(shellh(i)) * fmaf(lamx, (float)cxh(i), lamy * (float)cyh(i));
        d[i] += ev[shellh(i)] + od;
        d[i + NPAIR] += ev[shellh(i)] - od;
    }
}

// Store a site's deviations and, on wall rows, the wall halo rows from the site's post-collision
// fields (rho, u + g, T; FP64 arithmetic on the six wall rows only).
template <bool kMirror = true>
__device__ __forceinline__ void split_store(float* __restrict__ dst, const StepParams& P, int x,
                                            int y, const float* d, const SplitPre& s,
                                            int* __restrict__ flag) {
    const long long dsto = (long long)(y + HALO) * P.Lx + x;
    char* const base = reinterpret_cast<char*>(dst + dsto);
#pragma unroll
    // plain write-back stores: measured ~1 % faster than evict-first (st.cs) for this kernel
    for (int i = 0; i < NPOP; ++i) *reinterpret_cast<float*>(base + P.plane_b32[i]) = d[i];
    if (!P.y_periodic && (y < HALO || y >= P.Ly - HALO))  // FP64 work on the six wall rows only
        wall_rows32<kMirror>(dst, P, x, y, 1.0 + (double)s.s0, (double)s.ux + P.gx, (double)s.uy + P.gy,
                             (double)s.T, flag);
}

// One fused FP32-deviation step of site (x, y) with exact-split FP32 moment accumulation and an
// FP32 projection residual (no FP64 arithmetic except on the six wall rows). Flag bits: 1 =
// non-finite or non-positive density/temperature, 2 = a deviation outside the exact-split range.
// C: lattice constants (r, shell coefficients), M: this lattice's sizes, relaxation, gravity and
// walls (the same object for a single lattice).
// Pull with precomputed byte offsets from the site's own element: valid unless the source wraps.
// The loads ask L2 to fetch 256-byte blocks (L2::256B): the neighbouring warp's row segment then
// comes from L2 (measured +1.4 % for the single lattice, +1.6 % for the ensemble at 2304 x 8192;
// 128-byte blocks: no change; L1 evict-first or no-allocate: -6 %, the neighbours' misaligned
// segments are shared through L1).
template <int I>
struct PullFast32 {
    __device__ __forceinline__ static void run(const char* base, float* d, const StepParams& M) {
        PullFast32<I - 1>::run(base, d, M);
        float v;
        asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(base + M.pull_b32[I]));
        d[I] = v;
    }
};
template <>
struct PullFast32<-1> {
    __device__ __forceinline__ static void run(const char*, float*, const StepParams&) {}
};

__device__ __forceinline__ void pull32(const float* __restrict__ src, float* d, const StepParams& M, int x,
                                       int y) {
    const bool interior = x >= HALO && x < M.Lx - HALO && (!M.y_periodic || (y >= HALO && y < M.Ly - HALO));
    if (interior)
        PullFast32<NPOP - 1>::run(reinterpret_cast<const char*>(src + (long long)(y + HALO) * M.Lx + x), d, M);
    else
        Pull32<NPOP - 1>::run(src, d, x, y, M.Lx, M.Ly, M.y_periodic, M.plane);
}

template <bool kMirror = true>
__device__ __forceinline__ void fp32split_site(const float* __restrict__ src, float* __restrict__ dst,
                                               const StepParams& C, const StepParams& M, int x, int y,
                                               int* __restrict__ flag) {
    float d[NPOP];
    pull32(src, d, M, x, y);
    SplitPre s;
    split_pre(d, C, s, flag);
    split_collide(d, C, M, s);
    split_project(d, C, M, s);
    split_store<kMirror>(dst, M, x, y, d, s, flag);
}

}  // namespace lbg
