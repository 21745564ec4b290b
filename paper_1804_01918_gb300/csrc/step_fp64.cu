// step_fp64.cu -- FP64 D2Q37 kernels: fused time step, stand-alone propagate, init, moments, halos.
//
// Layout in HBM (structure of arrays, Sec. 4 / Fig. 2 "SoA"): f[i][y + HALO][x], x fastest,
// plane pitch (Ly + 2*HALO) * Lx doubles, three halo rows below row 0 and above row Ly-1 that
// hold the wall populations. Two copies (the prv/nxt double buffer of the Fig. 3 listing).
//
// The fused step (one thread per site; a warp covers 32 consecutive x of one row):
//   1. pull: f_i(x, y) = src_i((x - c_ix) mod Lx, y - c_iy) (Fig. 3 listing: read at an offset);
//      every source element is read by exactly one destination site, so a warp's 37 loads are
//      37 coalesced row segments, shifted by at most 3 elements;
//   2. collide (Sec. 3): moments from bins of equal c_x / equal c_y, shifted Hermite equilibrium
//      evaluated once per opposite pair (even/odd split), BGK relaxation;
//   3. store to dst with evict-first hints (write-once stream; GPU stores do no read-for-ownership,
//      the effect the paper gets from non-temporal stores, Sec. 4);
//   4. threads of rows 0..2 and Ly-3..Ly-1 also write the wall halo rows of dst.
// On GB300 this kernel is bound by the FP64 pipe (about 380 FP64 operations per site against 592
// bytes of traffic), so the code minimises FP64 operations; index math is integer-only.
#include <cuda_runtime.h>

#include <cstdint>

#include "d2q37_gpu.cuh"
#include "fixed96.cuh"
#include "kernels.cuh"

namespace lbg {

namespace {

__device__ __forceinline__ long long plane_off(int i, long long plane) { return (long long)i * plane; }

// Source index of population i for destination site (x, y) under the pull.
template <int I>
__device__ __forceinline__ int pull_index(int x, int y, int Lx, int Ly, int y_periodic) {
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

// True unless v is a positive finite double (integer test on the bit pattern).
__device__ __forceinline__ bool bad_positive(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b - 1ull) >= 0x7FEFFFFFFFFFFFFFull;
}

template <int I>
struct PullAll {
    __device__ __forceinline__ static void run(const double* __restrict__ src, double* f, int x,
                                               int y, int Lx, int Ly, int yp, long long plane) {
        PullAll<I - 1>::run(src, f, x, y, Lx, Ly, yp, plane);
        f[I] = __ldg(src + plane_off(I, plane) + pull_index<I>(x, y, Lx, Ly, yp));
    }
};
template <>
struct PullAll<-1> {
    __device__ __forceinline__ static void run(const double*, double*, int, int, int, int, int,
                                               long long) {}
};

struct SiteMoments {
    double rho, ux, uy, T;
};

// rho, u, T of one site from bins of equal c_x and equal c_y:
//   rho = sum f, rho u = r sum f c, rho (u^2 + D T) = r^2 sum f |c|^2.
// The bins and their combinations are exact 96-bit fixed-point sums on the integer pipe
// (fixed96.cuh); each of the four sums is rounded to FP64 once. *bad gets the status-word bit of a
// population outside the exact range: 1 for an infinity or NaN, 2 for a finite |f| >= 16, else 0.
__device__ __forceinline__ SiteMoments site_moments(const double* f, double r, double r2, int* bad) {
    using namespace fx;
    I96 bx[7], by[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) bx[k] = by[k] = zero96();
    unsigned emax = 0u;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const I96 n = to96(f[i], emax);
        add96(bx[cx_of(i) + 3], n);
        add96(by[cy_of(i) + 3], n);
    }
    *bad = emax == 0x7FFu ? 1 : (emax > EXP_LIMIT ? 2 : 0);
    const I96 px1 = plus96(bx[4], bx[2]), px2 = plus96(bx[5], bx[1]), px3 = plus96(bx[6], bx[0]);
    const I96 py1 = plus96(by[4], by[2]), py2 = plus96(by[5], by[1]), py3 = plus96(by[6], by[0]);
    const I96 n0 = plus96(plus96(bx[3], px1), plus96(px2, px3));
    const I96 nx = plus96(plus96(times3(minus96(bx[6], bx[0])), times2(minus96(bx[5], bx[1]))),
                          minus96(bx[4], bx[2]));
    const I96 ny = plus96(plus96(times3(minus96(by[6], by[0])), times2(minus96(by[5], by[1]))),
                          minus96(by[4], by[2]));
    const I96 ne = plus96(plus96(plus96(times9(px3), times4(px2)), px1),
                          plus96(plus96(times9(py3), times4(py2)), py1));
    // the four sums in units of 2^-48: the scale cancels in u and T
    const double n0d = to_double48(n0);
    const double inv = 1.0 / n0d;
    const double rinv = r * inv;
    SiteMoments m;
    m.rho = n0d * 0x1p-48;
    m.ux = to_double48(nx) * rinv;
    m.uy = to_double48(ny) * rinv;
    const double u2 = m.ux * m.ux + m.uy * m.uy;
    m.T = 0.5 * fma(r2 * inv, to_double48(ne), -u2);
    return m;
}

// xi.u of pair I from the multiples U[k] = k r u_x, V[k] = k r u_y (k = 1, 2, 3): a copy for the
// axis pairs, one add or subtract for the others.
template <int I>
__device__ __forceinline__ double pair_a(const double* U, const double* V) {
    constexpr int cx = cxh(I), cy = cyh(I);
    if (cy == 0) return U[cx];
    if (cx == 0) return cy > 0 ? V[cy] : -V[-cy];
    return cy > 0 ? U[cx] + V[cy] : U[cx] - V[-cy];
}

// Relax pair I (populations I and I + NPAIR, opposite vectors) of shell S. With the prefactor
// W = w rho / tau folded into the shell coefficients (WA0 = W A0, WA2 = W A2, WB1 = W B1,
// W24 = W / 24, W6 = W / 6):  W E = WA0 + a^2 (WA2 + a^2 W24),  W O = a (WB1 + a^2 W6),
// W f_eq(+-c) = W E +- W O, and f' = (1 - 1/tau) f + W f_eq -- one multiply (a^2) and 7 FMAs.
template <int I>
__device__ __forceinline__ void relax_pair(const double* f, double* __restrict__ dst, long long dsto,
                                           long long plane, const double* U, const double* V,
                                           const double* WA0, const double* WA2, const double* WB1,
                                           const double* W24, const double* W6, double omc) {
    constexpr int S = shellh(I);
    const double a = pair_a<I>(U, V);
    const double a2 = a * a;
    const double we = fma(a2, fma(a2, W24[S], WA2[S]), WA0[S]);
    const double q = fma(a2, W6[S], WB1[S]);
    const double gp = fma(a, q, we);
    const double gm = fma(-a, q, we);
    __stcs(dst + plane_off(I, plane) + dsto, fma(omc, f[I], gp));
    __stcs(dst + plane_off(I + NPAIR, plane) + dsto, fma(omc, f[I + NPAIR], gm));
}

template <int I>
struct RelaxAll {
    __device__ __forceinline__ static void run(const double* f, double* __restrict__ dst,
                                               long long dsto, long long plane, const double* U,
                                               const double* V, const double* WA0, const double* WA2,
                                               const double* WB1, const double* W24, const double* W6,
                                               double omc) {
        RelaxAll<I - 1>::run(f, dst, dsto, plane, U, V, WA0, WA2, WB1, W24, W6, omc);
        relax_pair<I>(f, dst, dsto, plane, U, V, WA0, WA2, WB1, W24, W6, omc);
    }
};
template <>
struct RelaxAll<0> {
    __device__ __forceinline__ static void run(const double*, double*, long long, long long, const double*,
                                               const double*, const double*, const double*, const double*,
                                               const double*, const double*, double) {}
};

// The multiples k r u (k = 1, 2, 3) of the shifted velocity, for pair_a.
__device__ __forceinline__ void velocity_multiples(double urx, double ury, double* U, double* V) {
    U[0] = V[0] = 0.0;
    U[1] = urx;
    V[1] = ury;
    U[2] = urx + urx;
    V[2] = ury + ury;
    U[3] = U[2] + urx;
    V[3] = V[2] + ury;
}

// Per-shell coefficients of the equilibrium at (theta, u2) scaled by prefactor W_s = wscale w_s.
__device__ __forceinline__ void shell_coefficients(const StepParams& P, double th, double u2,
                                                   double wscale, double* A0, double* A2,
                                                   double* B1, double* W) {
    const double a00 = fma(u2, fma(u2, 0.125, -0.5), 1.0);
    const double a20 = fma(u2, -0.25, 0.5);
    const double b10 = fma(u2, -0.5, 1.0);
    const double thu2 = th * u2;
    const double th2 = th * th;
#pragma unroll
    for (int s = 0; s < NSHELL; ++s) {
        A0[s] = fma(P.sh[s].gamma, th2, fma(P.sh[s].beta, thu2, fma(P.sh[s].alpha, th, a00)));
        A2[s] = fma(P.sh[s].delta, th, a20);
        B1[s] = fma(P.sh[s].eps, th, b10);
        W[s] = wscale * P.sh[s].w;
    }
}

// The same coefficients already multiplied by W_s = rw w_s, from site quantities scaled by rw:
//   W A0 = w rw a00 + (alpha w) rw theta + (beta w) rw theta u2 + (gamma w) rw theta^2, etc.
__device__ __forceinline__ void shell_coefficients_scaled(const StepParams& P, double th, double u2,
                                                          double rw, double* WA0, double* WA2,
                                                          double* WB1, double* W24, double* W6) {
    const double r0 = rw * fma(u2, fma(u2, 0.125, -0.5), 1.0);
    const double r20 = rw * fma(u2, -0.25, 0.5);
    const double r10 = rw * fma(u2, -0.5, 1.0);
    const double r1 = rw * th;
    const double ru = r1 * u2;
    const double r2 = r1 * th;
#pragma unroll
    for (int s = 0; s < NSHELL; ++s) {
        WA0[s] = fma(P.sh[s].gw, r2, fma(P.sh[s].bw, ru, fma(P.sh[s].aw, r1, P.sh[s].w * r0)));
        WA2[s] = fma(P.sh[s].dw, r1, P.sh[s].w * r20);
        WB1[s] = fma(P.sh[s].ew, r1, P.sh[s].w * r10);
        W24[s] = rw * P.sh[s].w24;
        W6[s] = rw * P.sh[s].w6;
    }
}

__global__ void __launch_bounds__(SITE_BLOCK)
step_fp64_kernel(const double* __restrict__ src, double* __restrict__ dst, const StepParams P,
                 int* __restrict__ flag) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long plane = P.plane;

    double f[NPOP];
    PullAll<NPOP - 1>::run(src, f, x, y, Lx, Ly, P.y_periodic, plane);

    int bad;
    const SiteMoments m = site_moments(f, P.r, P.r2, &bad);
    if (bad_positive(m.rho) || bad_positive(m.T) || bad) atomicOr(flag, bad ? bad : 1);

    // forcing: equilibrium at u + tau g, T + tau (1 - tau) |g|^2 / D
    const double uxs = m.ux + P.tgx;
    const double uys = m.uy + P.tgy;
    const double th = (m.T + P.dT_force) - 1.0;
    const double u2 = uxs * uxs + uys * uys;
    double WA0[NSHELL], WA2[NSHELL], WB1[NSHELL], W24[NSHELL], W6[NSHELL];
    shell_coefficients_scaled(P, th, u2, m.rho * P.omega, WA0, WA2, WB1, W24, W6);

    const long long dsto = (long long)(y + HALO) * Lx + x;
    __stcs(dst + dsto, fma(P.omc, f[0], WA0[0]));
    double U[4], V[4];
    velocity_multiples(P.r * uxs, P.r * uys, U, V);
    RelaxAll<NPAIR>::run(f, dst, dsto, plane, U, V, WA0, WA2, WB1, W24, W6, P.omc);

    // wall halo rows of dst from this site's post-collision fields (rho, u + g, T)
    write_wall_rows(P, x, y, m.rho, m.ux + P.gx, m.uy + P.gy, m.T, flag,
                    [&](int i, long long o, double v) { __stcs(dst + plane_off(i, plane) + o, v); });
}

// Collide only, in place (the paper's separate collide kernel, Sec. 3-5 and Table 1): each thread
// reads the 37 populations of its own site, relaxes them exactly as the fused step does, writes
// them back, and on rows 0..2 and Ly-3..Ly-1 writes the wall halo rows. After propagate this gives
// the same populations, bit for bit, as one fused step.
__global__ void __launch_bounds__(SITE_BLOCK)
collide_fp64_kernel(double* __restrict__ f, const StepParams P, int* __restrict__ flag) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long plane = P.plane;
    const long long o = (long long)(y + HALO) * Lx + x;
    double v[NPOP];
#pragma unroll
    for (int i = 0; i < NPOP; ++i) v[i] = f[plane_off(i, plane) + o];
    int bad;
    const SiteMoments m = site_moments(v, P.r, P.r2, &bad);
    if (bad_positive(m.rho) || bad_positive(m.T) || bad) atomicOr(flag, bad ? bad : 1);
    const double uxs = m.ux + P.tgx;
    const double uys = m.uy + P.tgy;
    const double th = (m.T + P.dT_force) - 1.0;
    const double u2 = uxs * uxs + uys * uys;
    double WA0[NSHELL], WA2[NSHELL], WB1[NSHELL], W24[NSHELL], W6[NSHELL];
    shell_coefficients_scaled(P, th, u2, m.rho * P.omega, WA0, WA2, WB1, W24, W6);
    __stcs(f + o, fma(P.omc, v[0], WA0[0]));
    double U[4], V[4];
    velocity_multiples(P.r * uxs, P.r * uys, U, V);
    RelaxAll<NPAIR>::run(v, f, o, plane, U, V, WA0, WA2, WB1, W24, W6, P.omc);
    write_wall_rows(P, x, y, m.rho, m.ux + P.gx, m.uy + P.gy, m.T, flag,
                    [&](int i, long long oh, double val) { __stcs(f + plane_off(i, plane) + oh, val); });
}

__global__ void __launch_bounds__(SITE_BLOCK)
propagate_fp64_kernel(const double* __restrict__ src, double* __restrict__ dst, const StepParams P) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long plane = P.plane;
    double f[NPOP];
    PullAll<NPOP - 1>::run(src, f, x, y, Lx, Ly, P.y_periodic, plane);
    const long long dsto = (long long)(y + HALO) * Lx + x;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) dst[plane_off(i, plane) + dsto] = f[i];
    if (y < HALO) {  // carry the halo rows over unchanged
        const long long ob = (long long)y * Lx + x;
        const long long ot = (long long)(Ly + HALO + y) * Lx + x;
#pragma unroll
        for (int i = 0; i < NPOP; ++i) {
            dst[plane_off(i, plane) + ob] = src[plane_off(i, plane) + ob];
            dst[plane_off(i, plane) + ot] = src[plane_off(i, plane) + ot];
        }
    }
}

// Full (unshifted) equilibrium of one site into out[37].
__device__ __forceinline__ void site_equilibrium(const StepParams& P, double rho, double ux,
                                                 double uy, double T, double* out) {
    double A0[NSHELL], A2[NSHELL], B1[NSHELL], W[NSHELL];
    shell_coefficients(P, T - 1.0, ux * ux + uy * uy, rho, A0, A2, B1, W);
    out[0] = W[0] * A0[0];
    const double urx = P.r * ux, ury = P.r * uy;
#pragma unroll
    for (int i = 1; i <= NPAIR; ++i) {
        const int s = shellh(i);
        const double a = cxh(i) * urx + cyh(i) * ury;
        const double a2 = a * a;
        const double e = fma(a2, fma(a2, 1.0 / 24.0, A2[s]), A0[s]);
        const double o = a * fma(a2, 1.0 / 6.0, B1[s]);
        out[i] = W[s] * (e + o);
        out[i + NPAIR] = W[s] * (e - o);
    }
}

__global__ void __launch_bounds__(SITE_BLOCK)
init_fp64_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                 const double* __restrict__ uy, const double* __restrict__ T,
                 double* __restrict__ f, const StepParams P) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    double fe[NPOP];
    site_equilibrium(P, rho[site], ux[site], uy[site], T[site], fe);
    const long long o = (long long)(y + HALO) * Lx + x;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) f[plane_off(i, P.plane) + o] = fe[i];
}

// Wall halos of f from the current interior rows 0..2 and Ly-3..Ly-1 (their moments), as the
// step writes them: thread t handles interior row k = t / Lx of each wall.
__global__ void halo_fp64_kernel(double* __restrict__ f, const StepParams P, int* __restrict__ flag) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= HALO * Lx) return;
    const int k = t / Lx;
    const int x = t - k * Lx;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int y = side == 0 ? k : Ly - 1 - k;
        if (side == 1 && y < HALO) continue;  // lattices with Ly < 6: that row was handled already
        const long long o = (long long)(HALO + y) * Lx + x;
        double v[NPOP];
#pragma unroll
        for (int i = 0; i < NPOP; ++i) v[i] = f[plane_off(i, P.plane) + o];
        int bad;
        const SiteMoments m = site_moments(v, P.r, P.r2, &bad);
        if (bad) atomicOr(flag, bad);
        write_wall_rows(P, x, y, m.rho, m.ux, m.uy, m.T, flag,
                        [&](int i, long long oh, double val) { f[plane_off(i, P.plane) + oh] = val; });
    }
}

__global__ void __launch_bounds__(SITE_BLOCK)
moments_fp64_kernel(const double* __restrict__ f, const StepParams P, double* __restrict__ rho,
                    double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T,
                    int half_step) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long o = (long long)(y + HALO) * Lx + x;
    double v[NPOP];
#pragma unroll
    for (int i = 0; i < NPOP; ++i) v[i] = f[plane_off(i, P.plane) + o];
    int bad;
    SiteMoments m = site_moments(v, P.r, P.r2, &bad);
    if (half_step) half_step_shift(P, m.ux, m.uy, m.T);
    rho[site] = m.rho;
    ux[site] = m.ux;
    uy[site] = m.uy;
    T[site] = m.T;
}

inline int site_blocks(const StepParams& P) {
    const long long n = (long long)P.Lx * P.Ly;
    return (int)((n + SITE_BLOCK - 1) / SITE_BLOCK);
}

}  // namespace

cudaError_t launch_step_fp64(const double* src, double* dst, const StepParams& P, int* flag,
                             cudaStream_t s) {
    step_fp64_kernel<<<site_blocks(P), SITE_BLOCK, 0, s>>>(src, dst, P, flag);
    return cudaGetLastError();
}

cudaError_t launch_collide_fp64(double* f, const StepParams& P, int* flag, cudaStream_t s) {
    collide_fp64_kernel<<<site_blocks(P), SITE_BLOCK, 0, s>>>(f, P, flag);
    return cudaGetLastError();
}

cudaError_t launch_propagate_fp64(const double* src, double* dst, const StepParams& P,
                                  cudaStream_t s) {
    propagate_fp64_kernel<<<site_blocks(P), SITE_BLOCK, 0, s>>>(src, dst, P);
    return cudaGetLastError();
}

cudaError_t launch_init_fp64(const double* rho, const double* ux, const double* uy,
                             const double* T, double* f, const StepParams& P, int* flag, cudaStream_t s) {
    init_fp64_kernel<<<site_blocks(P), SITE_BLOCK, 0, s>>>(rho, ux, uy, T, f, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || P.y_periodic) return e;
    return launch_halo_fp64(f, P, flag, s);
}

cudaError_t launch_moments_fp64(const double* f, const StepParams& P, double* rho, double* ux,
                                double* uy, double* T, int half_step, cudaStream_t s) {
    moments_fp64_kernel<<<site_blocks(P), SITE_BLOCK, 0, s>>>(f, P, rho, ux, uy, T, half_step);
    return cudaGetLastError();
}

cudaError_t launch_halo_fp64(double* f, const StepParams& P, int* flag, cudaStream_t s) {
    const int n = HALO * P.Lx;
    halo_fp64_kernel<<<(n + 127) / 128, 128, 0, s>>>(f, P, flag);
    return cudaGetLastError();
}

}  // namespace lbg
