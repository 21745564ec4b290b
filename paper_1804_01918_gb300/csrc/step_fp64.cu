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
// On GB300 this kernel is bound by the FP64 pipe (FP64 instructions per site against 592 bytes of
// traffic), so the code minimises FP64 operations: moment sums on the integer pipe, equilibrium
// coefficients shared per shell (relax_site_terms, shell_relax), integer-only index math.
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

// The four moment sums of one site in units of 2^-48: n0 = sum f, nx = sum f c_x, ny = sum f c_y,
// ne = sum f |c|^2. They are exact 96-bit fixed-point sums on the integer pipe (fixed96.cuh) over
// bins of equal c_x and equal c_y, each rounded to FP64 once. *bad gets the status-word bit of a
// population outside the exact range: 1 for an infinity or NaN, 2 for a finite |f| >= 16, else 0.
struct SiteSums {
    double n0, nx, ny, ne;
};

// The moment sums as an accumulator over populations given one at a time (add<I>), so that a caller
// can take the populations in batches.
struct SumBins {
    fx::I96 bx[7], by[7];
    unsigned emax;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < 7; ++k) bx[k] = by[k] = fx::zero96();
        emax = 0u;
    }
    template <int I>
    __device__ __forceinline__ void add(double v) {
        const fx::I96 n = fx::to96(v, emax);
        fx::add96(bx[cx_of(I) + 3], n);
        fx::add96(by[cy_of(I) + 3], n);
    }
    // The same for a positive v with 2^-28 <= v < 16 (biased exponent 995 .. 1026): no sign, no
    // right shift, no clamping, and nothing to report through emax.
    template <int I>
    __device__ __forceinline__ void add_in_range(double v) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
        const unsigned k = (hi >> 20) - 995u;
        const unsigned mh = (hi & 0xFFFFFu) | 0x100000u;
        const fx::I96 n{lo << k, __funnelshift_l(lo, mh, k), __funnelshift_l(mh, 0u, k)};
        fx::add96(bx[cx_of(I) + 3], n);
        fx::add96(by[cy_of(I) + 3], n);
    }
    __device__ __forceinline__ SiteSums finish(int* bad) const {
        using namespace fx;
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
        return SiteSums{to_double48(n0), to_double48(nx), to_double48(ny), to_double48(ne)};
    }
};

template <int I>
struct AddAll {
    __device__ __forceinline__ static void run(SumBins& b, const double* f) {
        AddAll<I - 1>::run(b, f);
        b.add<I>(f[I]);
    }
};
template <>
struct AddAll<-1> {
    __device__ __forceinline__ static void run(SumBins&, const double*) {}
};

__device__ __forceinline__ SiteSums site_sums(const double* f, int* bad) {
    SumBins b;
    b.init();
    AddAll<NPOP - 1>::run(b, f);
    return b.finish(bad);
}

struct SiteMoments {
    double rho, ux, uy, T;
};

// rho, u, T of one site (Sec. 3): rho = sum f, rho u = r sum f c, rho (u^2 + D T) = r^2 sum f |c|^2.
// The 2^-48 scale of the sums cancels in u and T.
__device__ __forceinline__ SiteMoments site_moments(const double* f, double r, double r2, int* bad) {
    const SiteSums s = site_sums(f, bad);
    const double inv = 1.0 / s.n0;
    const double rinv = r * inv;
    SiteMoments m;
    m.rho = s.n0 * 0x1p-48;
    m.ux = s.nx * rinv;
    m.uy = s.ny * rinv;
    const double u2 = m.ux * m.ux + m.uy * m.uy;
    m.T = 0.5 * fma(r2 * inv, s.ne, -u2);
    return m;
}

// Populations A .. B of the pull for (x, y), loaded together, then each added to the sums and
// written to the thread's shared-memory column fs[i * SITE_BLOCK] (population 0 kept in *f0).
template <int A, int I, int B>
__device__ __forceinline__ void batch_load(const double* __restrict__ src, double* g, int x, int y, int Lx, int Ly,
                                           int yp, long long plane) {
    if constexpr (I <= B) {
        g[I - A] = __ldg(src + plane_off(I, plane) + pull_index<I>(x, y, Lx, Ly, yp));
        batch_load<A, I + 1, B>(src, g, x, y, Lx, Ly, yp, plane);
    }
}
template <int A, int I, int B, bool kInRange>
__device__ __forceinline__ void batch_add_as(SumBins& acc, const double* g, double* fs, double* f0) {
    if constexpr (I <= B) {
        if constexpr (kInRange)
            acc.add_in_range<I>(g[I - A]);
        else
            acc.add<I>(g[I - A]);
        if constexpr (I == 0)
            *f0 = g[0];
        else
            fs[I * SITE_BLOCK] = g[I - A];
        batch_add_as<A, I + 1, B, kInRange>(acc, g, fs, f0);
    }
}
// Whether every value of the batch is positive with 2^-28 <= v < 16 (the range of add_in_range).
template <int A, int I, int B>
__device__ __forceinline__ bool batch_in_range(const double* g) {
    if constexpr (I <= B) {
        const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(g[I - A]) >> 32);
        return (hi - (995u << 20)) < (32u << 20) && batch_in_range<A, I + 1, B>(g);
    } else {
        return true;
    }
}
template <int A, int I, int B>
__device__ __forceinline__ void batch_add(SumBins& acc, const double* g, double* fs, double* f0) {
    if (batch_in_range<A, A, B>(g))
        batch_add_as<A, A, B, true>(acc, g, fs, f0);
    else
        batch_add_as<A, A, B, false>(acc, g, fs, f0);
}
// The same for a site's own populations (the in-place collide): population i at site + i plane.
template <int A, int I, int B>
__device__ __forceinline__ void own_load(const double* site, double* g, long long plane) {
    if constexpr (I <= B) {
        g[I - A] = site[plane_off(I, plane)];
        own_load<A, I + 1, B>(site, g, plane);
    }
}
template <int A, int B>
__device__ __forceinline__ void own_batch(const double* site, long long plane, SumBins& acc, double* fs, double* f0) {
    double g[B - A + 1];
    own_load<A, A, B>(site, g, plane);
    batch_add<A, A, B>(acc, g, fs, f0);
}

template <int A, int B>
__device__ __forceinline__ void pull_batch(const double* __restrict__ src, int x, int y, int Lx, int Ly, int yp,
                                           long long plane, SumBins& acc, double* fs, double* f0) {
    double g[B - A + 1];
    batch_load<A, A, B>(src, g, x, y, Lx, Ly, yp, plane);
    batch_add<A, A, B>(acc, g, fs, f0);
}

// The relaxation of one site toward the shifted equilibrium f_eq(rho, u*, T*), u* = u + tau g,
// T* = T + tau (1 - tau) |g|^2 / D (Sec. 3 model; ShellCoef gives the polynomial), written so that
// the FP64 pipe does as little as possible:
//   - pair variable b = lambda xi.u* with lambda = 1/4; with W = w rho / tau per shell,
//       W E = WA0 + b^2 (WA2 + C b^2),  W O = b (WB1 + C b^2),
//       WA0 = W A0, WA2 = 16 W A2, WB1 = 4 W B1, C = (32/3) W
//     (lambda = 1/4 makes the b^4 coefficient of E and the b^3 coefficient of O the same number C);
//   - the shell coefficients grouped by powers of xi^2 (D = 2, h = theta / 2, m = 1/2 - |u*|^2 / 4):
//       A0 = 2 m^2 + 1/2 + 2h (1 - 4m + 2h) + xi^2 h (2m - 4h) + xi^4 h^2 / 2,
//       A2 = m - 3h + xi^2 h / 2,  B1 = 2m - 4h + xi^2 h,
//     so that each shell costs 7-8 operations on site values shared by all shells (ShellRelax);
//   - b from U1 = lambda r u*_x and V1 = lambda r u*_y: for the shells (2,0), (2,2) and (3,0) the
//     pair variable is kappa beta with kappa = 2, 2, 3 and beta = U1, V1 or U1 +- V1, whose squares
//     are already at hand, and the powers of kappa are folded into that shell's constants
//     (W E = WA0 + beta^2 (k^2 WA2 + k^4 C beta^2), W O = beta (k WB1 + k^3 C beta^2)); the other
//     diagonal pairs take b from one FMA (2 U1 + V1, U1 + 3 V1, ...);
//   - the 2^-48 scale of the sums folded into the constants of StepParams (om48, lr2).
// Per pair, f'(+-c) = (1 - 1/tau) f(+-c) + W E +- W O: 7 FMAs after beta and beta^2.
struct Relax64 {
    double U1, V1, U1s, V1s;  // lambda r u*_x, lambda r u*_y and their squares
    double B11[2], S11[2];    // beta and beta^2 of the pairs (1, 1) and (1, -1)
    double rw, t, Rb, P1, P2, R0h;  // site terms of the shell coefficients
    double h;                 // (T* - 1) / 2
    double X;                 // temperature_sum: T = r^2 X / (2 n0) before the forcing shift
};

// 1 / x for a positive normal x (the site's n0, a density times 2^48): the hardware approximation
// (rcp.approx.ftz.f64; relative error below 2^-20 measured over the densities 0.05-20) refined by
// two Newton-Raphson steps y <- y + y (1 - x y), each of which squares the relative error, so the
// result is within about one ulp of 1 / x (on 4 M sampled densities it equalled the correctly
// rounded 1.0 / x). Non-positive or non-finite x are flagged by the caller and the value unused.
__device__ __forceinline__ double recip_nr(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
}

// X and a = 1 / n0 of the sums (the temperature is T = r^2 a X / 2), computed first so that the
// caller can check them before the coefficients.
__device__ __forceinline__ double temperature_sum(const SiteSums& s, double a) {
    return fma(-a, fma(s.nx, s.nx, s.ny * s.ny), s.ne);
}

// The site terms (everything shared by the shells); rw = rho / tau, or that factor times a power of
// two (the fixed-point path below), which every term that carries it then carries too.
__device__ __forceinline__ void relax_site_terms(const StepParams& P, const SiteSums& s, double a,
                                                 double rw, Relax64& R) {
    const double k = P.lr2 * a;                        // lambda r^2 / N0
    R.U1 = fma(s.nx, k, P.lrtgx);                      // lambda r u*_x
    R.V1 = fma(s.ny, k, P.lrtgy);
    R.U1s = R.U1 * R.U1;
    R.V1s = R.V1 * R.V1;
    const double h = fma(R.X, k, P.hdT);               // (T* - 1) / 2
    const double m = fma(R.U1s + R.V1s, P.mu4, 0.5);   // 1/2 - |u*|^2 / 4
    R.rw = rw;                                         // rho / tau (times 2^-E)
    R.h = h;
    R.t = R.rw * h;
    const double bq = fma(h, -2.0, m);                 // m - 2h
    R.Rb = R.rw * bq;
    R.P1 = R.t * bq;
    R.P2 = R.t * h;
    // rw A0(xi = 0) / 2 = rw (2 m^2 + 1/2 + 2h (1 - 4m + 2h)) / 2 = rw / 4 + t + Rb bq - 2 P2
    R.R0h = fma(-2.0, R.P2, fma(R.Rb, bq, fma(R.rw, 0.25, R.t)));
}

// The coefficients of shell S (S >= 1). The groupings of A2 and B1 give WA2 - WB1 = WB1 - 16 w t,
// so a pair forms its even factor from the odd one: with k = kappa and the shell's scaled
// constants (k WB1, k^2 WA2, k^3 C, k^4 C),
//   k^2 WA2 + k^4 C beta^2 = k q + DA,  q = k WB1 + k^3 C beta^2,  DA = k^2 (WA2 - WB1),
// and the shell keeps DA (one or two operations) instead of WA2 (two) and k^4 C (one).
struct ShellRelax {
    double WA0, DA, WB1, CO;  // CO = k^3 C
};

template <int S>
__device__ __forceinline__ ShellRelax shell_relax(const StepParams& P, const Relax64& R) {
    const ShellCoef& c = P.sh[S];
    ShellRelax q;
    q.WA0 = fma(c.q_a2, R.P2, fma(c.q_a1, R.P1, c.q_a0 * R.R0h));
    q.WB1 = fma(c.q_b1, R.t, c.q_b0 * R.Rb);                       // k WB1
    constexpr double k = shell_kappa(S);
    q.DA = fma(-c.q_e0, R.t, k == 1.0 ? q.WB1 : k * q.WB1);        // q_e0 = 16 k^2 w
    q.CO = c.q_co * R.rw;
    return q;
}

// beta and beta^2 of pair I (b = kappa beta, kappa = shell_kappa of its shell).
template <int I>
__device__ __forceinline__ void pair_base(const Relax64& R, double& b, double& b2) {
    constexpr int cx = cxh(I), cy = cyh(I);  // cx >= 0 for populations 1..18
    if constexpr (cy == 0) {
        b = R.U1;
        b2 = R.U1s;
    } else if constexpr (cx == 0) {
        b = R.V1;
        b2 = R.V1s;
    } else if constexpr (cx == cy || cx == -cy) {
        b = R.B11[cy > 0 ? 0 : 1];
        b2 = R.S11[cy > 0 ? 0 : 1];
    } else {
        if constexpr (cx == 1)
            b = fma(R.V1, (double)cy, R.U1);
        else
            b = fma(R.U1, (double)cx, cy > 0 ? R.V1 : -R.V1);
        b2 = b * b;
    }
}

// Relax pair I (populations I and I + NPAIR, opposite vectors) with its shell's coefficients;
// store(i, v) writes population i.
template <int I, class Store>
__device__ __forceinline__ void relax_pair(const double* f, const Relax64& R, const ShellRelax& c,
                                           double omc, Store& store) {
    double b, b2;
    pair_base<I>(R, b, b2);
    const double q = fma(b2, c.CO, c.WB1);
    constexpr double k = shell_kappa(shellh(I));
    const double e2 = k == 1.0 ? q + c.DA : fma(k, q, c.DA);  // k^2 WA2 + k^4 C beta^2
    const double we = fma(b2, e2, c.WA0);
    store(I, fma(omc, f[I], fma(b, q, we)));
    store(I + NPAIR, fma(omc, f[I + NPAIR], fma(-b, q, we)));
}

// All pairs I <= N of shell S.
template <int S, int N>
struct ShellPairs {
    template <class Store>
    __device__ __forceinline__ static void run(const double* f, const Relax64& R, const ShellRelax& c,
                                               double omc, Store& store) {
        ShellPairs<S, N - 1>::run(f, R, c, omc, store);
        if constexpr (shellh(N) == S) relax_pair<N>(f, R, c, omc, store);
    }
};
template <int S>
struct ShellPairs<S, 0> {
    template <class Store>
    __device__ __forceinline__ static void run(const double*, const Relax64&, const ShellRelax&, double,
                                               Store&) {}
};

template <int S, class Store>
__device__ __forceinline__ void relax_shell(const double* f, const StepParams& P, const Relax64& R,
                                            Store& store) {
    const ShellRelax c = shell_relax<S>(P, R);
    ShellPairs<S, NPAIR>::run(f, R, c, P.omc, store);
}

// All 37 populations, shell by shell in an order that ends the live ranges of U1^2, V1^2 and the
// (1, +-1) betas early: the axis shells, then (1,1) with (2,2), then the rest.
template <class Store>
__device__ __forceinline__ void relax_all(const double* f, const StepParams& P, Relax64& R,
                                          Store& store) {
    store(0, fma(P.omc, f[0], P.sh[0].q_a0 * R.R0h));
    relax_shell<1>(f, P, R, store);
    relax_shell<3>(f, P, R, store);
    relax_shell<6>(f, P, R, store);
    R.B11[0] = R.U1 + R.V1;
    R.B11[1] = R.U1 - R.V1;
    R.S11[0] = R.B11[0] * R.B11[0];
    R.S11[1] = R.B11[1] * R.B11[1];
    relax_shell<2>(f, P, R, store);
    relax_shell<5>(f, P, R, store);
    relax_shell<4>(f, P, R, store);
    relax_shell<7>(f, P, R, store);
}

// ---- the pair terms in fixed point on the integer pipe --------------------------------------
// GB300's FP64 pipe issues two instructions per clock per SM and binds this kernel; 64-bit integer
// multiplies and adds run on the integer pipes at many times that rate. So, inside a domain of
// moderate velocities and temperatures, each pair's equilibrium term G(+-c) = WA0 + b^2 e2 +- b q
// (relax_pair) is formed in two's-complement fixed point from the shell's FP64 coefficients, and
// only f' = (1 - 1/tau) f + G runs on the FP64 pipe: 2 FP64 instructions per pair instead of 7.
//   - b = lambda xi.u* (beta on the rescaled shells) in Q.64 (value x 2^64; |b| < 1/2), b^2 the
//     high word of b b (Q.64);
//   - two units per shell S: the coarse 2^-C(S) for k WB1, DA, k^3 C and q = WB1 + hi(CO b^2),
//     e2 = k q + DA (large numbers that only enter multiplied by b or b^2), and the fine 2^-F(S)
//     for WA0 and G; the products b^2 e2 and b q are taken from the exact 128-bit product F(S) -
//     C(S) bits below its high word, so G = WA0 + b^2 e2 +- b q keeps the fine unit;
//   - rho / tau = mant 2^E with mant in [1, 2): the FP64 site terms carry mant, and 2^E is applied
//     when G is rounded to FP64 (from_fixed; the rest population by an exponent shift).
// C(S) and F(S) are the largest scales that keep every intermediate of shell S below 2^61 over the
// domain |u*_x|, |u*_y| <= FX_UMAX and |T* - 1| / 2 <= FX_HB (bounds of the polynomials of
// shell_relax and relax_pair over that box, density factor below 2). Evaluated exactly in integer
// arithmetic against rational arithmetic, G then has the relative error of its final rounding
// (<= 2.2e-16 in the Rayleigh-Taylor and strong-flow regimes; the FP64 evaluation: 4e-16 - 6e-16).
// A site outside the domain takes the FP64 evaluation.
namespace fxp {

__host__ __device__ constexpr int coarse_of(int s) { return fx_coarse_unit(s); }
__host__ __device__ constexpr int fine_of(int s) { return fx_fine_unit(s); }

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// The domain test on bit patterns (integer compares; NaN fails it). P.fx_ub / P.fx_hb hold the bit
// patterns of lambda r FX_UMAX and FX_HB (set on the host).
__device__ __forceinline__ bool in_domain(const StepParams& P, const Relax64& R) {
    return abs_bits(R.U1) <= P.fx_ub && abs_bits(R.V1) <= P.fx_ub && abs_bits(R.h) <= P.fx_hb;
}

// g 2^-s rounded to FP64 on the integer pipe: to nearest, a tie rounded away from zero (within half
// an ulp like ties-to-even, and fewer instructions).
__device__ __forceinline__ double from_fixed(long long g, int s) {
    const unsigned long long sm = (unsigned long long)(g >> 63);      // 0 or all ones
    const unsigned long long u = ((unsigned long long)g ^ sm) - sm;   // |g|
    const int z = __clzll((long long)u);                              // 64 only for g = 0
    const unsigned long long w = u << (z & 63);                       // leading one at bit 63
    const unsigned long long sig = ((w >> 10) + 1ull) >> 1;           // 53 bits, or 2^53 on a carry
    const unsigned long long e1 = (unsigned long long)(1085 - z - s); // biased exponent - 1
    const unsigned long long bits = ((e1 << 52) + sig) | (sm & 0x8000000000000000ull);
    return u ? __longlong_as_double((long long)bits) : 0.0;
}

// v 2^S as a two's-complement integer, truncated toward zero (|v| 2^S < 2^62 in the domain).
__device__ __forceinline__ long long to_fixed_rt(double v, int S) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (e ? 0x0010000000000000ull : 0ull);
    const int sh = e - 1075 + S;  // v 2^S = m 2^sh
    const unsigned long long r = sh >= 0 ? (m << min(sh, 63)) : (m >> min(-sh, 63));
    return (long long)b < 0 ? -(long long)r : (long long)r;
}

// floor(a b 2^-64): the high word of the 128-bit product.
__device__ __forceinline__ long long hi(long long a, long long b) { return __mul64hi(a, b); }

// floor(a b 2^(D - 64)) for 1 <= D <= 63 given at run time.
__device__ __forceinline__ long long prod_at_rt(long long a, long long b, int D) {
    const unsigned long long h = (unsigned long long)__mul64hi(a, b);
    const unsigned long long l = (unsigned long long)a * (unsigned long long)b;
    return (long long)((h << D) | (l >> (64 - D)));
}

}  // namespace fxp

// The pairs in shell order with the coefficients of their pair variable (cx, cy) / kappa, and per
// shell its first pair, kappa and fixed-point units: the tables of the rolled pair loop below.
struct PairTable {
    int pop[NPAIR], bx[NPAIR], by[NPAIR];
    int first[NSHELL + 1], kappa[NSHELL], coarse[NSHELL], fine[NSHELL];
};
__host__ __device__ constexpr PairTable make_pair_table() {
    // (the rolled loop takes the pairs of a shell two at a time: every shell has 2 or 4)
    PairTable t{};
    int n = 0;
    for (int S = 0; S < NSHELL; ++S) {
        t.first[S] = n;
        t.kappa[S] = shell_kappa(S);
        t.coarse[S] = fxp::coarse_of(S);
        t.fine[S] = fxp::fine_of(S);
        for (int I = 1; I <= NPAIR; ++I)
            if (shellh(I) == S) {
                t.pop[n] = I;
                t.bx[n] = cxh(I) / shell_kappa(S);
                t.by[n] = cyh(I) / shell_kappa(S);
                ++n;
            }
    }
    t.first[NSHELL] = n;
    return t;
}
__constant__ PairTable c_pairs = make_pair_table();

// All 37 populations with the pair terms in fixed point (site terms carrying 2^-E, see above), as
// one compact loop over shells and their pairs: the populations are read from the thread's column
// fs[i * SITE_BLOCK] of the block's shared-memory copy, so one loop body serves every pair (the
// fully unrolled form overflowed the instruction cache). f0 is the rest population.
template <class Store>
__device__ __forceinline__ void relax_all_fx(const double* fs, double f0, const StepParams& P, const Relax64& R,
                                             int E, Store& store) {
    using namespace fxp;
    // rest population: the shell-0 term (a positive normal number) scaled back by 2^E in its exponent
    const double g0 = P.sh[0].q_a0 * R.R0h;
    store(0, fma(P.omc, f0, __longlong_as_double(__double_as_longlong(g0) + ((long long)E << 52))));
    const long long U = to_fixed_rt(R.U1, 64), V = to_fixed_rt(R.V1, 64);
    // the site terms of the integer products in fixed point (bounds over the domain: |t| < 1/2,
    // |Rb| and the density factor's mantissa < 2)
    const long long mq = to_fixed_rt(R.rw, 62), T = to_fixed_rt(R.t, 64), Rb = to_fixed_rt(R.Rb, 62);
#pragma unroll 1
    for (int S = 1; S < NSHELL; ++S) {
        const long long k = c_pairs.kappa[S];
        const int sf = c_pairs.fine[S], D = sf - c_pairs.coarse[S];
        // shell_relax's coefficients: WA0 in FP64 (3 FP64 instructions), rounded to the fine unit;
        // k WB1, DA and k^3 C as integer products of the host's fixed-point constants (ShellFx) and
        // the site terms, in the coarse unit (measured fastest: all four as integer products, or
        // all but k^3 C in FP64, were 5 % and 3 % slower)
        const ShellFx& q = P.shfx[S];
        const ShellCoef& c = P.sh[S];
        const long long xA0 = to_fixed_rt(fma(c.q_a2, R.P2, fma(c.q_a1, R.P1, c.q_a0 * R.R0h)), sf);
        const long long xB1 = hi(q.b1, T) + hi(q.b0, Rb);
        const long long xDA = k * xB1 - hi(q.e0, T);
        const long long xCO = hi(q.co, mq);
        const int se = sf - E;
        // two pairs per iteration (every shell has an even number of pairs): two independent chains
#pragma unroll 1
        for (int j = c_pairs.first[S]; j < c_pairs.first[S + 1]; j += 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int I = c_pairs.pop[j + h];
                const long long b = (long long)c_pairs.bx[j + h] * U + (long long)c_pairs.by[j + h] * V;
                const long long b2 = hi(b, b);
                const long long q = xB1 + hi(xCO, b2);
                const long long e2 = k * q + xDA;
                const long long we = xA0 + prod_at_rt(b2, e2, D);
                const long long bq = prod_at_rt(b, q, D);
                store(I, fma(P.omc, fs[I * SITE_BLOCK], from_fixed(we + bq, se)));
                store(I + NPAIR, fma(P.omc, fs[(I + NPAIR) * SITE_BLOCK], from_fixed(we - bq, se)));
            }
        }
    }
}

// The same relaxation in FP64 throughout (sites outside the fixed-point domain), as the same compact
// loop over the shared-memory copy: per pair b from the table's (cx, cy) / kappa, then relax_pair's
// arithmetic.
template <class Store>
__device__ __noinline__ void relax_all_fp64_rolled(const double* fs, double f0, const StepParams& P,
                                                   const Relax64& R, Store& store) {
    store(0, fma(P.omc, f0, P.sh[0].q_a0 * R.R0h));
#pragma unroll 1
    for (int S = 1; S < NSHELL; ++S) {
        const ShellCoef& c = P.sh[S];
        const double k = (double)c_pairs.kappa[S];
        const double WA0 = fma(c.q_a2, R.P2, fma(c.q_a1, R.P1, c.q_a0 * R.R0h));
        const double WB1 = fma(c.q_b1, R.t, c.q_b0 * R.Rb);
        const double DA = fma(-c.q_e0, R.t, k * WB1);
        const double CO = c.q_co * R.rw;
#pragma unroll 1
        for (int j = c_pairs.first[S]; j < c_pairs.first[S + 1]; ++j) {
            const int I = c_pairs.pop[j];
            const double b = fma((double)c_pairs.bx[j], R.U1, (double)c_pairs.by[j] * R.V1);
            const double b2 = b * b;
            const double q = fma(b2, CO, WB1);
            const double we = fma(b2, fma(k, q, DA), WA0);
            store(I, fma(P.omc, fs[I * SITE_BLOCK], fma(b, q, we)));
            store(I + NPAIR, fma(P.omc, fs[(I + NPAIR) * SITE_BLOCK], fma(-b, q, we)));
        }
    }
}

// Collide site (x, y) with populations f (Sec. 3: moments, shifted equilibrium, BGK relaxation):
// store(i, o, v) writes population i at element offset o of its plane (the site's own offset,
// then the wall halo rows the site feeds). Shared by the fused step and the collide kernel, so the
// two give the same bits.
template <class Store>
__device__ __forceinline__ void collide_from_sums(const SiteSums& s, int bad, double f0, const double* fs,
                                                  const StepParams& P, int x, int y, int* __restrict__ flag,
                                                  Store&& store);

// Collide with the populations f in registers (copied to the thread's shared-memory column first).
template <class Store>
__device__ __forceinline__ void collide_site(const double* f, double* fs, const StepParams& P, int x, int y,
                                             int* __restrict__ flag, Store&& store) {
    int bad;
    const SiteSums s = site_sums(f, &bad);
#pragma unroll
    for (int i = 1; i < NPOP; ++i) fs[i * SITE_BLOCK] = f[i];  // this thread's column of the block's copy
    collide_from_sums(s, bad, f[0], fs, P, x, y, flag, store);
}

// The collide of a site whose moment sums are s (status bits bad), rest population f0 and other
// populations in the thread's shared-memory column fs.
template <class Store>
__device__ __forceinline__ void collide_from_sums(const SiteSums& s, int bad, double f0, const double* fs,
                                                  const StepParams& P, int x, int y, int* __restrict__ flag,
                                                  Store&& store) {
    const double a = recip_nr(s.n0);
    Relax64 R;
    R.X = temperature_sum(s, a);
    if (bad_positive(s.n0) || bad_positive(R.X) || bad) atomicOr(flag, bad ? bad : 1);
    // rho / tau = mant 2^E, mant in [1, 2): the site terms carry mant, the pair terms' conversion
    // back to FP64 adds E to the exponent
    const double rw = s.n0 * P.om48;
    const unsigned long long rb = (unsigned long long)__double_as_longlong(rw);
    const int E = (int)((rb >> 52) & 0x7FFu) - 1023;
    relax_site_terms(P, s, a, __longlong_as_double((long long)((rb & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull)),
                     R);

    const long long o = (long long)(y + HALO) * P.Lx + x;
    auto own = [&](int i, double v) { store(i, o, v); };
    if (fxp::in_domain(P, R)) {
        relax_all_fx(fs, f0, P, R, E, own);
    } else {  // outside the fixed-point formats: the FP64 evaluation with rho / tau itself
        relax_site_terms(P, s, a, rw, R);
        relax_all_fp64_rolled(fs, f0, P, R, own);
    }

    // wall halo rows from this site's post-collision fields (rho, u + g, T)
    if (!P.y_periodic && (y < HALO || y >= P.Ly - HALO)) {
        const double ra = P.r * a;
        const double T = (P.r2 * 0.5) * a * R.X;
        write_wall_rows(P, x, y, s.n0 * 0x1p-48, fma(s.nx, ra, P.gx), fma(s.ny, ra, P.gy), T, flag,
                        store);
    }
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

// Sites site0 .. site1 - 1 (the whole lattice, or a band of rows of a slab). Three blocks (12 warps)
// per SM: the register cap that keeps the occupancy of the FP64-only version.
constexpr int STEP_BLOCKS_PER_SM = 5;
__global__ void __launch_bounds__(SITE_BLOCK, STEP_BLOCKS_PER_SM)
step_fp64_kernel(const double* __restrict__ src, double* __restrict__ dst, const StepParams P,
                 int* __restrict__ flag, int site0, int site1) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = site0 + blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= site1) return;
    const int y = row_of(site, P);
    const int x = site - y * Lx;
    const long long plane = P.plane;

    // the pull in two batches of loads (the compiler barrier keeps the second batch after the first's
    // consumers), each population added to the moment sums and staged in shared memory as it is
    // used: about half the population registers of loading all 37 at once
    __shared__ double fs[NPOP * SITE_BLOCK];
    double* col = fs + threadIdx.x;
    SumBins acc;
    acc.init();
    double f0;
    pull_batch<0, 18>(src, x, y, Lx, Ly, P.y_periodic, plane, acc, col, &f0);
    asm volatile("" ::: "memory");
    pull_batch<19, NPOP - 1>(src, x, y, Lx, Ly, P.y_periodic, plane, acc, col, &f0);
    int bad;
    const SiteSums s = acc.finish(&bad);
    collide_from_sums(s, bad, f0, col, P, x, y, flag,
                      [&](int i, long long o, double v) { __stcs(dst + plane_off(i, plane) + o, v); });
}

// Collide only, in place (the paper's separate collide kernel, Sec. 3-5 and Table 1): each thread
// reads the 37 populations of its own site, relaxes them exactly as the fused step does, writes
// them back, and on rows 0..2 and Ly-3..Ly-1 writes the wall halo rows. After propagate this gives
// the same populations, bit for bit, as one fused step.
__global__ void __launch_bounds__(SITE_BLOCK, STEP_BLOCKS_PER_SM)
collide_fp64_kernel(double* __restrict__ f, const StepParams P, int* __restrict__ flag) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = row_of(site, P);
    const int x = site - y * Lx;
    const long long plane = P.plane;
    const long long o = (long long)(y + HALO) * Lx + x;
    __shared__ double fs[NPOP * SITE_BLOCK];
    double* col = fs + threadIdx.x;
    SumBins acc;
    acc.init();
    double f0;
    own_batch<0, 18>(f + o, plane, acc, col, &f0);
    asm volatile("" ::: "memory");
    own_batch<19, NPOP - 1>(f + o, plane, acc, col, &f0);
    int bad;
    const SiteSums s = acc.finish(&bad);
    collide_from_sums(s, bad, f0, col, P, x, y, flag,
                      [&](int i, long long oh, double val) { __stcs(f + plane_off(i, plane) + oh, val); });
}

__global__ void __launch_bounds__(SITE_BLOCK)
propagate_fp64_kernel(const double* __restrict__ src, double* __restrict__ dst, const StepParams P) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = row_of(site, P);
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
    const int y = row_of(site, P);
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
    const int y = row_of(site, P);
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
    step_fp64_kernel<<<site_blocks(P), SITE_BLOCK, 0, s>>>(src, dst, P, flag, 0, P.Lx * P.Ly);
    return cudaGetLastError();
}

cudaError_t launch_step_fp64_rows(const double* src, double* dst, const StepParams& P, int* flag,
                                  int row0, int row1, cudaStream_t s) {
    if (row1 <= row0) return cudaSuccess;
    const int n = (row1 - row0) * P.Lx;
    step_fp64_kernel<<<(n + SITE_BLOCK - 1) / SITE_BLOCK, SITE_BLOCK, 0, s>>>(src, dst, P, flag, row0 * P.Lx,
                                                                             row1 * P.Lx);
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
