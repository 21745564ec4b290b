// d2q37_gpu.cuh -- D2Q37 model tables and per-step coefficients of the CUDA path.
//
// The model (paper, Sec. 3): 37 populations per site, hopping up to three lattice points, with an
// equilibrium that yields the perfect-gas law p = rho T. The velocity set, weights and Hermite
// equilibrium are those of the D2Q37 references the paper cites; this header is the CUDA path's
// own copy (the CPU oracle keeps a separate one).
//
// Population order used on the device and in the C ABI:
//   0        rest particle
//   1 .. 18  one vector of each opposite pair, shell by shell
//   19 .. 36 population 18 + k moves opposite to population k
// Pairing opposite vectors lets the collide evaluate the even and odd parts of the equilibrium
// polynomial once per pair (f_eq(+c) and f_eq(-c) differ only in the sign of the odd part).
#pragma once

#include <cstddef>
#include <cstdint>

namespace lbg {

constexpr int NPOP = 37;
constexpr int NPAIR = 18;
constexpr int NSHELL = 8;
constexpr int HALO = 3;
constexpr double DIM = 2.0;
// Domain of the FP64 step's fixed-point pair terms (step_fp64.cu): |u*_x|, |u*_y| <= 0.2, i.e.
// |lambda r u*| components <= 0.25 r 0.2, and |h| = |T* - 1| / 2 <= 0.2 (T* in [0.6, 1.4]).
constexpr double FX_UMAX = 0.2;
constexpr double FX_HB = 0.2;
// Its per-shell units: values in units of 2^-coarse (k WB1, DA, k^3 C, q, e2) and 2^-fine (WA0 and
// the pair term G); the largest scales that keep every intermediate below 2^61 over the domain.
__host__ __device__ constexpr int fx_coarse_unit(int s) {
    constexpr int t[NSHELL] = {0, 59, 60, 59, 64, 63, 63, 67};
    return t[s];
}
__host__ __device__ constexpr int fx_fine_unit(int s) {
    constexpr int t[NSHELL] = {0, 62, 63, 64, 65, 67, 69, 68};
    return t[s];
}

// Tables are constexpr functions (usable in host code, device code and constant expressions).
// Lattice vectors of populations 0..18; 19..36 are their negatives.
__host__ __device__ constexpr int cxh(int i) {
    constexpr int t[NPAIR + 1] = {0, 1, 0, 1, 1, 2, 0, 2, 2, 1, 1, 2, 2, 3, 0, 3, 3, 1, 1};
    return t[i];
}
__host__ __device__ constexpr int cyh(int i) {
    constexpr int t[NPAIR + 1] = {0, 0, 1, 1, -1, 0, 2, 1, -1, 2, -2, 2, -2, 0, 3, 1, -1, 3, -3};
    return t[i];
}
// Shell of populations 0..18 (shell s = |c|-class: (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1)).
__host__ __device__ constexpr int shellh(int i) {
    constexpr int t[NPAIR + 1] = {0, 1, 1, 2, 2, 3, 3, 4, 4, 4, 4, 5, 5, 6, 6, 7, 7, 7, 7};
    return t[i];
}
// |c|^2 per shell.
__host__ __device__ constexpr int shell_c2(int s) {
    constexpr int t[NSHELL] = {0, 1, 2, 4, 5, 8, 9, 10};
    return t[s];
}
// Per shell, the factor kappa between the pair variable of the FP64 step and the base variable it
// is evaluated from (1 except the shells (2,0), (2,2), (3,0); step_fp64.cu, pair_base).
__host__ __device__ constexpr int shell_kappa(int s) {
    constexpr int t[NSHELL] = {1, 1, 1, 2, 1, 2, 3, 1};
    return t[s];
}
// D2Q37 quadrature weights per shell.
__host__ __device__ constexpr double shell_w(int s) {
    constexpr double t[NSHELL] = {
        0.23315066913235250228650, 0.10730609154221900241246, 0.05766785988879488203006,
        0.01420821615845075026469, 0.00535304900051377523273, 0.00101193759267357547541,
        0.00024530102775771734547, 0.00028341425299419821740};
    return t[s];
}

__host__ __device__ constexpr int cx_of(int i) { return i <= NPAIR ? cxh(i) : -cxh(i - NPAIR); }
__host__ __device__ constexpr int cy_of(int i) { return i <= NPAIR ? cyh(i) : -cyh(i - NPAIR); }
__host__ __device__ constexpr int shell_of(int i) { return i <= NPAIR ? shellh(i) : shellh(i - NPAIR); }

// Per-shell polynomial coefficients of the Hermite equilibrium, written for one pair (+c, -c)
// with a = xi.u, theta = T - 1, u2 = |u|^2 and X = xi^2 = r^2 |c|^2:
//   f_eq(+-c) / (w rho) = E(a^2) +- O(a)
//   E = A0 + A2 a^2 + a^4 / 24,  O = a (B1 + a^2 / 6)
//   A0 = 1 - u2/2 + u2^2/8 + alpha theta + beta theta u2 + gamma theta^2
//   A2 = 1/2 - u2/4 + delta theta,  B1 = 1 - u2/2 + eps theta
// with alpha = (X - D)/2, beta = (D + 2 - X)/4, gamma = (X^2 - 2(D + 2)X + D(D + 2))/8,
// delta = (X - D - 4)/4, eps = (X - D - 2)/2. This is the same polynomial as the 4th-order
// expansion, regrouped by powers of a.
struct ShellCoef {
    double w, alpha, beta, gamma, delta, eps;
    // constants of the FP64 step's relaxation (step_fp64.cu, shell_relax), X = xi^2 and
    // k = shell_kappa: W A0 = q_a0 R0 + q_a1 P1 + q_a2 P2, 4 k W B1 = q_b0 Rb + q_b1 t,
    // 16 k^2 W (A2 - B1 / 4) = k (4 k W B1) - q_e0 t, k^3 C = q_co rho / tau, with q_a0 = 2w,
    // q_a1 = 2wX, q_a2 = wX^2/2, q_b0 = 8 k w, q_b1 = 4 k wX, q_e0 = 16 k^2 w, q_co = 32 k^3 w/3
    double q_a0, q_a1, q_a2, q_b0, q_b1, q_e0, q_co;
};

// FP32 copies of the shell coefficients for the FP32 kernels (converting doubles on the device
// would run on GB300's narrow FP64 pipe).
struct ShellCoef32 {
    float w, alpha, beta, gamma, delta, eps;
    // constants of the FP32 relaxation (site_fp32dev.cuh, relax_coefficients32), X = xi^2:
    // q_a0 = w, q_a1 = 2wX, q_a2 = wX^2/2, q_e0 = 16w, q_e1 = 8wX, q_b0 = 8w, q_b1 = 4wX, q_c = 32w/3
    float q_a0, q_a1, q_a2, q_e0, q_e1, q_b0, q_b1, q_c;
};

// A shell's constants for the fixed-point pair terms of the FP64 step (step_fp64.cu), rounded to
// integers on the host: each is the high word's factor for a site term in the stated format, so
//   k WB1 = hi(b1, t Q.64) + hi(b0, Rb Q.62),  DA = k (k WB1) - hi(e0, t Q.64),
//   k^3 C = hi(co, mantissa of rho/tau Q.62)                      in 2^-coarse:
// b1 = q_b1 2^coarse, b0 = q_b0 2^(coarse + 2), e0 = q_e0 2^coarse, co = q_co 2^(coarse + 2)
// (all below 2^62).
struct ShellFx {
    long long b1, b0, e0, co;
};

// Everything a step kernel needs, passed by value as a kernel parameter.
struct StepParams {
    int Lx, Ly;
    int y_periodic;
    int wall_mode;         // lb_wall_mode: 0 rest-equilibrium halo rows, 1 mirror closure
    int cut;               // slab of a larger lattice: bit 0 = no wall below row 0, bit 1 = none
                           // above row Ly - 1 (those halo rows are ghost rows another slab fills)
    long long plane;       // elements per population plane, (Ly + 2*HALO) * Lx
    // row of a site index n < 2^31 without a division: y = (n * row_m) >> row_s (row_of)
    unsigned row_m;
    int row_s;
    double r;              // thermal scale, xi = r c
    double r2;             // r^2
    double omega;          // 1 / tau
    double omc;            // 1 - 1/tau
    double gx, gy;         // gravity
    double tgx, tgy;       // tau * g
    double dT_force;       // tau (1 - tau) |g|^2 / D
    // FP64 step (relax_site_terms, lambda = 1/4): lambda r^2, lambda r tau g, (dT_force - 1) / 2,
    // -1 / (4 lambda^2 r^2), 2^-48 / tau
    double lr2, lrtgx, lrtgy, hdT, mu4, om48;
    // bit patterns of the fixed-point pair terms' domain bounds (step_fp64.cu, fxp): |lambda r u*|
    // components <= FX_UB, |h| <= FX_HB
    unsigned long long fx_ub, fx_hb;
    // per shell the constants of shell_relax in fixed point (ShellFx)
    ShellFx shfx[NSHELL];
    double T_bot, T_top;   // wall temperatures below row 0 and above row Ly - 1
    ShellCoef sh[NSHELL];
    double wall_bot[NPOP]; // rest equilibrium per unit density at T_bottom, per population
    double wall_top[NPOP]; // same at T_top
    // FP32 copies of the scalars above and of the shell coefficients
    float r_f, r2_f, omega_f, omc_f, gx_f, gy_f, tgx_f, tgy_f, dT_force_f, lr_f;  // lr_f = r / 4
    ShellCoef32 sh32[NSHELL];
    // byte offsets for 4-byte populations: pull_b32[i] = 4 (i plane - c_iy Lx - c_ix) from a site's
    // own element (valid where the pull does not wrap), plane_b32[i] = 4 i plane
    long long pull_b32[NPOP];
    long long plane_b32[NPOP];
};

// y = n / Lx for 0 <= n < 2^31 by a multiply and a shift (Granlund & Montgomery 1994, Thm. 4.2:
// with l = ceil(log2 Lx) and m = ceil(2^(31 + l) / Lx) < 2^32, floor(n m / 2^(31 + l)) = floor(n / Lx)
// for all n < 2^31). Keeps the integer division's float conversions off the FP64 pipe.
__device__ __forceinline__ int row_of(int n, const StepParams& P) {
    return (int)(((unsigned long long)(unsigned)n * P.row_m) >> P.row_s);
}

// The equilibrium of one site (Sec. 3 model: 4th-order Hermite expansion, D = 2) in FP64, handed
// population by population to sink(i, f_eq_i) in the library's order. With theta = T - 1,
// u2 = |u|^2 and a = xi.u, per shell f_eq(+-c) = w rho (E +- O), E = A0 + a^2 (A2 + a^2 / 24),
// O = a (B1 + a^2 / 6). Used on the wall rows only.
template <class Sink>
__device__ __forceinline__ void for_each_equilibrium(const StepParams& P, double rho, double ux,
                                                     double uy, double T, Sink&& sink) {
    const double th = T - 1.0;
    const double u2 = ux * ux + uy * uy;
    const double a00 = fma(u2, fma(u2, 0.125, -0.5), 1.0);
    const double a20 = fma(u2, -0.25, 0.5);
    const double b10 = fma(u2, -0.5, 1.0);
    const double thu2 = th * u2, th2 = th * th;
    const double urx = P.r * ux, ury = P.r * uy;
    sink(0, rho * P.sh[0].w * fma(P.sh[0].gamma, th2, fma(P.sh[0].beta, thu2, fma(P.sh[0].alpha, th, a00))));
#pragma unroll
    for (int i = 1; i <= NPAIR; ++i) {
        const ShellCoef& c = P.sh[shellh(i)];
        const double A0 = fma(c.gamma, th2, fma(c.beta, thu2, fma(c.alpha, th, a00)));
        const double A2 = fma(c.delta, th, a20);
        const double B1 = fma(c.eps, th, b10);
        const double a = fma((double)cxh(i), urx, (double)cyh(i) * ury);
        const double a2 = a * a;
        const double e = fma(a2, fma(a2, 1.0 / 24.0, A2), A0);
        const double o = a * fma(a2, 1.0 / 6.0, B1);
        const double W = rho * c.w;
        sink(i, W * (e + o));
        sink(i + NPAIR, W * (e - o));
    }
}

// Halo row y_h (0..2 below the lattice, Ly+3..Ly+5 above, in padded row numbers) of the mirror
// closure: the equilibrium at the mirror site's density, the opposite of its velocity and the
// temperature 2 T_wall - T. Returns false (and writes nothing) when that temperature is not
// positive. The caller stores sink(i, f_eq_i).
template <class Sink>
__device__ __forceinline__ bool mirror_halo(const StepParams& P, bool bottom, double rho, double ux,
                                            double uy, double T, Sink&& sink) {
    const double Th = 2.0 * (bottom ? P.T_bot : P.T_top) - T;
    if (!(Th > 0.0)) return false;
    for_each_equilibrium(P, rho, -ux, -uy, Th, sink);
    return true;
}

// Half-step fields from the moments (u, T) of a post-collision state: the shifted-equilibrium
// collision adds g to u and keeps T, and the mean of the pre- and post-collision momentum and
// energy gives u - g / 2 and T + |g|^2 / (4 D).
__device__ __forceinline__ void half_step_shift(const StepParams& P, double& ux, double& uy, double& T) {
    ux -= 0.5 * P.gx;
    uy -= 0.5 * P.gy;
    T += (P.gx * P.gx + P.gy * P.gy) / (4.0 * DIM);
}

// The wall halo rows that interior site (x, y) feeds, written after its collide: halo row -1-y if
// y < 3, halo row Ly + (Ly-1-y) if y >= Ly - 3. (rho, ux, uy, T) are the site's post-collision
// fields. store(i, o, v) writes FP64 value v of population i at element offset o of a plane.
// Rest closure: rho times the rest equilibrium per unit density at the wall temperature; mirror
// closure: mirror_halo (a non-positive reflected temperature sets flag bit 1 and that halo site
// gets the rest closure instead). A side cut from a neighbouring slab (P.cut) has no wall: its halo
// rows are ghost rows that the exchange between slabs writes.
template <class Store>
__device__ __forceinline__ void write_wall_rows(const StepParams& P, int x, int y, double rho, double ux,
                                                double uy, double T, int* __restrict__ flag,
                                                Store&& store) {
    if (P.y_periodic) return;
    const int Lx = P.Lx, Ly = P.Ly;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const bool bottom = side == 0;
        if (bottom ? (y >= HALO || (P.cut & 1)) : (y < Ly - HALO || (P.cut & 2))) continue;
        const long long o = bottom ? (long long)(HALO - 1 - y) * Lx + x
                                   : (long long)(Ly + HALO + (Ly - 1 - y)) * Lx + x;
        if (P.wall_mode == 1) {
            if (mirror_halo(P, bottom, rho, ux, uy, T, [&](int i, double v) { store(i, o, v); })) continue;
            atomicOr(flag, 1);  // not reflectable: flag it and fall back to the rest closure
        }
        const double* wr = bottom ? P.wall_bot : P.wall_top;
#pragma unroll
        for (int i = 0; i < NPOP; ++i) store(i, o, rho * wr[i]);
    }
}

}  // namespace lbg
