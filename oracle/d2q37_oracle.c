/*
 * d2q37_oracle.c -- plain, slow FP64 CPU oracle of the D2Q37 lattice-Boltzmann time step.
 *
 * TEST INFRASTRUCTURE ONLY. This file exists to check the CUDA path. Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or constant with the CUDA sources; the only thing both sides share is the
 * seeded generator of macroscopic input fields.
 *
 * What the method computes (paper, Sec. 3): populations sitting on the sites of a regular
 * lattice first propagate from site to site and then collide, which mixes them; no site
 * depends on another within either phase. The D2Q37 model has 37 populations per site that
 * hop up to three lattice points (Sec. 3, Fig. 1) and enforces the perfect-gas equation of
 * state p = rho T. Propagate is a pull (Sec. 4, Fig. 3 listing): each population of the new
 * lattice is read from the old lattice at the site displaced by a fixed per-population offset.
 *
 * The paper defers the model's constants, equilibrium, collision operator, forcing and walls to
 * its references. The readings used here (each function states its own):
 *   - velocities c_i: the 8 shells (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1) with all
 *     sign/axis permutations, 37 in total; thermal velocities xi_i = r c_i;
 *   - weights: per shell, from the D2Q37 quadrature (exact for moments of degree <= 9);
 *   - r = 1 / sqrt(sum_i w_i c_ix^2), so that the reference temperature is 1;
 *   - equilibrium: 4th-order Hermite expansion of the Maxwellian, D = 2;
 *   - collision: single-relaxation-time BGK with relaxation time tau;
 *   - gravity g: the equilibrium is evaluated at u + tau g and T + tau (1 - tau) |g|^2 / D;
 *   - walls (top/bottom): three halo rows per wall hold the equilibrium at rest, at the wall
 *     temperature and at the density of the mirror interior row; an alternative mirror closure
 *     (opposite velocity, temperature reflected about the wall value) is also provided;
 *   - reported fields: moments of the stored populations; optionally the half-step fields that
 *     average the pre- and post-collision momentum and energy;
 *   - periodic in x (optionally in y, a test mode with no walls);
 *   - one step = write wall halos, propagate (pull), collide.
 *
 * Layout (the oracle's own, site-major): f[((y + 3) * Lx + x) * 37 + i], y in [-3, Ly + 2],
 * i.e. three halo rows below row 0 and three above row Ly - 1. Interior-only arrays drop the
 * halo rows: f[(y * Lx + x) * 37 + i].
 *
 * Summation runs over i = 0..36 in table order; build with -ffp-contract=off so no product is
 * fused into an addition.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NPOP 37
#define NSHELL 8
#define HALO 3
#define DIM 2.0

/* Shell representatives (a, b), a >= b >= 0. */
static const int shell_rep[NSHELL][2] = {
    {0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}, {3, 0}, {3, 1}};

/* Per-shell weights of the D2Q37 quadrature (the model of the paper's references [JFM, POF]). */
static const double shell_w[NSHELL] = {
    0.23315066913235250228650, 0.10730609154221900241246, 0.05766785988879488203006,
    0.01420821615845075026469, 0.00535304900051377523273, 0.00101193759267357547541,
    0.00024530102775771734547, 0.00028341425299419821740};

static int CX[NPOP], CY[NPOP];
static double W[NPOP];
static double R;
static int ready = 0;

static void setup(void) {
    if (ready) return;
    int n = 0;
    for (int s = 0; s < NSHELL; ++s) {
        const int a = shell_rep[s][0], b = shell_rep[s][1];
        const int cand[8][2] = {{a, b}, {b, a}, {-a, b}, {-b, a}, {a, -b}, {b, -a}, {-a, -b}, {-b, -a}};
        for (int k = 0; k < 8; ++k) {
            int dup = 0;
            for (int j = 0; j < n; ++j)
                if (CX[j] == cand[k][0] && CY[j] == cand[k][1]) dup = 1;
            if (!dup) {
                CX[n] = cand[k][0];
                CY[n] = cand[k][1];
                W[n] = shell_w[s];
                ++n;
            }
        }
    }
    double m2 = 0.0;
    for (int i = 0; i < NPOP; ++i) m2 += W[i] * (double)(CX[i] * CX[i]);
    R = 1.0 / sqrt(m2);
    ready = 1;
}

int or_npop(void) { return NPOP; }

/* Velocity table, weights and the scale r (xi = r c). */
void or_velocity_set(int* cx, int* cy, double* w, double* r) {
    setup();
    for (int i = 0; i < NPOP; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = W[i];
    }
    *r = R;
}

/* Equilibrium of one site: 4th-order Hermite expansion of the Maxwellian at (rho, u, T), D = 2,
 * theta = T - 1, with eu = xi.u, u2 = u.u and xi2 = xi.xi:
 *   f_eq = w rho [ 1 + eu + (eu^2 - u2 + theta (xi2 - D)) / 2
 *                  + eu (eu^2 - 3 u2 + 3 theta (xi2 - D - 2)) / 6
 *                  + ( eu^4 - 6 eu^2 u2 + 3 u2^2 + 6 theta (eu^2 (xi2 - D - 4) + u2 (D + 2 - xi2))
 *                      + 3 theta^2 (xi2^2 - 2 (D + 2) xi2 + D (D + 2)) ) / 24 ].
 * The paper names the model (Sec. 3: perfect gas p = rho T) and defers the formula to its
 * references; this is the standard Hermite form of those references. */
static void feq_site(double rho, double ux, double uy, double T, double* out) {
    const double th = T - 1.0;
    const double u2 = ux * ux + uy * uy;
    for (int i = 0; i < NPOP; ++i) {
        const double xx = R * CX[i], xy = R * CY[i];
        const double eu = xx * ux + xy * uy;
        const double xi2 = xx * xx + xy * xy;
        const double h1 = eu;
        const double h2 = 0.5 * (eu * eu - u2 + th * (xi2 - DIM));
        const double h3 = eu / 6.0 * (eu * eu - 3.0 * u2 + 3.0 * th * (xi2 - DIM - 2.0));
        const double h4 = (eu * eu * eu * eu - 6.0 * eu * eu * u2 + 3.0 * u2 * u2 +
                           6.0 * th * (eu * eu * (xi2 - DIM - 4.0) + u2 * (DIM + 2.0 - xi2)) +
                           3.0 * th * th * (xi2 * xi2 - 2.0 * (DIM + 2.0) * xi2 + DIM * (DIM + 2.0))) /
                          24.0;
        out[i] = W[i] * rho * (1.0 + h1 + h2 + h3 + h4);
    }
}

/* Macroscopic fields of one site: rho = sum f, rho u = sum f xi, rho (u^2 + D T) = sum f xi^2. */
static void moments_site(const double* f, double* rho, double* ux, double* uy, double* T) {
    double m0 = 0.0, mx = 0.0, my = 0.0, me = 0.0;
    for (int i = 0; i < NPOP; ++i) {
        const double xx = R * CX[i], xy = R * CY[i];
        m0 += f[i];
        mx += f[i] * xx;
        my += f[i] * xy;
        me += f[i] * (xx * xx + xy * xy);
    }
    const double vx = mx / m0, vy = my / m0;
    *rho = m0;
    *ux = vx;
    *uy = vy;
    *T = (me - m0 * (vx * vx + vy * vy)) / (DIM * m0);
}

/* Collide one site in place: BGK relaxation towards the equilibrium evaluated at the shifted
 * velocity u + tau g and temperature T + tau (1 - tau) |g|^2 / D (forcing by a shifted
 * equilibrium; exact consequences: the momentum changes by rho g, rho and T do not change). */
static void collide_site(double* f, double tau, double gx, double gy) {
    double rho, ux, uy, T, fe[NPOP];
    moments_site(f, &rho, &ux, &uy, &T);
    const double uxs = ux + tau * gx;
    const double uys = uy + tau * gy;
    const double Ts = T + tau * (1.0 - tau) * (gx * gx + gy * gy) / DIM;
    feq_site(rho, uxs, uys, Ts, fe);
    for (int i = 0; i < NPOP; ++i) f[i] = f[i] - (f[i] - fe[i]) / tau;
}

/* f[n][37] := equilibrium of each site's (rho, ux, uy, T). */
void or_equilibrium(size_t n, const double* rho, const double* ux, const double* uy,
                    const double* T, double* f) {
    setup();
    for (size_t s = 0; s < n; ++s) feq_site(rho[s], ux[s], uy[s], T[s], f + s * NPOP);
}

/* Macroscopic fields of n sites stored as f[n][37]. */
void or_moments(size_t n, const double* f, double* rho, double* ux, double* uy, double* T) {
    setup();
    for (size_t s = 0; s < n; ++s) moments_site(f + s * NPOP, rho + s, ux + s, uy + s, T + s);
}

/* Collide n sites stored as f[n][37], in place. */
void or_collide(size_t n, double* f, double tau, double gx, double gy, int nthreads) {
    setup();
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long long s = 0; s < (long long)n; ++s) collide_site(f + (size_t)s * NPOP, tau, gx, gy);
}

static long long wrap(long long v, long long L) {
    long long m = v % L;
    return m < 0 ? m + L : m;
}

/* Propagate, pull form (Fig. 3 listing: new[p][site] = old[p][site + OFF[p]]). A population
 * moving with velocity c_i arrives at site s from site s - c_i, so OFF_i = -c_i:
 *   dst_i(x, y) = src_i((x - c_ix) mod Lx, y - c_iy).
 * Rows y - c_iy outside [0, Ly) are read from the halo rows (walls) or wrap (y_periodic).
 * Both arrays carry halo rows; only the interior rows of dst are written. */
void or_propagate(int Lx, int Ly, int y_periodic, const double* src, double* dst, int nthreads) {
    setup();
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x)
            for (int i = 0; i < NPOP; ++i) {
                const long long xs = wrap((long long)x - CX[i], Lx);
                long long ys = (long long)y - CY[i];
                if (y_periodic) ys = wrap(ys, Ly);
                dst[((size_t)(y + HALO) * Lx + x) * NPOP + i] =
                    src[((size_t)(ys + HALO) * Lx + (size_t)xs) * NPOP + i];
            }
}

/* Wall step: the three halo rows below row 0 (y = -1 - k) hold the rest equilibrium at
 * T_bottom with the density of interior row k; the three above row Ly - 1 (y = Ly + k) hold the
 * rest equilibrium at T_top with the density of row Ly - 1 - k (k = 0, 1, 2). The density of a
 * row site is the sum of its current populations. */
void or_walls(int Lx, int Ly, double T_top, double T_bottom, double* f) {
    setup();
    for (int k = 0; k < HALO; ++k)
        for (int x = 0; x < Lx; ++x) {
            const double* fb = f + ((size_t)(k + HALO) * Lx + x) * NPOP;
            const double* ft = f + ((size_t)(Ly - 1 - k + HALO) * Lx + x) * NPOP;
            double rb = 0.0, rt = 0.0;
            for (int i = 0; i < NPOP; ++i) {
                rb += fb[i];
                rt += ft[i];
            }
            feq_site(rb, 0.0, 0.0, T_bottom, f + ((size_t)(HALO - 1 - k) * Lx + x) * NPOP);
            feq_site(rt, 0.0, 0.0, T_top, f + ((size_t)(Ly + HALO + k) * Lx + x) * NPOP);
        }
}

/* Mirror wall step (an alternative wall closure; the paper leaves walls to its references): the
 * halo row y = -1 - k holds the equilibrium at the density of its mirror row k, the opposite
 * velocity and the temperature 2 T_bottom - T(x, k); likewise above row Ly - 1 with T_top and
 * mirror row Ly - 1 - k. The fields of a mirror site are the moments of its current populations.
 * Linear interpolation between a row and its mirror halo row then gives zero velocity and the
 * wall temperature exactly on the plane half a site outside the last interior row (y = -1/2 and
 * y = Ly - 1/2): a no-slip wall at a fixed temperature. A mirror site hotter than twice the wall
 * temperature has no positive reflection; its halo site gets the rest closure instead. */
static void mirror_site(double rho, double ux, double uy, double T, double T_wall, double* out) {
    const double Th = 2.0 * T_wall - T;
    if (Th > 0.0)
        feq_site(rho, -ux, -uy, Th, out);
    else
        feq_site(rho, 0.0, 0.0, T_wall, out); /* not reflectable: the rest closure */
}

void or_walls_mirror(int Lx, int Ly, double T_top, double T_bottom, double* f) {
    setup();
    for (int k = 0; k < HALO; ++k)
        for (int x = 0; x < Lx; ++x) {
            double rho, ux, uy, T;
            moments_site(f + ((size_t)(k + HALO) * Lx + x) * NPOP, &rho, &ux, &uy, &T);
            mirror_site(rho, ux, uy, T, T_bottom, f + ((size_t)(HALO - 1 - k) * Lx + x) * NPOP);
            moments_site(f + ((size_t)(Ly - 1 - k + HALO) * Lx + x) * NPOP, &rho, &ux, &uy, &T);
            mirror_site(rho, ux, uy, T, T_top, f + ((size_t)(Ly + HALO + k) * Lx + x) * NPOP);
        }
}

/* Half-step ("physical") fields of n post-collision sites f[n][37] under gravity g: with the
 * shifted-equilibrium forcing a collision changes the momentum by rho g and the kinetic energy
 * sum f xi^2 / 2 by rho (u.g + |g|^2 / 2) while keeping rho and T, so the time averages of the
 * pre- and post-collision momentum and energy are those of the post-collision state minus half
 * of these changes: u_h = u_post - g / 2 and, from rho (|u_h|^2 + D T_h) = the averaged
 * energy, T_h = T_post + |g|^2 / (4 D). rho is unchanged. */
void or_moments_half_step(size_t n, const double* f, double gx, double gy, double* rho, double* ux,
                          double* uy, double* T) {
    setup();
    for (size_t s = 0; s < n; ++s) {
        moments_site(f + s * NPOP, rho + s, ux + s, uy + s, T + s);
        ux[s] -= 0.5 * gx;
        uy[s] -= 0.5 * gy;
        T[s] += (gx * gx + gy * gy) / (4.0 * DIM);
    }
}

/* Run nsteps time steps from interior populations f0[Ly*Lx][37] and store the interior result
 * in f_out (same layout). One step: wall halos (unless y_periodic; wall_mode 0 = rest
 * equilibrium at the wall temperature, 1 = mirror closure), pull propagate, collide. Returns 0,
 * or -1 when memory cannot be allocated. */
int or_run_walls(int Lx, int Ly, double tau, double gx, double gy, double T_top, double T_bottom,
                 int y_periodic, int wall_mode, int nsteps, int nthreads, const double* f0,
                 double* f_out) {
    setup();
    const size_t rows = (size_t)Ly + 2 * HALO;
    const size_t nfull = rows * (size_t)Lx * NPOP;
    const size_t nint = (size_t)Ly * (size_t)Lx * NPOP;
    double* a = (double*)calloc(nfull, sizeof(double));
    double* b = (double*)calloc(nfull, sizeof(double));
    if (!a || !b) {
        free(a);
        free(b);
        return -1;
    }
    memcpy(a + (size_t)HALO * Lx * NPOP, f0, nint * sizeof(double));
    for (int t = 0; t < nsteps; ++t) {
        if (!y_periodic) {
            if (wall_mode == 1)
                or_walls_mirror(Lx, Ly, T_top, T_bottom, a);
            else
                or_walls(Lx, Ly, T_top, T_bottom, a);
        }
        or_propagate(Lx, Ly, y_periodic, a, b, nthreads);
        or_collide((size_t)Ly * Lx, b + (size_t)HALO * Lx * NPOP, tau, gx, gy, nthreads);
        double* t2 = a;
        a = b;
        b = t2;
    }
    memcpy(f_out, a + (size_t)HALO * Lx * NPOP, nint * sizeof(double));
    free(a);
    free(b);
    return 0;
}

int or_run(int Lx, int Ly, double tau, double gx, double gy, double T_top, double T_bottom,
           int y_periodic, int nsteps, int nthreads, const double* f0, double* f_out) {
    return or_run_walls(Lx, Ly, tau, gx, gy, T_top, T_bottom, y_periodic, 0, nsteps, nthreads, f0,
                        f_out);
}
