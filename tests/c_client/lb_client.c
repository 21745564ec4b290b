/* A plain C client of the C ABI (include/lb_d2q37.h): no Python, no torch. It builds a small
 * lattice with deterministic fields, advances it, and prints the sums of the macroscopic fields
 * and of the populations with 17 significant digits, so that a test can compare them with the same
 * run through the Python binding. Exit status 0 on success, 1 on any library error. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lb_d2q37.h"

#define CHECK(call)                                                                    \
    do {                                                                               \
        lb_status s_ = (call);                                                         \
        if (s_ != LB_OK) {                                                             \
            fprintf(stderr, "%s: %s (%s)\n", #call, lb_status_str(s_), lb_last_error()); \
            return 1;                                                                  \
        }                                                                              \
    } while (0)

int main(int argc, char** argv) {
    const int Lx = 48, Ly = 40, steps = argc > 1 ? atoi(argv[1]) : 25;
    const int wall_mode = argc > 2 ? atoi(argv[2]) : LB_WALL_REST;
    const size_t n = (size_t)Lx * Ly;
    double* rho = malloc(n * sizeof(double));
    double* ux = malloc(n * sizeof(double));
    double* uy = malloc(n * sizeof(double));
    double* T = malloc(n * sizeof(double));
    double* f = malloc(LB_NPOP * n * sizeof(double));
    if (!rho || !ux || !uy || !T || !f) return 1;
    const double pi = 3.14159265358979323846;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            const size_t s = (size_t)y * Lx + x;
            rho[s] = 1.0 + 0.05 * sin(2.0 * pi * x / Lx) * cos(pi * y / Ly);
            ux[s] = 0.01 * cos(2.0 * pi * y / Ly);
            uy[s] = 0.005 * sin(2.0 * pi * x / Lx);
            T[s] = 1.0 + 0.1 * (0.5 - (double)y / (Ly - 1));
        }
    lb_params p = {0};
    p.Lx = Lx;
    p.Ly = Ly;
    p.tau = 0.8;
    p.gx = 0.0;
    p.gy = -1e-4;
    p.T_top = 0.95;
    p.T_bottom = 1.05;
    p.y_periodic = 0;
    p.precision = LB_FP64;
    p.wall_mode = wall_mode;
    p.stream = NULL;     /* the library creates its own stream */
    p.workspace = NULL;  /* and owns its device memory */
    lb_ctx* c = NULL;
    CHECK(lb_init(&p, rho, ux, uy, T, &c));
    CHECK(lb_step(c, steps));
    CHECK(lb_sync(c));
    long long done = 0;
    CHECK(lb_steps_done(c, &done));
    CHECK(lb_moments(c, rho, ux, uy, T));
    CHECK(lb_get_populations(c, f));
    lb_free(c);
    double m[4] = {0, 0, 0, 0}, fs = 0.0;
    for (size_t s = 0; s < n; ++s) {
        m[0] += rho[s];
        m[1] += rho[s] * ux[s];
        m[2] += rho[s] * uy[s];
        m[3] += T[s];
    }
    for (size_t k = 0; k < LB_NPOP * n; ++k) fs += f[k];
    printf("steps %lld\n", done);
    printf("sum_rho %.17g\nsum_jx %.17g\nsum_jy %.17g\nsum_T %.17g\nsum_f %.17g\n", m[0], m[1], m[2], m[3],
           fs);
    free(rho);
    free(ux);
    free(uy);
    free(T);
    free(f);
    return 0;
}
