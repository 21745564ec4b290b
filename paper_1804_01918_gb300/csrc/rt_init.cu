// rt_init.cu -- seeded Rayleigh-Taylor initial fields on the host, and the lattice and ensemble
// initialisations built on them (lb_rt_fields, lb_init_rt, lb_ensemble_init_rt).
//
// The paper runs the D2Q37 code on Rayleigh-Taylor problems (Sec. 3) but prints no initial
// condition; the recipe is a stated reading: walls top and bottom, periodic x; a cold heavy fluid
// above a hot light one, T_top = 2 / (1 + R), T_bottom = 2 R / (1 + R) (mean 1); the interface
// y_i(x) = Ly / 2 + Ly sum_{k=1..8} a_k cos(2 pi k x / Lx + phi_k) with a_k uniform draws scaled to
// sum 1e-3 and phi_k uniform in [0, 2 pi); T = 1 + (T_bottom - T_top) / 2 tanh((y_i - y) / 2);
// u = 0; rho = exp(-g (y - y_i) / T) / T (locally isothermal hydrostatic balance, p = 1 on the
// interface); g = 0.1 T_top / Ly downward. The draws come from SplitMix64 (Steele, Lea & Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014) seeded with `seed`: a_1..a_8,
// then phi_1..phi_8, each u = (next() >> 11) 2^-53. All arithmetic is plain IEEE double in the
// order written (no contraction), so another implementation of the same generator and recipe
// reproduces the fields up to the last-place rounding of cos, tanh and exp.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "../../include/lb_d2q37.h"
#include "../../include/lb_ensemble.h"

namespace {

constexpr int N_MODES = 8;
constexpr double AMPLITUDE = 1e-3;
constexpr double WIDTH = 2.0;
constexpr double G_FACTOR = 0.1;
constexpr double TWO_PI = 6.283185307179586476925286766559;

uint64_t splitmix64_next(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return (double)(splitmix64_next(s) >> 11) * 0x1p-53; }

}  // namespace

extern "C" lb_status lb_rt_fields(int Lx, int Ly, double R, uint64_t seed, double* rho, double* ux,
                                  double* uy, double* T, double* T_top, double* T_bottom, double* gy) {
    if (Lx < 1 || Ly < 1 || !(R > 0.0) || !std::isfinite(R) || !rho || !ux || !uy || !T) return LB_ERR_ARG;
    const double tt = 2.0 / (1.0 + R), tb = 2.0 * R / (1.0 + R);
    const double g = G_FACTOR * tt / Ly;
    uint64_t s = seed;
    double a[N_MODES], phi[N_MODES];
    double sum = 0.0;
    for (int k = 0; k < N_MODES; ++k) {
        a[k] = uniform01(s);
        sum = sum + a[k];
    }
    const double scale = AMPLITUDE / sum;
    for (int k = 0; k < N_MODES; ++k) a[k] = a[k] * scale;
    for (int k = 0; k < N_MODES; ++k) phi[k] = uniform01(s) * TWO_PI;
    std::vector<double> yi((size_t)Lx);
    for (int x = 0; x < Lx; ++x) {
        double acc = 0.0;
        for (int k = 0; k < N_MODES; ++k) {
            const double arg = ((TWO_PI * (double)(k + 1)) * (double)x) / (double)Lx + phi[k];
            const double term = a[k] * std::cos(arg);
            acc = acc + term;
        }
        const double spread = (double)Ly * acc;
        yi[(size_t)x] = (double)Ly / 2.0 + spread;
    }
    const double half_dT = 0.5 * (tb - tt);
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            const size_t i = (size_t)y * Lx + x;
            const double th = std::tanh((yi[(size_t)x] - (double)y) / WIDTH);
            const double dT = half_dT * th;
            const double t = 1.0 + dT;
            const double arg = (-g * ((double)y - yi[(size_t)x])) / t;
            T[i] = t;
            rho[i] = std::exp(arg) / t;
            ux[i] = 0.0;
            uy[i] = 0.0;
        }
    if (T_top) *T_top = tt;
    if (T_bottom) *T_bottom = tb;
    if (gy) *gy = -g;
    return LB_OK;
}

namespace {

struct Fields {
    std::vector<double> rho, ux, uy, T;
    double tt = 1.0, tb = 1.0, gy = 0.0;
    lb_status make(int Lx, int Ly, double R, uint64_t seed) {
        if (Lx < 1 || Ly < 1 || (long long)Lx * Ly > (1ll << 31)) return LB_ERR_ARG;
        const size_t n = (size_t)Lx * Ly;
        try {
            rho.resize(n);
            ux.resize(n);
            uy.resize(n);
            T.resize(n);
        } catch (...) {
            return LB_ERR_ALLOC;
        }
        return lb_rt_fields(Lx, Ly, R, seed, rho.data(), ux.data(), uy.data(), T.data(), &tt, &tb, &gy);
    }
};

}  // namespace

extern "C" lb_status lb_init_rt(const lb_params* p, double R, uint64_t seed, lb_ctx** out) {
    if (!p || !out) return LB_ERR_ARG;
    Fields f;
    lb_status st = f.make(p->Lx, p->Ly, R, seed);
    if (st != LB_OK) return st;
    lb_params q = *p;
    q.T_top = f.tt;
    q.T_bottom = f.tb;
    q.gy = f.gy;
    return lb_init(&q, f.rho.data(), f.ux.data(), f.uy.data(), f.T.data(), out);
}

extern "C" lb_status lb_ensemble_init_rt(int n, const lb_params* members, const double* R, const uint64_t* seeds,
                                         const lb_ensemble_opts* opts, lb_ensemble** out) {
    if (n < 1 || !members || !R || !seeds || !out) return LB_ERR_ARG;
    std::vector<Fields> f((size_t)n);
    std::vector<lb_params> q(members, members + n);
    std::vector<const double*> rho((size_t)n), ux((size_t)n), uy((size_t)n), T((size_t)n);
    for (int k = 0; k < n; ++k) {
        lb_status st = f[(size_t)k].make(members[k].Lx, members[k].Ly, R[k], seeds[k]);
        if (st != LB_OK) return st;
        q[(size_t)k].T_top = f[(size_t)k].tt;
        q[(size_t)k].T_bottom = f[(size_t)k].tb;
        q[(size_t)k].gy = f[(size_t)k].gy;
        rho[(size_t)k] = f[(size_t)k].rho.data();
        ux[(size_t)k] = f[(size_t)k].ux.data();
        uy[(size_t)k] = f[(size_t)k].uy.data();
        T[(size_t)k] = f[(size_t)k].T.data();
    }
    return lb_ensemble_init(n, q.data(), rho.data(), ux.data(), uy.data(), T.data(), opts, out);
}
