// step_fp32dev.cu -- D2Q37 step with populations stored in FP32 as deviations from the weights.
//
// Storage: d_i = f_i - w_i in FP32, same structure-of-arrays layout as the FP64 path (half the
// bytes: 296 B per site and step instead of 592). Deviations are small, so FP32 keeps far more
// of each population's significant digits than FP32 absolute values would.
//
// One fused step per site:
//   1. pull the 37 deviations (Fig. 3 listing, pull at an offset);
//   2. FP64 moment accumulation: rho = 1 + sum d, rho u = r sum d c (sum w c = 0),
//      sum f |c|^2 = D / r^2 + sum d |c|^2 (sum w xi^2 = D), then u and T in FP64;
//   3. FP32 collide: the shifted Hermite equilibrium written as a deviation,
//      f_eq - w = w (drho (1 + p) + p) with p = P - 1 small, drho = rho - 1, and BGK;
//   4. FP64 conservation projection: the FP64 moments of the FP32 results are compared with the
//      exact post-collision targets (mass rho, momentum rho u + rho g, energy
//      rho (|u + g|^2 + D T)) and the residual is removed by the weighted least-norm correction
//      d_i += w_i (l0 + lx c_x + ly c_y + le |c|^2);
//   5. store FP32 deviations; wall rows write their halo rows.
#include <cuda_runtime.h>

#include <cstdint>

#include "d2q37_gpu.cuh"
#include "kernels.cuh"

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
        const double v = (double)d[i];
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

// FP32 collide of pair I: deviations of the post-collision populations I and I + NPAIR.
template <int I>
__device__ __forceinline__ void collide_pair32(float* d, float urx, float ury, const float* A0m1,
                                               const float* A2, const float* B1, const float* Wd,
                                               float drho, float omc) {
    constexpr int S = shellh(I);
    constexpr float cx = (float)cxh(I);
    constexpr float cy = (float)cyh(I);
    float a;
    if (cyh(I) == 0)
        a = cx * urx;
    else if (cxh(I) == 0)
        a = cy * ury;
    else
        a = fmaf(cx, urx, cy * ury);
    const float a2 = a * a;
    const float em1 = fmaf(a2, fmaf(a2, 1.0f / 24.0f, A2[S]), A0m1[S]);
    const float o = a * fmaf(a2, 1.0f / 6.0f, B1[S]);
    const float pp = em1 + o, pm = em1 - o;
    // w (rho P - 1) = w (drho (1 + p) + p)
    const float qp = fmaf(drho, pp, drho + pp);
    const float qm = fmaf(drho, pm, drho + pm);
    d[I] = fmaf(omc, d[I], Wd[S] * qp);
    d[I + NPAIR] = fmaf(omc, d[I + NPAIR], Wd[S] * qm);
}

template <int I>
struct Collide32 {
    __device__ __forceinline__ static void run(float* d, float urx, float ury, const float* A0m1,
                                               const float* A2, const float* B1, const float* Wd,
                                               float drho, float omc) {
        Collide32<I - 1>::run(d, urx, ury, A0m1, A2, B1, Wd, drho, omc);
        collide_pair32<I>(d, urx, ury, A0m1, A2, B1, Wd, drho, omc);
    }
};
template <>
struct Collide32<0> {
    __device__ __forceinline__ static void run(float*, float, float, const float*, const float*,
                                               const float*, const float*, float, float) {}
};

__global__ void __launch_bounds__(SITE_BLOCK)
step_fp32dev_kernel(const float* __restrict__ src, float* __restrict__ dst, const StepParams P,
                    int* __restrict__ flag) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long plane = P.plane;

    float d[NPOP];
    Pull32<NPOP - 1>::run(src, d, x, y, Lx, Ly, P.y_periodic, plane);

    const DevSums pre = dev_sums(d);
    const Macro m = macro_of(pre, P.r, P.r2);
    if (bad_positive64(m.rho) || bad_positive64(m.T)) atomicOr(flag, 1);

    // shifted equilibrium (forcing), coefficients in FP32 from FP64 moments
    const double uxs = m.ux + P.tgx;
    const double uys = m.uy + P.tgy;
    const double th = (m.T + P.dT_force) - 1.0;
    const double u2 = uxs * uxs + uys * uys;
    const float thf = (float)th, u2f = (float)u2;
    const float a00m1 = (float)(u2 * fma(u2, 0.125, -0.5));  // (1 - u2/2 + u2^2/8) - 1
    const float a20 = fmaf(u2f, -0.25f, 0.5f);
    const float b10 = fmaf(u2f, -0.5f, 1.0f);
    const float thu2 = thf * u2f, th2 = thf * thf;
    const float omega = (float)P.omega;
    float A0m1[NSHELL], A2[NSHELL], B1[NSHELL], Wd[NSHELL];
#pragma unroll
    for (int s = 0; s < NSHELL; ++s) {
        A0m1[s] = fmaf((float)P.sh[s].gamma, th2,
                       fmaf((float)P.sh[s].beta, thu2, fmaf((float)P.sh[s].alpha, thf, a00m1)));
        A2[s] = fmaf((float)P.sh[s].delta, thf, a20);
        B1[s] = fmaf((float)P.sh[s].eps, thf, b10);
        Wd[s] = omega * (float)P.sh[s].w;
    }
    const float drho = (float)pre.s0;
    const float omc = (float)P.omc;
    d[0] = fmaf(omc, d[0], Wd[0] * fmaf(drho, A0m1[0], drho + A0m1[0]));
    Collide32<NPAIR>::run(d, (float)(P.r * uxs), (float)(P.r * uys), A0m1, A2, B1, Wd, drho, omc);

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

    if (!P.y_periodic) {
        if (y < HALO) {
            const long long o = (long long)(HALO - 1 - y) * Lx + x;
#pragma unroll
            for (int i = 0; i < NPOP; ++i)
                __stcs(dst + poff(i, plane) + o, (float)fma(m.rho, P.wall_bot[i], -shell_w(shell_of(i))));
        }
        if (y >= Ly - HALO) {
            const long long o = (long long)(Ly + HALO + (Ly - 1 - y)) * Lx + x;
#pragma unroll
            for (int i = 0; i < NPOP; ++i)
                __stcs(dst + poff(i, plane) + o, (float)fma(m.rho, P.wall_top[i], -shell_w(shell_of(i))));
        }
    }
}

__global__ void __launch_bounds__(SITE_BLOCK)
propagate_fp32dev_kernel(const float* __restrict__ src, float* __restrict__ dst, const StepParams P) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long plane = P.plane;
    float d[NPOP];
    Pull32<NPOP - 1>::run(src, d, x, y, Lx, Ly, P.y_periodic, plane);
    const long long dsto = (long long)(y + HALO) * Lx + x;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) dst[poff(i, plane) + dsto] = d[i];
    if (y < HALO) {
        const long long ob = (long long)y * Lx + x;
        const long long ot = (long long)(Ly + HALO + y) * Lx + x;
#pragma unroll
        for (int i = 0; i < NPOP; ++i) {
            dst[poff(i, plane) + ob] = src[poff(i, plane) + ob];
            dst[poff(i, plane) + ot] = src[poff(i, plane) + ot];
        }
    }
}

// Equilibrium deviation f_eq - w of one site, evaluated in FP64 (initialisation only).
__global__ void __launch_bounds__(SITE_BLOCK)
init_fp32dev_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                    const double* __restrict__ uy, const double* __restrict__ T,
                    float* __restrict__ f, const StepParams P) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const double r0 = rho[site], vx = ux[site], vy = uy[site];
    const double th = T[site] - 1.0;
    const double u2 = vx * vx + vy * vy;
    const double a00m1 = u2 * fma(u2, 0.125, -0.5);
    const double a20 = fma(u2, -0.25, 0.5), b10 = fma(u2, -0.5, 1.0);
    const double drho = r0 - 1.0;
    const long long o = (long long)(y + HALO) * Lx + x;
    const double urx = P.r * vx, ury = P.r * vy;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const int s = shell_of(i);
        const double A0m1 = P.sh[s].gamma * th * th + P.sh[s].beta * th * u2 + P.sh[s].alpha * th + a00m1;
        const double A2 = fma(P.sh[s].delta, th, a20), B1 = fma(P.sh[s].eps, th, b10);
        const double a = cx_of(i) * urx + cy_of(i) * ury;
        const double a2 = a * a;
        const double p = fma(a2, fma(a2, 1.0 / 24.0, A2), A0m1) + a * fma(a2, 1.0 / 6.0, B1);
        f[poff(i, P.plane) + o] = (float)(P.sh[s].w * fma(drho, p, drho + p));
    }
}

__global__ void halo_fp32dev_kernel(float* __restrict__ f, const StepParams P) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= HALO * Lx) return;
    const int k = t / Lx;
    const int x = t - k * Lx;
    const long long ib = (long long)(HALO + k) * Lx + x;
    const long long it = (long long)(HALO + Ly - 1 - k) * Lx + x;
    double rb = 1.0, rt = 1.0;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        rb += (double)f[poff(i, P.plane) + ib];
        rt += (double)f[poff(i, P.plane) + it];
    }
    const long long ob = (long long)(HALO - 1 - k) * Lx + x;
    const long long ot = (long long)(Ly + HALO + k) * Lx + x;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const double w = shell_w(shell_of(i));
        f[poff(i, P.plane) + ob] = (float)fma(rb, P.wall_bot[i], -w);
        f[poff(i, P.plane) + ot] = (float)fma(rt, P.wall_top[i], -w);
    }
}

__global__ void __launch_bounds__(SITE_BLOCK)
moments_fp32dev_kernel(const float* __restrict__ f, const StepParams P, double* __restrict__ rho,
                       double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long o = (long long)(y + HALO) * Lx + x;
    float d[NPOP];
#pragma unroll
    for (int i = 0; i < NPOP; ++i) d[i] = f[poff(i, P.plane) + o];
    const Macro m = macro_of(dev_sums(d), P.r, P.r2);
    rho[site] = m.rho;
    ux[site] = m.ux;
    uy[site] = m.uy;
    T[site] = m.T;
}

__global__ void plane_to_dev32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                                      double w, long long n) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = (float)(src[j] - w);
}

__global__ void plane_from_dev32_kernel(const float* __restrict__ src, double* __restrict__ dst,
                                        double w, long long n) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = w + (double)src[j];
}

inline int site_blocks32(const StepParams& P) {
    const long long n = (long long)P.Lx * P.Ly;
    return (int)((n + SITE_BLOCK - 1) / SITE_BLOCK);
}

}  // namespace

cudaError_t launch_step_fp32dev(const float* src, float* dst, const StepParams& P, int* flag,
                                cudaStream_t s) {
    step_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(src, dst, P, flag);
    return cudaGetLastError();
}

cudaError_t launch_propagate_fp32dev(const float* src, float* dst, const StepParams& P,
                                     cudaStream_t s) {
    propagate_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(src, dst, P);
    return cudaGetLastError();
}

cudaError_t launch_init_fp32dev(const double* rho, const double* ux, const double* uy,
                                const double* T, float* f, const StepParams& P, cudaStream_t s) {
    init_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(rho, ux, uy, T, f, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || P.y_periodic) return e;
    return launch_halo_fp32dev(f, P, s);
}

cudaError_t launch_moments_fp32dev(const float* f, const StepParams& P, double* rho, double* ux,
                                   double* uy, double* T, cudaStream_t s) {
    moments_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(f, P, rho, ux, uy, T);
    return cudaGetLastError();
}

cudaError_t launch_halo_fp32dev(float* f, const StepParams& P, cudaStream_t s) {
    const int n = HALO * P.Lx;
    halo_fp32dev_kernel<<<(n + 127) / 128, 128, 0, s>>>(f, P);
    return cudaGetLastError();
}

cudaError_t launch_plane_to_dev32(const double* src, float* dst, double w, long long n,
                                  cudaStream_t s) {
    plane_to_dev32_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, w, n);
    return cudaGetLastError();
}

cudaError_t launch_plane_from_dev32(const float* src, double* dst, double w, long long n,
                                    cudaStream_t s) {
    plane_from_dev32_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, w, n);
    return cudaGetLastError();
}

}  // namespace lbg
