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
#include "site_fp32dev.cuh"

namespace lbg {

namespace {

// Both step kernels cover sites site0 .. site1 - 1 (the whole lattice, or a band of rows of a slab).
__global__ void __launch_bounds__(SITE_BLOCK)
step_fp32dev_kernel(const float* __restrict__ src, float* __restrict__ dst, const StepParams P,
                    int* __restrict__ flag, int site0, int site1) {
    const int site = site0 + blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= site1) return;
    const int y = row_of(site, P);
    fp32dev_site(src, dst, P, site - y * P.Lx, y, flag);
}

__global__ void __launch_bounds__(SITE_BLOCK)
step_fp32split_kernel(const float* __restrict__ src, float* __restrict__ dst, const StepParams P,
                      int* __restrict__ flag, int site0, int site1) {
    const int site = site0 + blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= site1) return;
    const int y = row_of(site, P);
    fp32split_site(src, dst, P, P, site - y * P.Lx, y, flag);
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

// Wall halos of f from the current interior rows 0..2 and Ly-3..Ly-1 (their FP64 moments), as
// the step writes them: thread t handles interior row k = t / Lx of each wall.
__global__ void halo_fp32dev_kernel(float* __restrict__ f, const StepParams P, int* __restrict__ flag) {
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
        float d[NPOP];
#pragma unroll
        for (int i = 0; i < NPOP; ++i) d[i] = f[poff(i, P.plane) + o];
        const Macro m = macro_of(dev_sums(d), P.r, P.r2);
        write_wall_rows(P, x, y, m.rho, m.ux, m.uy, m.T, flag, [&](int i, long long oh, double v) {
            f[poff(i, P.plane) + oh] = (float)(v - shell_w(shell_of(i)));
        });
    }
}

__global__ void __launch_bounds__(SITE_BLOCK)
moments_fp32dev_kernel(const float* __restrict__ f, const StepParams P, double* __restrict__ rho,
                       double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T,
                       int half_step) {
    const int Lx = P.Lx, Ly = P.Ly;
    const int site = blockIdx.x * SITE_BLOCK + threadIdx.x;
    if (site >= Lx * Ly) return;
    const int y = site / Lx;
    const int x = site - y * Lx;
    const long long o = (long long)(y + HALO) * Lx + x;
    float d[NPOP];
#pragma unroll
    for (int i = 0; i < NPOP; ++i) d[i] = f[poff(i, P.plane) + o];
    Macro m = macro_of(dev_sums(d), P.r, P.r2);
    if (half_step) half_step_shift(P, m.ux, m.uy, m.T);
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
    step_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(src, dst, P, flag, 0, P.Lx * P.Ly);
    return cudaGetLastError();
}

cudaError_t launch_step_fp32split(const float* src, float* dst, const StepParams& P, int* flag,
                                  cudaStream_t s) {
    step_fp32split_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(src, dst, P, flag, 0, P.Lx * P.Ly);
    return cudaGetLastError();
}

cudaError_t launch_step_fp32_rows(bool split, const float* src, float* dst, const StepParams& P, int* flag,
                                  int row0, int row1, cudaStream_t s) {
    if (row1 <= row0) return cudaSuccess;
    const int n = (row1 - row0) * P.Lx, blocks = (n + SITE_BLOCK - 1) / SITE_BLOCK;
    if (split)
        step_fp32split_kernel<<<blocks, SITE_BLOCK, 0, s>>>(src, dst, P, flag, row0 * P.Lx, row1 * P.Lx);
    else
        step_fp32dev_kernel<<<blocks, SITE_BLOCK, 0, s>>>(src, dst, P, flag, row0 * P.Lx, row1 * P.Lx);
    return cudaGetLastError();
}

cudaError_t launch_propagate_fp32dev(const float* src, float* dst, const StepParams& P,
                                     cudaStream_t s) {
    propagate_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(src, dst, P);
    return cudaGetLastError();
}

cudaError_t launch_init_fp32dev(const double* rho, const double* ux, const double* uy,
                                const double* T, float* f, const StepParams& P, int* flag, cudaStream_t s) {
    init_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(rho, ux, uy, T, f, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || P.y_periodic) return e;
    return launch_halo_fp32dev(f, P, flag, s);
}

cudaError_t launch_moments_fp32dev(const float* f, const StepParams& P, double* rho, double* ux,
                                   double* uy, double* T, int half_step, cudaStream_t s) {
    moments_fp32dev_kernel<<<site_blocks32(P), SITE_BLOCK, 0, s>>>(f, P, rho, ux, uy, T, half_step);
    return cudaGetLastError();
}

cudaError_t launch_halo_fp32dev(float* f, const StepParams& P, int* flag, cudaStream_t s) {
    const int n = HALO * P.Lx;
    halo_fp32dev_kernel<<<(n + 127) / 128, 128, 0, s>>>(f, P, flag);
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
