// noalloc.cu -- macroscopic fields of caller-owned populations without any device allocation.
//
// lb_moments stages its four output fields in the context's device workspace before copying them
// to the host. Callers that cannot allocate device memory (their memory belongs to a host
// framework's own allocator, or they run where cudaMalloc is not allowed) use
// lb_moments_noalloc instead: the staging area is a fixed static device array that exists in
// every process that loads the library, and the kernel is the same moments kernel.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/lb_d2q37.h"
#include "d2q37_gpu.cuh"
#include "kernels.cuh"

using namespace lbg;

namespace lbg {
void set_last_error(const char* msg);  // lb_capi.cu: the message lb_last_error() returns
}

namespace {

// Four fields (rho, ux, uy, T) of at most LB_NOALLOC_MAX_SITES sites: 2 MiB per GPU, held by
// every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[4 * LB_NOALLOC_MAX_SITES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {nullptr};


// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lb_status lb_moments_noalloc(const lb_params* p, const void* f, double* rho, double* ux,
                                        double* uy, double* T) {
    if (!p || !f) return LB_ERR_ARG;
    if (p->Lx < 4 || p->Ly < 4) return LB_ERR_ARG;
    if (p->precision != LB_FP64 && p->precision != LB_FP32DEV && p->precision != LB_FP32SPLIT)
        return LB_ERR_ARG;
    const long long n = (long long)p->Lx * p->Ly;
    if (n > LB_NOALLOC_MAX_SITES) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "lb_moments_noalloc: %d x %d = %lld sites exceeds the static scratch of %d sites",
                      p->Lx, p->Ly, n, LB_NOALLOC_MAX_SITES);
        set_last_error(msg);
        return LB_ERR_ARG;
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "lb_moments_noalloc: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
        set_last_error(msg);
        return LB_ERR_CUDA;
    }
    // the kernel parameters of the context path (lattice constants, row reciprocal for the site's
    // row); the fields this call ignores get neutral values so that nothing the caller left in
    // them reaches the kernel
    lb_params q;
    std::memset(&q, 0, sizeof q);
    q.Lx = p->Lx;
    q.Ly = p->Ly;
    q.tau = 1.0;
    q.T_top = q.T_bottom = 1.0;
    q.precision = p->precision;
    q.wall_mode = LB_WALL_REST;
    StepParams sp;
    fill_step_params(q, sp);
    cudaStream_t s = (cudaStream_t)p->stream;
    if (p->precision == LB_FP64)
        e = launch_moments_fp64((const double*)f, sp, scratch, scratch + n, scratch + 2 * n,
                                scratch + 3 * n, 0, s);
    else
        e = launch_moments_fp32dev((const float*)f, sp, scratch, scratch + n, scratch + 2 * n,
                                   scratch + 3 * n, 0, s);
    double* dst[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (dst[k])
            e = cudaMemcpyAsync(dst[k], scratch + k * n, (size_t)n * sizeof(double),
                                cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "lb_moments_noalloc: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return LB_ERR_CUDA;
    }
    return LB_OK;
}
