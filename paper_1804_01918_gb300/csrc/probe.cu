// probe.cu -- FMA-throughput probe (roofline denominator of the ALU-bound kernels).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/lb_probe.h"
#include "tc_helpers.cuh"

namespace {

template <typename T>
__global__ void fma_chains_kernel(T* __restrict__ out, int iters, T m, T a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T x0 = (T)(t & 7), x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int k = 0; k < iters; ++k) {
        x0 = x0 * m + a; x1 = x1 * m + a; x2 = x2 * m + a; x3 = x3 * m + a;
        x4 = x4 * m + a; x5 = x5 * m + a; x6 = x6 * m + a; x7 = x7 * m + a;
    }
    out[t] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// The same chains with operands that keep changing: each chain alternates its addend between two
// values, so no chain settles on a fixed point (the FP64 pipe of GB300 runs measurably faster on
// operands that stop changing, so this is the rate a real kernel's varying data sees).
template <typename T>
__global__ void fma_chains_varying_kernel(T* __restrict__ out, int iters, T m, T a, T b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T x0 = (T)(t & 7), x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int k = 0; k < iters; ++k) {
        const T c = (k & 1) ? a : b;
        x0 = x0 * m + c; x1 = x1 * m + c; x2 = x2 * m + c; x3 = x3 * m + c;
        x4 = x4 * m + c; x5 = x5 * m + c; x6 = x6 * m + c; x7 = x7 * m + c;
    }
    out[t] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// The bounded-wait path of the library's tensor-core and TMA kernels, checked on its own: one
// thread initialises an mbarrier expecting one arrival and waits on it with the library's bounded
// wait. With arrive = 0 nothing ever arrives (no asynchronous operation targets the barrier, so
// nothing is in flight when the wait gives up); with arrive = 1 the thread arrives first and the
// wait succeeds at once. out[0] = 1 if the wait gave up, out[1] = nanoseconds it took.
__global__ void wait_probe_kernel(unsigned long long limit_ns, int arrive, unsigned long long* out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    lbg::tc::mbar_init(&bar, 1);
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(lbg::tc::smem_u32(&bar)) : "memory");
    const uint64_t t0 = lbg::tc::globaltimer_ns();
    const bool got = lbg::tc::mbar_wait_bounded(&bar, 0u, limit_ns);
    const uint64_t t1 = lbg::tc::globaltimer_ns();
    if (got) lbg::tc::mbar_inval(&bar);
    out[0] = got ? 0ull : 1ull;
    out[1] = t1 - t0;
}

}  // namespace

extern "C" lb_status lb_probe_wait(unsigned long long limit_ns, int arrive, void* stream,
                                   unsigned long long* out) {
    if (!out || limit_ns == 0 || limit_ns > 10000000000ull || (arrive != 0 && arrive != 1)) return LB_ERR_ARG;
    wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(limit_ns, arrive, out);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

extern "C" lb_status lb_probe_fma(int kind, void* stream, int blocks, int threads, int iters,
                                  void* out) {
    if (blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0 || !out) return LB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0)
        fma_chains_kernel<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.9999999, 1e-7);
    else if (kind == 1)
        fma_chains_kernel<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.9999f, 1e-4f);
    else if (kind == 2)
        fma_chains_varying_kernel<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.9999999, 1e-7, 3e-7);
    else
        return LB_ERR_ARG;
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
