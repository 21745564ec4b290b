/*
 * lb_probe.h -- device-throughput probe of the D2Q37 library.
 *
 * The paper rates collide against the processor's peak floating-point throughput (Sec. 5:
 * ~1 TFlops sustained, ~30% of the KNL's raw peak). On GB300 the FP64 and FP32 CUDA-core peaks
 * are not published per part, so the library carries its own probe: a kernel of independent
 * fused multiply-add chains whose time, measured by the caller with CUDA events, gives the
 * achievable FMA rate used as the roofline denominator of the ALU-bound step kernels.
 */
#ifndef LB_PROBE_H
#define LB_PROBE_H

#include "lb_d2q37.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Launch blocks x threads threads; each runs 8 independent FMA chains of `iters` steps in FP64
 * (kind 0) or FP32 (kind 1), i.e. 16 * iters flops per thread, and writes one value per thread
 * to out (device memory of blocks*threads elements of that type, caller-owned). The chains of
 * kinds 0 and 1 converge to a fixed point, after which their operands stop changing; kind 2 is
 * FP64 with an addend that alternates every step, so the operands keep changing as in a real
 * kernel (GB300's FP64 pipe sustains a lower rate on such data). Asynchronous on
 * `stream` (cudaStream_t, NULL = legacy default stream). LB_ERR_ARG for non-positive sizes,
 * threads > 1024 or an unknown kind. */
lb_status lb_probe_fma(int kind, void* stream, int blocks, int threads, int iters, void* out);

/* Self-check of the failure path of the library's asynchronous waits (the paper has no
 * counterpart). Every wait of the tensor-core and TMA kernels on a shared-memory barrier gives up
 * after a time limit (2 s of the GPU's global timer), sets a status bit that the host reads and
 * lets the kernel return, so a stuck operation never hangs the GPU. This call runs that wait
 * alone in a one-thread kernel: with arrive = 0 on a barrier that nothing ever completes (no
 * asynchronous operation targets it, so nothing is left in flight), with arrive = 1 on one the
 * thread completes first. limit_ns: 1 .. 1e10. out: device memory of two unsigned 64-bit values,
 * caller-owned: out[0] = 1 if the wait gave up (0 if it succeeded), out[1] = the nanoseconds it
 * waited. Asynchronous on `stream`; LB_ERR_ARG for a NULL out or a limit out of range. */
lb_status lb_probe_wait(unsigned long long limit_ns, int arrive, void* stream, unsigned long long* out);

#ifdef __cplusplus
}
#endif

#endif /* LB_PROBE_H */
