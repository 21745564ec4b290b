// kernels.cuh -- launchers of the D2Q37 kernels, called by the C ABI layer (lb_capi.cu).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "d2q37_gpu.cuh"

#include "lb_d2q37.h"

namespace lbg {

// ---- host helpers (lb_capi.cu) ----
double thermal_scale();                                   // r = 1 / sqrt(sum w c_x^2)
void fill_step_params(const lb_params& p, StepParams& sp);  // per-lattice kernel parameters
void set_last_error(const char* msg);                     // message returned by lb_last_error()

// A named NVTX range for the lifetime of a scope: the C ABI marks each entry point, so profilers
// (ncu --nvtx, nsys) can attribute the kernels they capture to the call that queued them. Costs
// nothing measurable when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Threads per block of the site-parallel kernels.
constexpr int SITE_BLOCK = 128;

// ---- FP64 populations (step_fp64.cu) ----
cudaError_t launch_step_fp64(const double* src, double* dst, const StepParams& P, int* flag,
                             cudaStream_t s);
cudaError_t launch_propagate_fp64(const double* src, double* dst, const StepParams& P,
                                  cudaStream_t s);
cudaError_t launch_collide_fp64(double* f, const StepParams& P, int* flag, cudaStream_t s);
// the fused step on rows row0 .. row1 - 1 only (a slab's boundary bands or its interior)
cudaError_t launch_step_fp64_rows(const double* src, double* dst, const StepParams& P, int* flag,
                                  int row0, int row1, cudaStream_t s);
cudaError_t launch_init_fp64(const double* rho, const double* ux, const double* uy,
                             const double* T, double* f, const StepParams& P, int* flag, cudaStream_t s);
// half_step != 0: the half-step fields (u - g/2, T + |g|^2 / (4 D)) instead of the plain moments
cudaError_t launch_moments_fp64(const double* f, const StepParams& P, double* rho, double* ux,
                                double* uy, double* T, int half_step, cudaStream_t s);
cudaError_t launch_halo_fp64(double* f, const StepParams& P, int* flag, cudaStream_t s);

// ---- FP32 deviation populations (step_fp32dev.cu) ----
cudaError_t launch_step_fp32dev(const float* src, float* dst, const StepParams& P, int* flag,
                                cudaStream_t s);
// same storage, exact-split FP32 accumulation instead of FP64 (site_fp32dev.cuh)
cudaError_t launch_step_fp32split(const float* src, float* dst, const StepParams& P, int* flag,
                                  cudaStream_t s);
// either FP32 step (split = exact-split or FP64-sum form) on rows row0 .. row1 - 1 only
cudaError_t launch_step_fp32_rows(bool split, const float* src, float* dst, const StepParams& P, int* flag,
                                  int row0, int row1, cudaStream_t s);
// the same step with TMA-staged pulls (step_fp32split_tma.cu); tmap is a CUtensorMap of src
cudaError_t launch_step_fp32split_tma(const void* tmap, const float* src, float* dst,
                                      const StepParams& P, int* flag, int grid, cudaStream_t s);
cudaError_t make_fp32_tensor_map(void* tmap_out, const float* base, const StepParams& P);
int fp32split_tma_grid();
cudaError_t launch_propagate_fp32dev(const float* src, float* dst, const StepParams& P,
                                     cudaStream_t s);
cudaError_t launch_init_fp32dev(const double* rho, const double* ux, const double* uy,
                                const double* T, float* f, const StepParams& P, int* flag, cudaStream_t s);
cudaError_t launch_moments_fp32dev(const float* f, const StepParams& P, double* rho, double* ux,
                                   double* uy, double* T, int half_step, cudaStream_t s);
cudaError_t launch_halo_fp32dev(float* f, const StepParams& P, int* flag, cudaStream_t s);
// plane i interior: FP64 absolute populations <-> FP32 deviations
cudaError_t launch_plane_to_dev32(const double* src, float* dst_plane_interior, double w,
                                  long long n, cudaStream_t s);
cudaError_t launch_plane_from_dev32(const float* src_plane_interior, double* dst, double w,
                                    long long n, cudaStream_t s);

// ---- learned collide (learned.cu) ----
struct LearnedState;
lb_status learned_create(const struct lb_mlp* net, int Lx, int Ly, double bound, int check_every,
                         LearnedState** out);
void learned_destroy(LearnedState* ls);
// the network, bound and check interval a learned state was created with
lb_status learned_info(const LearnedState* ls, const struct lb_mlp** net, double* bound, int* check_every);
cudaError_t launch_step_learned(const float* src, float* dst, const StepParams& P, LearnedState* ls,
                                int* flag, cudaStream_t s);
cudaError_t launch_pairs(const float* src, const StepParams& P, const int* sites, int n, float* pre,
                         float* post, int* flag, cudaStream_t s);
// host copy of the per-tile decisions (1 = plain collide) of a learned state with ntiles tiles
lb_status learned_tiles(LearnedState* ls, int ntiles, unsigned char* modes, cudaStream_t s);
lb_status learned_stats(LearnedState* ls, long long* checked, long long* fallback, double* max_res,
                        cudaStream_t s);

// ---- slabs of a lattice cut along y (slab.cu): 26 ghost population-rows per cut and direction ----
int ghost_row_count();
cudaError_t launch_slab_pack(size_t elem, const void* f, void* buf, const StepParams& P, int side, cudaStream_t s);
cudaError_t launch_slab_unpack(size_t elem, const void* buf, void* f, const StepParams& P, int side,
                               cudaStream_t s);
cudaError_t launch_slab_exchange(size_t elem, void* f_lo, const StepParams& Plo, void* f_hi,
                                 const StepParams& Phi, cudaStream_t s);

}  // namespace lbg
