// step_fp32split_tma.cu -- the exact-split FP32 step with TMA-staged pulls (persistent kernel).
//
// The per-site arithmetic is that of step_fp32split_kernel (site_fp32dev.cuh); what changes is how
// the 37 shifted population rows reach the threads. A CTA of 128 threads owns tiles of 32 x 4
// sites. For each tile one thread issues, per population i, a TMA copy (cp.async.bulk.tensor) of
// the box of 40 columns x 4 rows that contains the tile shifted by -c_i: columns x0 - 4 .. x0 + 35
// (x0 a multiple of 32, so the box start is 16-byte aligned for every shift |c_x| <= 3) and rows
// y0 - c_iy .. y0 - c_iy + 3 of the halo-padded plane. Tiles are prefetched STAGES = 2 deep into
// a shared-memory ring (47 KB per CTA, so four CTAs -- 16 warps -- share an SM), so the next
// tile's loads are in flight while the current tile computes. Interior tiles read every
// population from the staged box at a compile-time offset; tiles whose sources wrap around x (the
// first and last tile columns; in the y-periodic test mode also the first and last tile rows)
// read the wrapping populations directly from global memory: the TMA box holds fill values there.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "d2q37_gpu.cuh"
#include "kernels.cuh"
#include "site_fp32dev.cuh"
#include "tc_helpers.cuh"

namespace lbg {
namespace tma32 {

constexpr int TX = 32, TY = 4;
constexpr int BOXW = TX + 8;                 // 40 columns, 160 bytes (a multiple of 16)
constexpr int BOX_FLOATS = BOXW * TY;        // 160 floats = 640 bytes per population
constexpr int STAGE_BYTES = NPOP * BOX_FLOATS * 4;
constexpr int STAGES = 2;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 64;
constexpr uint64_t WAIT_LIMIT = tc::WAIT_LIMIT_NS;
constexpr int ERR_TIMEOUT = 8;

__device__ __forceinline__ void arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(tc::smem_u32(mbar))
        : "memory");
}

template <int I>
struct IssueAll {
    __device__ __forceinline__ static void run(char* stage, const CUtensorMap* map, int x0, int y0,
                                               uint64_t* mbar) {
        IssueAll<I - 1>::run(stage, map, x0, y0, mbar);
        tma_load_3d(stage + I * BOX_FLOATS * 4, map, x0 - 4, y0 - cy_of(I) + HALO, I, mbar);
    }
};
template <>
struct IssueAll<-1> {
    __device__ __forceinline__ static void run(char*, const CUtensorMap*, int, int, uint64_t*) {}
};

// Population I of site (x, y): from the staged box, or from global memory where the source wraps.
template <int I>
struct GatherAll {
    __device__ __forceinline__ static void run(const float* stage, const float* __restrict__ src,
                                               float* d, int x, int y, int x0, int ty,
                                               const StepParams& P) {
        GatherAll<I - 1>::run(stage, src, d, x, y, x0, ty, P);
        constexpr int cx = cx_of(I), cy = cy_of(I);
        const int xu = x - cx, yu = y - cy;
        const bool wrap_x = (cx > 0 && xu < 0) || (cx < 0 && xu >= P.Lx);
        const bool wrap_y = P.y_periodic && ((cy > 0 && yu < 0) || (cy < 0 && yu >= P.Ly));
        if (!(wrap_x || wrap_y)) {
            d[I] = stage[I * BOX_FLOATS + ty * BOXW + (xu - x0 + 4)];
        } else {
            int xs = wrap_x ? (cx > 0 ? xu + P.Lx : xu - P.Lx) : xu;
            int ys = wrap_y ? (cy > 0 ? yu + P.Ly : yu - P.Ly) : yu;
            d[I] = __ldg(src + (long long)I * P.plane + (long long)(ys + HALO) * P.Lx + xs);
        }
    }
};
template <>
struct GatherAll<-1> {
    __device__ __forceinline__ static void run(const float*, const float*, float*, int, int, int, int,
                                               const StepParams&) {}
};

// Population I of thread (tx, ty) of an interior tile: always inside the staged box.
template <int I>
struct GatherFast {
    __device__ __forceinline__ static void run(const float* stage, float* d, int tx, int ty) {
        GatherFast<I - 1>::run(stage, d, tx, ty);
        d[I] = stage[I * BOX_FLOATS + ty * BOXW + tx + (4 - cx_of(I))];
    }
};
template <>
struct GatherFast<-1> {
    __device__ __forceinline__ static void run(const float*, float*, int, int) {}
};

__global__ void __launch_bounds__(128)
step_fp32split_tma_kernel(const __grid_constant__ CUtensorMap tsrc, const float* __restrict__ src,
                          float* __restrict__ dst, const StepParams P, int* __restrict__ flag) {
    extern __shared__ __align__(1024) char sm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + STAGES * STAGE_BYTES);
    const int tid = threadIdx.x;
    const int ntx = (P.Lx + TX - 1) / TX, nty = (P.Ly + TY - 1) / TY, ntiles = ntx * nty;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) tc::mbar_init(&full[s], 1);
    }
    __syncthreads();
    auto issue = [&](int t, int s) {
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        arrive_expect_tx(&full[s], STAGE_BYTES);
        IssueAll<NPOP - 1>::run(sm + s * STAGE_BYTES, &tsrc, x0, y0, &full[s]);
    };
    if (tid == 0)
        for (int s = 0; s < STAGES; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < ntiles) issue(t, s);
        }
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % STAGES;
        const uint32_t parity = (uint32_t)((k / STAGES) & 1);
        const bool got = tc::mbar_wait_bounded(&full[s], parity, WAIT_LIMIT);
        if (__syncthreads_or(!got)) {
            if (tid == 0) atomicOr(flag, ERR_TIMEOUT);
            break;
        }
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        const int ty = tid >> 5;
        const int x = x0 + (tid & 31), y = y0 + ty;
        const bool active = x < P.Lx && y < P.Ly;
        // tile-uniform: does any source of this tile wrap around x (or, y-periodic, around y)?
        const bool edge = x0 < HALO || x0 + TX + HALO > P.Lx ||
                          (P.y_periodic && (y0 < HALO || y0 + TY + HALO > P.Ly));
        float d[NPOP];
        const float* stage = reinterpret_cast<const float*>(sm + s * STAGE_BYTES);
        if (active) {
            if (edge)
                GatherAll<NPOP - 1>::run(stage, src, d, x, y, x0, ty, P);
            else
                GatherFast<NPOP - 1>::run(stage, d, tid & 31, ty);
        }
        __syncthreads();  // every thread has read stage s: refill it with a later tile
        if (tid == 0) {
            const int tn = t + STAGES * gridDim.x;
            if (tn < ntiles) {
                tc::fence_async_smem();
                issue(tn, s);
            }
        }
        if (active) {
            SplitPre sp;
            split_pre(d, P, sp, flag);
            split_collide(d, P, P, sp);
            split_project(d, P, P, sp);
            split_store(dst, P, x, y, d, sp, flag);
        }
    }
    // drain: wait (bounded) for copies still in flight before the block's shared memory goes away;
    // a stage whose copy did not arrive in time keeps its barrier valid (the copy may still land)
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            const int kk = k + s;  // the next use of each stage, if it was issued
            const int tt = blockIdx.x + kk * gridDim.x;
            const bool idle = tt >= ntiles ||
                              tc::mbar_wait_bounded(&full[kk % STAGES], (uint32_t)((kk / STAGES) & 1), WAIT_LIMIT);
            if (idle) tc::mbar_inval(&full[kk % STAGES]);
        }
    }
}

}  // namespace tma32

cudaError_t launch_step_fp32split_tma(const void* tmap, const float* src, float* dst, const StepParams& P,
                                      int* flag, int grid, cudaStream_t s) {
    tma32::step_fp32split_tma_kernel<<<grid, 128, tma32::SMEM_BYTES, s>>>(
        *reinterpret_cast<const CUtensorMap*>(tmap), src, dst, P, flag);
    return cudaGetLastError();
}

// Tensor map of one FP32 population copy: dims (x, row, population) = (Lx, Ly + 6, 37), box
// 40 x 4 x 1, zero fill outside. Needs Lx a multiple of 4 (16-byte row pitch).
cudaError_t make_fp32_tensor_map(void* tmap_out, const float* base, const StepParams& P) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    if (P.Lx % 4 != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)P.Lx, (cuuint64_t)P.Ly + 2 * HALO, (cuuint64_t)NPOP};
    const cuuint64_t strides[2] = {(cuuint64_t)P.Lx * 4, (cuuint64_t)P.plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)tma32::BOXW, (cuuint32_t)tma32::TY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(tmap_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int fp32split_tma_grid() {
    // co-resident CTAs of the current device (cached per device; the shared-memory attribute is
    // per device too)
    constexpr int MAXDEV = 64;
    static std::atomic<int> cached[MAXDEV];
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < MAXDEV && cached[dev].load() > 0) return cached[dev].load();
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(tma32::step_fp32split_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tma32::SMEM_BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tma32::step_fp32split_tma_kernel, 128, tma32::SMEM_BYTES);
    const int grid = (per > 0 ? per : 1) * sms;
    if (dev >= 0 && dev < MAXDEV) cached[dev].store(grid);
    return grid;
}

}  // namespace lbg
