// ensemble.cu -- batched ensemble of independent D2Q37 lattices in one launch per step.
//
// Device data: every member's two FP32-deviation population copies (same layout as a single
// lattice), a member table (kernel parameters + buffer pointers), a global list of work items
// (member, x0, y0, log2 of the tile width) covering all members with tiles of tile_x x tile_y
// sites -- narrowed to the widest power of two >= 32 that divides a member's Lx, and heightened to
// keep the tile's site count, so that no tile overhangs a member's right edge -- a host-exchange
// staging area sized for the largest member, and a status word.
//
// One launch of the step kernel covers every member: by default a persistent grid of the
// co-resident blocks, each taking the next unclaimed work item from a counter, so that the items in
// flight stay a contiguous window of the list (on request one block per item, within 1 % of it;
// a persistent grid whose block b took items b, b + grid, ... drifted apart and measured 21 %
// slower, its pulls' neighbouring rows no longer in L2). For each item the
// block copies the member's parameters to shared memory (unless it already holds them) and its
// threads run the same per-site update as the single-lattice FP32 kernels. Items are ordered member
// by member, row band by row band, so the blocks in flight work on neighbouring tiles and the
// pull's row offsets (up to 3 rows) hit in L2.
#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lb_ensemble.h"
#include "d2q37_gpu.cuh"
#include "kernels.cuh"
#include "site_fp32dev.cuh"

using namespace lbg;

// Named namespace: nvcc's host stubs for templated kernels cannot name types declared in a second
// anonymous namespace of the same translation unit.
namespace lbg {
namespace ens {

constexpr int ENS_BLOCK = 128;
constexpr size_t ALIGN = 256;
constexpr int CLAIM_WORD = 32;  // int offset of the persistent grid's item counter in the status area

struct MemberDesc {
    StepParams P;
    float* buf[2];
};

inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

template <bool kSplit>
__global__ void __launch_bounds__(ENS_BLOCK, kSplit ? 5 : 1)  // split: 20 warps per SM, <= 102 registers
ensemble_step_kernel(const StepParams Pc, const MemberDesc* __restrict__ members,
                     const int4* __restrict__ items, int nitems, int tile_sites, int parity,
                     int* __restrict__ claim, int* __restrict__ flag) {
    __shared__ __align__(16) StepParams sP;
    __shared__ const float* s_src;
    __shared__ float* s_dst;
    __shared__ int s_item[2];
    constexpr int NWORDS = (int)(sizeof(StepParams) / sizeof(unsigned long long));
    int staged = -1;  // member whose parameters sit in sP (block-uniform)
    // claim != nullptr: a persistent grid whose blocks take the next unclaimed item from a counter
    // (so the items in flight stay a contiguous window of the list, as with one block per item);
    // else block b takes items b, b + grid, ...
    int t = blockIdx.x;
    if (claim) {
        if (threadIdx.x == 0) s_item[0] = atomicAdd(claim, 1);
        __syncthreads();
        t = s_item[0];
    }
    for (int j = 1; t < nitems; ++j) {
        const int4 it = items[t];
        if (it.x != staged) {  // items run member by member: most items reuse the staged member
            __syncthreads();   // the previous item is finished with sP
            const unsigned long long* g = reinterpret_cast<const unsigned long long*>(&members[it.x].P);
            unsigned long long* s = reinterpret_cast<unsigned long long*>(&sP);
            for (int k = threadIdx.x; k < NWORDS; k += ENS_BLOCK) s[k] = g[k];
            if (threadIdx.x == 0) {
                s_src = members[it.x].buf[parity];
                s_dst = members[it.x].buf[parity ^ 1];
            }
            __syncthreads();
            staged = it.x;
        }
        const int xmask = (1 << it.w) - 1;  // it.w: log2 of this item's tile width
        for (int k = threadIdx.x; k < tile_sites; k += ENS_BLOCK) {
            const int x = it.y + (k & xmask);
            const int y = it.z + (k >> it.w);
            if (x < sP.Lx && y < sP.Ly) {
                if (kSplit)
                    fp32split_site<false>(s_src, s_dst, Pc, sP, x, y, flag);  // constants from Pc
                else
                    fp32dev_site<false>(s_src, s_dst, sP, x, y, flag);
            }
        }
        if (claim) {
            // two slots: a slot is rewritten two items later, after every thread has read it
            if (threadIdx.x == 0) s_item[j & 1] = atomicAdd(claim, 1);
            __syncthreads();
            t = s_item[j & 1];
        } else {
            t += gridDim.x;
        }
    }
}

static_assert(sizeof(StepParams) % sizeof(unsigned long long) == 0, "StepParams is copied in words");

}  // namespace ens
}  // namespace lbg

using namespace lbg::ens;

namespace {

int log2_exact(int v) {
    int k = 0;
    while ((1 << k) < v) ++k;
    return (1 << k) == v ? k : -1;
}

struct Candidate {
    int tx, ty;
};

std::vector<Candidate> candidates() {
    std::vector<Candidate> out;
    for (int tx : {32, 64, 128, 256})
        for (int ty : {1, 2, 4, 8, 16})
            if (tx * ty >= 128 && tx * ty <= 2048) out.push_back({tx, ty});
    return out;
}

// The tile width used for a member of width Lx: the widest power of two in [32, tx] that divides
// Lx (no partial tiles at the right edge), else tx; the height keeps tx * ty sites per tile.
int member_tile_x(int Lx, int tx) {
    for (int w = tx; w >= 32; w >>= 1)
        if (Lx % w == 0) return w;
    return tx;
}

long long count_items(const std::vector<lb_params>& m, int tx, int ty) {
    long long n = 0;
    for (const auto& p : m) {
        const int w = member_tile_x(p.Lx, tx), h = tx * ty / w;
        n += (long long)((p.Lx + w - 1) / w) * ((p.Ly + h - 1) / h);
    }
    return n;
}

lb_status fail(cudaError_t e, const char* where) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", where, cudaGetErrorString(e));
    set_last_error(msg);
    return LB_ERR_CUDA;
}

#define ENS_CUDA(call)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return fail(e_, #call);       \
    } while (0)

}  // namespace

struct lb_ensemble {
    std::vector<lb_params> params;
    std::vector<StepParams> sp;
    std::vector<float*> buf0, buf1;
    std::vector<size_t> sites;
    int precision = LB_FP32SPLIT;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* ws = nullptr;
    bool own_ws = false;
    MemberDesc* d_members = nullptr;
    int4* d_items = nullptr;
    long long max_items = 0;
    int nitems = 0;
    int tile_x = 64, tile_y = 4;
    double* stage = nullptr;
    int* flag = nullptr;
    int cur = 0;
    int graph_steps = 100;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_failed = false;
    int grid = 0;         // co-resident blocks of the step kernel (persistent launch)
    bool persistent = false;
    long long total_sites = 0;
};

namespace {

struct EnsLayout {
    std::vector<size_t> off_buf;  // per member, copy A; copy B follows at + buf_bytes[k]
    std::vector<size_t> buf_bytes;
    size_t off_members, off_items, off_stage, off_flag, total;
    long long max_items;
};

EnsLayout ens_layout(const std::vector<lb_params>& m) {
    EnsLayout L;
    size_t off = 0;
    size_t max_sites = 0;
    for (const auto& p : m) {
        const size_t plane = (size_t)p.Lx * ((size_t)p.Ly + 2 * HALO);
        const size_t b = align_up(plane * NPOP * sizeof(float));
        L.off_buf.push_back(off);
        L.buf_bytes.push_back(b);
        off += 2 * b;
        max_sites = std::max(max_sites, (size_t)p.Lx * p.Ly);
    }
    L.max_items = 0;
    for (const auto& c : candidates()) L.max_items = std::max(L.max_items, count_items(m, c.tx, c.ty));
    L.off_members = off;
    off += align_up(m.size() * sizeof(MemberDesc));
    L.off_items = off;
    off += align_up((size_t)L.max_items * sizeof(int4));
    L.off_stage = off;
    off += align_up(4 * max_sites * sizeof(double));
    L.off_flag = off;
    off += ALIGN;
    L.total = off;
    return L;
}

lb_status check_members(int n, const lb_params* m) {
    if (n < 1 || !m) return LB_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        const lb_params& p = m[k];
        if (p.Lx < 4 || p.Ly < 4 || (long long)p.Lx * ((long long)p.Ly + 2 * HALO) >= (1ll << 31) - 1)
            return LB_ERR_ARG;
        // the single-lattice checks: finite relaxation time above 1/2, finite positive wall
        // temperatures, finite gravity
        if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return LB_ERR_ARG;
        if (!(p.T_top > 0.0) || !(p.T_bottom > 0.0) || !std::isfinite(p.T_top) || !std::isfinite(p.T_bottom))
            return LB_ERR_ARG;
        if (!std::isfinite(p.gx) || !std::isfinite(p.gy)) return LB_ERR_ARG;
        if (p.wall_mode != LB_WALL_REST) return LB_ERR_ARG;  // members use the rest closure
    }
    return LB_OK;
}

int opts_precision(const lb_ensemble_opts* o) {
    if (!o || o->precision == 0) return LB_FP32SPLIT;
    return o->precision;
}

lb_status upload_items(lb_ensemble* e, int tx, int ty) {
    std::vector<int4> items;
    items.reserve((size_t)count_items(e->params, tx, ty));
    for (int k = 0; k < (int)e->params.size(); ++k) {
        const lb_params& p = e->params[k];
        const int w = member_tile_x(p.Lx, tx), h = tx * ty / w, wl = log2_exact(w);
        for (int y0 = 0; y0 < p.Ly; y0 += h)
            for (int x0 = 0; x0 < p.Lx; x0 += w) items.push_back(make_int4(k, x0, y0, wl));
    }
    if ((long long)items.size() > e->max_items) return LB_ERR_STATE;
    ENS_CUDA(cudaMemcpyAsync(e->d_items, items.data(), items.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, e->stream));
    ENS_CUDA(cudaStreamSynchronize(e->stream));
    e->nitems = (int)items.size();
    e->tile_x = tx;
    e->tile_y = ty;
    for (int k = 0; k < 2; ++k)
        if (e->graph[k]) {
            cudaGraphExecDestroy(e->graph[k]);
            e->graph[k] = nullptr;
        }
    e->graph_failed = false;
    return LB_OK;
}

cudaError_t launch_ensemble(lb_ensemble* e, int parity) {
    // the lattice constants (r, shell coefficients) are the same for every member: they travel as
    // a kernel parameter (constant bank); each member's own values are staged in shared memory
    // default: the persistent grid claiming items from a counter; on request one block per item
    const int grid = e->persistent ? std::max(1, std::min(e->grid, e->nitems)) : std::max(1, e->nitems);
    // the persistent grid's item counter (a word of the status area), zeroed before each launch
    int* claim = e->persistent ? e->flag + CLAIM_WORD : nullptr;
    if (claim) {
        const cudaError_t m = cudaMemsetAsync(claim, 0, sizeof(int), e->stream);
        if (m != cudaSuccess) return m;
    }
    if (e->precision == LB_FP32SPLIT)
        ensemble_step_kernel<true><<<grid, ENS_BLOCK, 0, e->stream>>>(
            e->sp[0], e->d_members, e->d_items, e->nitems, e->tile_x * e->tile_y, parity, claim, e->flag);
    else
        ensemble_step_kernel<false><<<grid, ENS_BLOCK, 0, e->stream>>>(
            e->sp[0], e->d_members, e->d_items, e->nitems, e->tile_x * e->tile_y, parity, claim, e->flag);
    return cudaGetLastError();
}

bool capture(lb_ensemble* e, int par) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(e->stream, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone)
        return false;
    if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = true;
    for (int k = 0; k < e->graph_steps && ok; ++k) ok = launch_ensemble(e, par ^ (k & 1)) == cudaSuccess;
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(e->stream, &g);
    if (!ok || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    e->graph[par] = ex;
    return true;
}

}  // namespace

extern "C" {

lb_status lb_ensemble_workspace_bytes(int n, const lb_params* members, const lb_ensemble_opts* o,
                                      size_t* bytes) {
    (void)o;
    if (!bytes || check_members(n, members) != LB_OK) return LB_ERR_ARG;
    *bytes = ens_layout(std::vector<lb_params>(members, members + n)).total;
    return LB_OK;
}

void lb_ensemble_free(lb_ensemble* e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    for (int k = 0; k < 2; ++k)
        if (e->graph[k]) cudaGraphExecDestroy(e->graph[k]);
    if (e->own_ws && e->ws) cudaFree(e->ws);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

lb_status lb_ensemble_init(int n, const lb_params* members, const double* const* rho,
                           const double* const* ux, const double* const* uy,
                           const double* const* T, const lb_ensemble_opts* opts,
                           lb_ensemble** out) {
    lbg::NvtxRange nvtx_("lb_ensemble_init");
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    if (check_members(n, members) != LB_OK || !rho || !ux || !uy || !T) return LB_ERR_ARG;
    for (int k = 0; k < n; ++k)
        if (!rho[k] || !ux[k] || !uy[k] || !T[k]) return LB_ERR_ARG;
    const int prec = opts_precision(opts);
    if (prec != LB_FP32SPLIT && prec != LB_FP32DEV) return LB_ERR_ARG;
    int gsteps = opts && opts->graph_steps ? opts->graph_steps : 100;
    if (gsteps < 2 || (gsteps & 1)) return LB_ERR_ARG;
    int tx = opts && opts->tile_x ? opts->tile_x : 64;
    int ty = opts && opts->tile_y ? opts->tile_y : 4;
    if (log2_exact(tx) < 0 || ty < 1 || tx * ty < 32 || tx * ty > 4096) return LB_ERR_ARG;

    std::vector<lb_params> m(members, members + n);
    for (auto& p : m) p.precision = prec;
    const EnsLayout L = ens_layout(m);
    if (count_items(m, tx, ty) > L.max_items) return LB_ERR_ARG;
    if (opts && opts->workspace &&
        (opts->workspace_bytes < L.total || ((uintptr_t)opts->workspace % ALIGN) != 0))
        return LB_ERR_ARG;

    lb_ensemble* e = new (std::nothrow) lb_ensemble();
    if (!e) return LB_ERR_ALLOC;
    e->params = m;
    e->precision = prec;
    e->graph_steps = gsteps;
    e->max_items = L.max_items;
    e->persistent = !(opts && opts->per_item);
    if (opts && opts->stream) {
        e->stream = (cudaStream_t)opts->stream;
    } else {
        cudaError_t ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            delete e;
            return fail(ce, "cudaStreamCreateWithFlags");
        }
        e->own_stream = true;
    }
    if (opts && opts->workspace) {
        e->ws = (char*)opts->workspace;
    } else {
        cudaError_t ce = cudaMalloc((void**)&e->ws, L.total);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            e->ws = nullptr;
            lb_ensemble_free(e);
            char msg[128];
            std::snprintf(msg, sizeof msg, "cudaMalloc(%zu) for the ensemble failed", L.total);
            set_last_error(msg);
            return LB_ERR_ALLOC;
        }
        e->own_ws = true;
    }
    e->d_members = (MemberDesc*)(e->ws + L.off_members);
    e->d_items = (int4*)(e->ws + L.off_items);
    e->stage = (double*)(e->ws + L.off_stage);
    e->flag = (int*)(e->ws + L.off_flag);

    std::vector<MemberDesc> hd(n);
    for (int k = 0; k < n; ++k) {
        StepParams sp;
        fill_step_params(m[k], sp);
        e->sp.push_back(sp);
        e->buf0.push_back((float*)(e->ws + L.off_buf[k]));
        e->buf1.push_back((float*)(e->ws + L.off_buf[k] + L.buf_bytes[k]));
        e->sites.push_back((size_t)m[k].Lx * m[k].Ly);
        e->total_sites += (long long)m[k].Lx * m[k].Ly;
        hd[k].P = sp;
        hd[k].buf[0] = e->buf0[k];
        hd[k].buf[1] = e->buf1[k];
    }
    lb_status st = LB_OK;
    do {
        cudaError_t ce = cudaMemcpyAsync(e->d_members, hd.data(), n * sizeof(MemberDesc),
                                         cudaMemcpyHostToDevice, e->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(e->flag, 0, sizeof(int), e->stream);
        for (int k = 0; k < n && ce == cudaSuccess; ++k) {
            const size_t ns = e->sites[k];
            const double* src[4] = {rho[k], ux[k], uy[k], T[k]};
            for (int f = 0; f < 4 && ce == cudaSuccess; ++f)
                ce = cudaMemcpyAsync(e->stage + f * ns, src[f], ns * sizeof(double),
                                     cudaMemcpyHostToDevice, e->stream);
            if (ce == cudaSuccess)
                ce = launch_init_fp32dev(e->stage, e->stage + ns, e->stage + 2 * ns, e->stage + 3 * ns,
                                         e->buf0[k], e->sp[k], e->flag, e->stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);  // staging is reused
        }
        if (ce != cudaSuccess) {
            st = fail(ce, "ensemble initialisation");
            break;
        }
        int per_sm = 0, dev = 0, sms = 0;
        ce = cudaGetDevice(&dev);
        if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce == cudaSuccess)
            ce = prec == LB_FP32SPLIT
                     ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_step_kernel<true>,
                                                                     ENS_BLOCK, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_step_kernel<false>,
                                                                     ENS_BLOCK, 0);
        if (ce != cudaSuccess) {
            st = fail(ce, "occupancy query");
            break;
        }
        e->grid = std::max(1, per_sm) * std::max(1, sms);
        st = upload_items(e, tx, ty);
    } while (0);
    if (st != LB_OK) {
        lb_ensemble_free(e);
        return st;
    }
    *out = e;
    return LB_OK;
}

lb_status lb_ensemble_step(lb_ensemble* e, int n) {
    lbg::NvtxRange nvtx_("lb_ensemble_step");
    if (!e || n < 0) return LB_ERR_ARG;
    while (n >= e->graph_steps && !e->graph_failed) {
        if (!e->graph[e->cur] && !capture(e, e->cur)) {
            e->graph_failed = true;
            break;
        }
        ENS_CUDA(cudaGraphLaunch(e->graph[e->cur], e->stream));
        n -= e->graph_steps;  // even: parity unchanged
    }
    for (; n > 0; --n) {
        ENS_CUDA(launch_ensemble(e, e->cur));
        e->cur ^= 1;
    }
    return LB_OK;
}

lb_status lb_ensemble_sync(lb_ensemble* e) {
    if (!e) return LB_ERR_ARG;
    ENS_CUDA(cudaStreamSynchronize(e->stream));
    int h = 0;
    ENS_CUDA(cudaMemcpyAsync(&h, e->flag, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    ENS_CUDA(cudaStreamSynchronize(e->stream));
    if (h) {
        ENS_CUDA(cudaMemsetAsync(e->flag, 0, sizeof(int), e->stream));
        ENS_CUDA(cudaStreamSynchronize(e->stream));
        return (h & 2) ? LB_ERR_RANGE : LB_ERR_NONFINITE;
    }
    return LB_OK;
}

lb_status lb_ensemble_autotune(lb_ensemble* e, int steps, int* tile_x, int* tile_y, double* mlups) {
    lbg::NvtxRange nvtx_("lb_ensemble_autotune");
    if (!e || steps < 1) return LB_ERR_ARG;
    cudaEvent_t a, b;
    ENS_CUDA(cudaEventCreate(&a));
    ENS_CUDA(cudaEventCreate(&b));
    double best = -1.0;
    Candidate bestc{e->tile_x, e->tile_y};
    lb_status st = LB_OK;
    for (const auto& c : candidates()) {
        st = upload_items(e, c.tx, c.ty);
        if (st != LB_OK) break;
        // trial launches read the current copy and write the other one without swapping
        cudaError_t ce = launch_ensemble(e, e->cur);
        if (ce == cudaSuccess) ce = cudaEventRecord(a, e->stream);
        for (int k = 0; k < steps && ce == cudaSuccess; ++k) ce = launch_ensemble(e, e->cur);
        if (ce == cudaSuccess) ce = cudaEventRecord(b, e->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(b);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, b);
        if (ce != cudaSuccess) {
            st = fail(ce, "autotune trial");
            break;
        }
        const double rate = (double)e->total_sites * steps / (ms * 1e-3) / 1e6;
        if (rate > best) {
            best = rate;
            bestc = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != LB_OK) return st;
    st = upload_items(e, bestc.tx, bestc.ty);
    if (st != LB_OK) return st;
    if (tile_x) *tile_x = bestc.tx;
    if (tile_y) *tile_y = bestc.ty;
    if (mlups) *mlups = best;
    return LB_OK;
}

lb_status lb_ensemble_info(const lb_ensemble* e, int* tile_x, int* tile_y, int* ntiles,
                           long long* sites) {
    if (!e) return LB_ERR_ARG;
    if (tile_x) *tile_x = e->tile_x;
    if (tile_y) *tile_y = e->tile_y;
    if (ntiles) *ntiles = e->nitems;
    if (sites) *sites = e->total_sites;
    return LB_OK;
}

lb_status lb_ensemble_moments(lb_ensemble* e, int k, double* rho, double* ux, double* uy,
                              double* T) {
    if (!e || k < 0 || k >= (int)e->params.size()) return LB_ERR_ARG;
    const size_t n = e->sites[k];
    const float* cur = e->cur ? e->buf1[k] : e->buf0[k];
    ENS_CUDA(launch_moments_fp32dev(cur, e->sp[k], e->stage, e->stage + n, e->stage + 2 * n,
                                    e->stage + 3 * n, 0, e->stream));
    double* dst[4] = {rho, ux, uy, T};
    for (int f = 0; f < 4; ++f)
        if (dst[f])
            ENS_CUDA(cudaMemcpyAsync(dst[f], e->stage + f * n, n * sizeof(double),
                                     cudaMemcpyDeviceToHost, e->stream));
    ENS_CUDA(cudaStreamSynchronize(e->stream));
    return LB_OK;
}

lb_status lb_ensemble_get_populations(lb_ensemble* e, int k, double* f) {
    if (!e || !f || k < 0 || k >= (int)e->params.size()) return LB_ERR_ARG;
    const size_t n = e->sites[k];
    const float* cur = e->cur ? e->buf1[k] : e->buf0[k];
    const size_t skip = (size_t)HALO * e->params[k].Lx;
    for (int i = 0; i < NPOP; ++i) {
        ENS_CUDA(launch_plane_from_dev32(cur + (size_t)i * e->sp[k].plane + skip, e->stage,
                                         shell_w(shell_of(i)), (long long)n, e->stream));
        ENS_CUDA(cudaMemcpyAsync(f + i * n, e->stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                                 e->stream));
        ENS_CUDA(cudaStreamSynchronize(e->stream));
    }
    return LB_OK;
}

}  // extern "C"
