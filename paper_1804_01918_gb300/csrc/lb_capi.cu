// lb_capi.cu -- host runtime behind the C ABI of include/lb_d2q37.h.
//
// A context owns: two population copies (double buffer), a staging area for host exchange
// (4 fields of Lx*Ly doubles, also used plane by plane for population copies), a device status
// word, the stream, and up to two instantiated CUDA graphs of GRAPH_STEPS fused steps (one per
// buffer parity), replayed by lb_step so that short lattices are not launch-bound.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/lb_d2q37.h"
#include "../../include/lb_learned.h"
#include "../../include/lb_slab.h"
#include "d2q37_gpu.cuh"
#include "kernels.cuh"

using namespace lbg;

namespace {

constexpr size_t ALIGN = 256;
constexpr int GRAPH_STEPS = 16;  // even: a replay returns the state to the same buffer

thread_local char g_last_error[256] = "";

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

lb_status cuda_fail(cudaError_t e, const char* where) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
    return LB_ERR_CUDA;
}

#define LB_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

struct Layout {
    size_t esize, plane_elems, buf_bytes, stage_bytes, flag_bytes, total;
    size_t off_a, off_b, off_stage, off_flag;
};

bool valid_sizes(int Lx, int Ly) {
    if (Lx < 4 || Ly < 4) return false;
    const long long full = (long long)Lx * ((long long)Ly + 2 * HALO);
    return full < (1ll << 31) - 1;
}

Layout layout_of(int Lx, int Ly, int precision) {
    Layout L;
    L.esize = precision == LB_FP64 ? sizeof(double) : sizeof(float);
    L.plane_elems = (size_t)Lx * ((size_t)Ly + 2 * HALO);
    L.buf_bytes = align_up(L.plane_elems * NPOP * L.esize);
    L.stage_bytes = align_up((size_t)4 * Lx * Ly * sizeof(double));
    L.flag_bytes = ALIGN;
    L.off_a = 0;
    L.off_b = L.off_a + L.buf_bytes;
    L.off_stage = L.off_b + L.buf_bytes;
    L.off_flag = L.off_stage + L.stage_bytes;
    L.total = L.off_flag + L.flag_bytes;
    return L;
}

lb_status check_params(const lb_params* p) {
    if (!p) return LB_ERR_ARG;
    if (!valid_sizes(p->Lx, p->Ly)) return LB_ERR_ARG;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return LB_ERR_ARG;
    if (!std::isfinite(p->gx) || !std::isfinite(p->gy)) return LB_ERR_ARG;
    if (!(p->T_top > 0.0) || !(p->T_bottom > 0.0) || !std::isfinite(p->T_top) ||
        !std::isfinite(p->T_bottom))
        return LB_ERR_ARG;
    if (p->precision != LB_FP64 && p->precision != LB_FP32DEV && p->precision != LB_FP32SPLIT)
        return LB_ERR_ARG;
    if (p->wall_mode != LB_WALL_REST && p->wall_mode != LB_WALL_MIRROR) return LB_ERR_ARG;
    return LB_OK;
}

}  // namespace

namespace lbg {
// r = 1 / sqrt(sum_i w_i c_ix^2): xi = r c puts the reference temperature at 1.
double thermal_scale() {
    double m2 = 0.0;
    for (int i = 0; i < NPOP; ++i) m2 += shell_w(shell_of(i)) * (double)(cx_of(i) * cx_of(i));
    return 1.0 / std::sqrt(m2);
}

// StepParams is passed by value as a kernel parameter: it must fit the classic 4 KB parameter space.
static_assert(sizeof(StepParams) <= 4096, "StepParams must fit the 4 KB kernel parameter space");

void fill_step_params(const lb_params& p, StepParams& sp) {
    std::memset(&sp, 0, sizeof sp);
    sp.Lx = p.Lx;
    sp.Ly = p.Ly;
    sp.y_periodic = p.y_periodic ? 1 : 0;
    sp.wall_mode = p.wall_mode == LB_WALL_MIRROR ? 1 : 0;
    sp.T_bot = p.T_bottom;
    sp.T_top = p.T_top;
    sp.plane = (long long)p.Lx * ((long long)p.Ly + 2 * HALO);
    {
        int l = 0;
        while ((1ll << l) < (long long)p.Lx) ++l;
        const unsigned long long num = 1ull << (31 + l);
        sp.row_m = (unsigned)((num + (unsigned long long)p.Lx - 1) / (unsigned long long)p.Lx);
        sp.row_s = 31 + l;
    }
    const double r = thermal_scale();
    sp.r = r;
    sp.r2 = r * r;
    sp.omega = 1.0 / p.tau;
    sp.omc = 1.0 - 1.0 / p.tau;
    sp.gx = p.gx;
    sp.gy = p.gy;
    sp.tgx = p.tau * p.gx;
    sp.tgy = p.tau * p.gy;
    sp.dT_force = p.tau * (1.0 - p.tau) * (p.gx * p.gx + p.gy * p.gy) / DIM;
    for (int s = 0; s < NSHELL; ++s) {
        const double X = sp.r2 * shell_c2(s);
        sp.sh[s].w = shell_w(s);
        sp.sh[s].alpha = (X - DIM) / 2.0;
        sp.sh[s].beta = (DIM + 2.0 - X) / 4.0;
        sp.sh[s].gamma = (X * X - 2.0 * (DIM + 2.0) * X + DIM * (DIM + 2.0)) / 8.0;
        sp.sh[s].delta = (X - DIM - 4.0) / 4.0;
        sp.sh[s].eps = (X - DIM - 2.0) / 2.0;
        const double w = sp.sh[s].w, k = shell_kappa(s);
        sp.sh[s].q_a0 = 2.0 * w;
        sp.sh[s].q_a1 = 2.0 * w * X;
        sp.sh[s].q_a2 = 0.5 * w * X * X;
        sp.sh[s].q_b0 = 8.0 * k * w;
        sp.sh[s].q_b1 = 4.0 * k * w * X;
        sp.sh[s].q_e0 = 16.0 * k * k * w;
        sp.sh[s].q_co = 32.0 * k * k * k * w / 3.0;
    }
    constexpr double lambda = 0.25;
    sp.lr2 = lambda * sp.r2;
    sp.lrtgx = lambda * r * sp.tgx;
    sp.lrtgy = lambda * r * sp.tgy;
    sp.hdT = 0.5 * (sp.dT_force - 1.0);
    sp.mu4 = -1.0 / (4.0 * lambda * lambda * sp.r2);
    sp.om48 = std::ldexp(sp.omega, -48);
    {
        const double ub = 0.25 * r * FX_UMAX, hb = FX_HB;
        std::memcpy(&sp.fx_ub, &ub, 8);
        std::memcpy(&sp.fx_hb, &hb, 8);
        for (int s = 1; s < NSHELL; ++s) {
            const ShellCoef& c = sp.sh[s];
            const int co = fx_coarse_unit(s);
            ShellFx& q = sp.shfx[s];
            q.b1 = std::llround(std::ldexp(c.q_b1, co));
            q.b0 = std::llround(std::ldexp(c.q_b0, co + 2));
            q.e0 = std::llround(std::ldexp(c.q_e0, co));
            q.co = std::llround(std::ldexp(c.q_co, co + 2));
        }
    }
    sp.r_f = (float)sp.r;
    sp.r2_f = (float)sp.r2;
    sp.omega_f = (float)sp.omega;
    sp.omc_f = (float)sp.omc;
    sp.gx_f = (float)sp.gx;
    sp.gy_f = (float)sp.gy;
    sp.tgx_f = (float)sp.tgx;
    sp.tgy_f = (float)sp.tgy;
    sp.dT_force_f = (float)sp.dT_force;
    sp.lr_f = (float)(0.25 * sp.r);
    for (int s = 0; s < NSHELL; ++s) {
        sp.sh32[s].w = (float)sp.sh[s].w;
        sp.sh32[s].alpha = (float)sp.sh[s].alpha;
        sp.sh32[s].beta = (float)sp.sh[s].beta;
        sp.sh32[s].gamma = (float)sp.sh[s].gamma;
        sp.sh32[s].delta = (float)sp.sh[s].delta;
        sp.sh32[s].eps = (float)sp.sh[s].eps;
        const double w = sp.sh[s].w, X = sp.r2 * shell_c2(s);
        sp.sh32[s].q_a0 = (float)w;
        sp.sh32[s].q_a1 = (float)(2.0 * w * X);
        sp.sh32[s].q_a2 = (float)(0.5 * w * X * X);
        sp.sh32[s].q_e0 = (float)(16.0 * w);
        sp.sh32[s].q_e1 = (float)(8.0 * w * X);
        sp.sh32[s].q_b0 = (float)(8.0 * w);
        sp.sh32[s].q_b1 = (float)(4.0 * w * X);
        sp.sh32[s].q_c = (float)(32.0 * w / 3.0);
    }
    for (int i = 0; i < NPOP; ++i) {
        sp.plane_b32[i] = 4ll * i * sp.plane;
        sp.pull_b32[i] = 4ll * ((long long)i * sp.plane - (long long)cy_of(i) * p.Lx - cx_of(i));
    }
    // rest equilibrium per unit density: w (1 + alpha theta + gamma theta^2) at u = 0
    for (int i = 0; i < NPOP; ++i) {
        const ShellCoef& c = sp.sh[shell_of(i)];
        const double tb = p.T_bottom - 1.0, tt = p.T_top - 1.0;
        sp.wall_bot[i] = c.w * (1.0 + c.alpha * tb + c.gamma * tb * tb);
        sp.wall_top[i] = c.w * (1.0 + c.alpha * tt + c.gamma * tt * tt);
    }
}

// Record the message lb_last_error() returns on this thread (used by the allocation-free entry
// point, which lives in its own translation unit).
void set_last_error(const char* msg) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s", msg);
}
}  // namespace lbg

struct lb_ctx {
    lb_params p;
    StepParams sp;
    Layout L;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* ws = nullptr;
    bool own_ws = false;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    double* stage = nullptr;
    int* flag = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_failed = false;
    long long steps = 0;
    LearnedState* learned = nullptr;  // learned collide, when set
    lb_mlp* own_net = nullptr;        // network owned by the context (lb_collide_train/load)
    alignas(64) unsigned char tmap[2][128];  // TMA descriptors of the two FP32 population copies
    bool tma_ready = false;                  // tensor maps built (FP32SPLIT, Lx % 4 == 0)
    bool use_tma = false;                    // step with the TMA-staged kernel
    bool band_done = false;                  // slab: boundary bands of a split step written, swap pending
    cudaEvent_t ev = nullptr;                // slab: orders an exchange after this context's queued work
};

namespace {

lb_status launch_one_step(lb_ctx* c) {
    cudaError_t e;
    if (c->learned)
        e = launch_step_learned((const float*)c->buf[c->cur], (float*)c->buf[c->cur ^ 1], c->sp,
                                c->learned, c->flag, c->stream);
    else if (c->p.precision == LB_FP64)
        e = launch_step_fp64((const double*)c->buf[c->cur], (double*)c->buf[c->cur ^ 1], c->sp,
                             c->flag, c->stream);
    else if (c->p.precision == LB_FP32SPLIT && c->use_tma)
        e = launch_step_fp32split_tma(c->tmap[c->cur], (const float*)c->buf[c->cur],
                                      (float*)c->buf[c->cur ^ 1], c->sp, c->flag,
                                      fp32split_tma_grid(), c->stream);
    else if (c->p.precision == LB_FP32SPLIT)
        e = launch_step_fp32split((const float*)c->buf[c->cur], (float*)c->buf[c->cur ^ 1], c->sp,
                                  c->flag, c->stream);
    else
        e = launch_step_fp32dev((const float*)c->buf[c->cur], (float*)c->buf[c->cur ^ 1], c->sp,
                                c->flag, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    c->cur ^= 1;
    c->steps += 1;
    return LB_OK;
}

// Capture GRAPH_STEPS fused steps starting from buffer parity `par` into c->graph[par].
bool capture_graph(lb_ctx* c, int par) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone)
        return false;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int saved_cur = c->cur;
    const long long saved_steps = c->steps;
    c->cur = par;
    bool ok = true;
    for (int k = 0; k < GRAPH_STEPS && ok; ++k) ok = launch_one_step(c) == LB_OK;
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    c->cur = saved_cur;
    c->steps = saved_steps;
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
    c->graph[par] = ex;
    return true;
}

lb_status read_flag(lb_ctx* c) {
    int h = 0;
    LB_CUDA(cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    if (h) {
        LB_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
        LB_CUDA(cudaStreamSynchronize(c->stream));
        return (h & 2) ? LB_ERR_RANGE : LB_ERR_NONFINITE;
    }
    return LB_OK;
}

lb_status launch_moments(lb_ctx* c, double* rho, double* ux, double* uy, double* T, int half_step = 0) {
    cudaError_t e;
    if (c->p.precision == LB_FP64)
        e = launch_moments_fp64((const double*)c->buf[c->cur], c->sp, rho, ux, uy, T, half_step, c->stream);
    else
        e = launch_moments_fp32dev((const float*)c->buf[c->cur], c->sp, rho, ux, uy, T, half_step,
                                   c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments kernel launch");
    return LB_OK;
}

lb_status rewrite_halos(lb_ctx* c) {
    if (c->p.y_periodic) return LB_OK;
    cudaError_t e = c->p.precision == LB_FP64
                        ? launch_halo_fp64((double*)c->buf[c->cur], c->sp, c->flag, c->stream)
                        : launch_halo_fp32dev((float*)c->buf[c->cur], c->sp, c->flag, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "halo kernel launch");
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_status_str(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_ERR_ARG: return "invalid argument";
        case LB_ERR_ALLOC: return "allocation failed";
        case LB_ERR_CUDA: return "CUDA error";
        case LB_ERR_NONFINITE: return "non-finite or non-positive density/temperature";
        case LB_ERR_STATE: return "invalid state";
        case LB_ERR_RANGE: return "population deviation outside the exact-split range";
    }
    return "unknown status";
}

const char* lb_last_error(void) { return g_last_error; }

lb_status lb_velocity_set(int* cx, int* cy, double* w, double* r) {
    for (int i = 0; i < NPOP; ++i) {
        if (cx) cx[i] = cx_of(i);
        if (cy) cy[i] = cy_of(i);
        if (w) w[i] = shell_w(shell_of(i));
    }
    if (r) *r = thermal_scale();
    return LB_OK;
}

lb_status lb_workspace_bytes(const lb_params* p, size_t* bytes) {
    if (!p || !bytes || !valid_sizes(p->Lx, p->Ly)) return LB_ERR_ARG;
    if (p->precision != LB_FP64 && p->precision != LB_FP32DEV && p->precision != LB_FP32SPLIT)
        return LB_ERR_ARG;
    *bytes = layout_of(p->Lx, p->Ly, p->precision).total;
    return LB_OK;
}

void lb_free(lb_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
    learned_destroy(c->learned);
    lb_mlp_free(c->own_net);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

namespace {
// lb_init of a whole lattice (cuts = 0) or of one slab of a larger lattice (cuts: bit 0 = cut
// below row 0, bit 1 = cut above row Ly - 1; those sides get no wall halo rows).
lb_status init_ctx(const lb_params* p, int cuts, const double* rho, const double* ux, const double* uy,
                   const double* T, lb_ctx** out) {
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    lb_status st = check_params(p);
    if (st != LB_OK) return st;
    if (!rho || !ux || !uy || !T) return LB_ERR_ARG;
    const Layout L = layout_of(p->Lx, p->Ly, p->precision);
    if (p->workspace) {
        if (p->workspace_bytes < L.total || ((uintptr_t)p->workspace % ALIGN) != 0) return LB_ERR_ARG;
    }
    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return LB_ERR_ALLOC;
    c->p = *p;
    c->L = L;
    fill_step_params(*p, c->sp);
    c->sp.cut = cuts;
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        c->own_stream = true;
    }
    if (p->workspace) {
        c->ws = (char*)p->workspace;
    } else {
        cudaError_t e = cudaMalloc((void**)&c->ws, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->ws = nullptr;
            lb_free(c);
            std::snprintf(g_last_error, sizeof g_last_error, "cudaMalloc(%zu): %s", L.total,
                          cudaGetErrorString(e));
            return LB_ERR_ALLOC;
        }
        c->own_ws = true;
    }
    c->buf[0] = c->ws + L.off_a;
    c->buf[1] = c->ws + L.off_b;
    if (p->precision == LB_FP32SPLIT && p->Lx % 4 == 0) {
        c->tma_ready = make_fp32_tensor_map(c->tmap[0], (const float*)c->buf[0], c->sp) == cudaSuccess &&
                       make_fp32_tensor_map(c->tmap[1], (const float*)c->buf[1], c->sp) == cudaSuccess;
        c->use_tma = false;  // opt-in: measured slower than plain loads for this issue-bound kernel
    }
    c->stage = (double*)(c->ws + L.off_stage);
    c->flag = (int*)(c->ws + L.off_flag);

    const size_t n = (size_t)p->Lx * p->Ly;
    lb_status rs = LB_OK;
    do {
        cudaError_t e = cudaSuccess;
        const double* src[4] = {rho, ux, uy, T};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            e = cudaMemcpyAsync(c->stage + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream);
        }
        if (e != cudaSuccess) { rs = cuda_fail(e, "cudaMemcpyAsync(fields)"); break; }
        e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) { rs = cuda_fail(e, "cudaMemsetAsync(flag)"); break; }
        if (p->precision == LB_FP64)
            e = launch_init_fp64(c->stage, c->stage + n, c->stage + 2 * n, c->stage + 3 * n,
                                 (double*)c->buf[0], c->sp, c->flag, c->stream);
        else
            e = launch_init_fp32dev(c->stage, c->stage + n, c->stage + 2 * n, c->stage + 3 * n,
                                    (float*)c->buf[0], c->sp, c->flag, c->stream);
        if (e != cudaSuccess) { rs = cuda_fail(e, "init kernel launch"); break; }
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { rs = cuda_fail(e, "cudaStreamSynchronize(init)"); break; }
    } while (0);
    if (rs != LB_OK) {
        lb_free(c);
        return rs;
    }
    *out = c;
    return LB_OK;
}
}  // namespace

extern "C" {

lb_status lb_init(const lb_params* p, const double* rho, const double* ux, const double* uy,
                  const double* T, lb_ctx** out) {
    lbg::NvtxRange nvtx_("lb_init");
    return init_ctx(p, 0, rho, ux, uy, T, out);
}

lb_status lb_step(lb_ctx* c, int n) {
    lbg::NvtxRange nvtx_("lb_step");
    if (!c || n < 0) return LB_ERR_ARG;
    // a slab needs the ghost-row exchange between its steps
    if ((c->sp.cut && n > 1) || c->band_done) return LB_ERR_STATE;
    // the learned step's check schedule varies from step to step: launch it directly
    while (n >= GRAPH_STEPS && !c->graph_failed && !c->learned) {
        const int par = c->cur;
        if (!c->graph[par] && !capture_graph(c, par)) {
            c->graph_failed = true;
            break;
        }
        LB_CUDA(cudaGraphLaunch(c->graph[par], c->stream));
        c->steps += GRAPH_STEPS;
        n -= GRAPH_STEPS;
    }
    for (; n > 0; --n) {
        lb_status st = launch_one_step(c);
        if (st != LB_OK) return st;
    }
    return LB_OK;
}

lb_status lb_propagate(lb_ctx* c) {
    lbg::NvtxRange nvtx_("lb_propagate");
    if (!c) return LB_ERR_ARG;
    cudaError_t e = c->p.precision == LB_FP64
                        ? launch_propagate_fp64((const double*)c->buf[c->cur],
                                                (double*)c->buf[c->cur ^ 1], c->sp, c->stream)
                        : launch_propagate_fp32dev((const float*)c->buf[c->cur],
                                                   (float*)c->buf[c->cur ^ 1], c->sp, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "propagate kernel launch");
    c->cur ^= 1;
    c->steps += 1;
    return LB_OK;
}

lb_status lb_set_staging(lb_ctx* c, int use_tma) {
    if (!c) return LB_ERR_ARG;
    if (use_tma && (!c->tma_ready || c->sp.cut)) return LB_ERR_STATE;
    LB_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
    c->graph_failed = false;
    c->use_tma = use_tma != 0;
    return LB_OK;
}

lb_status lb_collide(lb_ctx* c) {
    lbg::NvtxRange nvtx_("lb_collide");
    if (!c) return LB_ERR_ARG;
    if (c->p.precision != LB_FP64 || c->learned) return LB_ERR_STATE;
    cudaError_t e = launch_collide_fp64((double*)c->buf[c->cur], c->sp, c->flag, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "collide kernel launch");
    return LB_OK;
}

lb_status lb_sync(lb_ctx* c) {
    if (!c) return LB_ERR_ARG;
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return read_flag(c);
}

lb_status lb_moments_device(lb_ctx* c, double* rho, double* ux, double* uy, double* T) {
    if (!c) return LB_ERR_ARG;
    const size_t n = (size_t)c->p.Lx * c->p.Ly;
    return launch_moments(c, rho ? rho : c->stage, ux ? ux : c->stage + n,
                          uy ? uy : c->stage + 2 * n, T ? T : c->stage + 3 * n);
}

namespace {
lb_status moments_to_host(lb_ctx* c, double* rho, double* ux, double* uy, double* T, int half_step) {
    lbg::NvtxRange nvtx_("lb_moments");
    if (!c) return LB_ERR_ARG;
    const size_t n = (size_t)c->p.Lx * c->p.Ly;
    lb_status st = launch_moments(c, c->stage, c->stage + n, c->stage + 2 * n, c->stage + 3 * n, half_step);
    if (st != LB_OK) return st;
    double* dst[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            LB_CUDA(cudaMemcpyAsync(dst[k], c->stage + k * n, n * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return read_flag(c);
}
}  // namespace

lb_status lb_moments(lb_ctx* c, double* rho, double* ux, double* uy, double* T) {
    return moments_to_host(c, rho, ux, uy, T, 0);
}

lb_status lb_moments_half_step(lb_ctx* c, double* rho, double* ux, double* uy, double* T) {
    return moments_to_host(c, rho, ux, uy, T, 1);
}

lb_status lb_get_populations(lb_ctx* c, double* f) {
    lbg::NvtxRange nvtx_("lb_get_populations");
    if (!c || !f) return LB_ERR_ARG;
    const size_t n = (size_t)c->p.Lx * c->p.Ly;
    const size_t skip = (size_t)HALO * c->p.Lx;
    for (int i = 0; i < NPOP; ++i) {
        if (c->p.precision == LB_FP64) {
            const double* src = (const double*)c->buf[c->cur] + (size_t)i * c->sp.plane + skip;
            LB_CUDA(cudaMemcpyAsync(f + i * n, src, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
        } else {
            const float* src = (const float*)c->buf[c->cur] + (size_t)i * c->sp.plane + skip;
            cudaError_t e = launch_plane_from_dev32(src, c->stage, shell_w(shell_of(i)), (long long)n,
                                                    c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "plane conversion launch");
            LB_CUDA(cudaMemcpyAsync(f + i * n, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
            LB_CUDA(cudaStreamSynchronize(c->stream));  // the staging plane is reused
        }
    }
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return read_flag(c);
}

lb_status lb_set_populations(lb_ctx* c, const double* f) {
    lbg::NvtxRange nvtx_("lb_set_populations");
    if (!c || !f) return LB_ERR_ARG;
    const size_t n = (size_t)c->p.Lx * c->p.Ly;
    const size_t skip = (size_t)HALO * c->p.Lx;
    for (int i = 0; i < NPOP; ++i) {
        if (c->p.precision == LB_FP64) {
            double* dst = (double*)c->buf[c->cur] + (size_t)i * c->sp.plane + skip;
            LB_CUDA(cudaMemcpyAsync(dst, f + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream));
        } else {
            float* dst = (float*)c->buf[c->cur] + (size_t)i * c->sp.plane + skip;
            LB_CUDA(cudaMemcpyAsync(c->stage, f + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream));
            cudaError_t e = launch_plane_to_dev32(c->stage, dst, shell_w(shell_of(i)), (long long)n,
                                                  c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "plane conversion launch");
        }
    }
    lb_status st = rewrite_halos(c);
    if (st != LB_OK) return st;
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_collect_pairs(lb_ctx* c, const int* sites, int n, float* pre, float* post) {
    if (!c || !sites || !pre || !post || n < 0) return LB_ERR_ARG;
    if (c->p.precision != LB_FP32SPLIT) return LB_ERR_STATE;
    if (n == 0) return LB_OK;
    cudaError_t e = launch_pairs((const float*)c->buf[c->cur], c->sp, sites, n, pre, post, c->flag,
                                 c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pairs kernel launch");
    return LB_OK;
}

lb_status lb_set_collide_learned(lb_ctx* c, const lb_mlp* net, double bound, int check_every) {
    if (!c || !net) return LB_ERR_ARG;
    if (c->p.precision != LB_FP32SPLIT || c->sp.cut) return LB_ERR_STATE;
    LearnedState* ls = nullptr;
    lb_status st = learned_create(net, c->p.Lx, c->p.Ly, bound, check_every, &ls);
    if (st != LB_OK) return st;
    LB_CUDA(cudaStreamSynchronize(c->stream));
    learned_destroy(c->learned);
    c->learned = ls;
    return LB_OK;
}

lb_status lb_collide_train(lb_ctx* c, const float* pre, const float* post, size_t npairs, int epochs,
                           uint64_t seed) {
    lbg::NvtxRange nvtx_("lb_collide_train");
    if (!c || !pre || !post || npairs < (size_t)LB_MLP_TILE || epochs < 1) return LB_ERR_ARG;
    if (c->p.precision != LB_FP32SPLIT || c->p.Lx % 32 || c->p.Ly % 32) return LB_ERR_STATE;
    if (npairs > (size_t)((1ll << 31) - 1)) return LB_ERR_ARG;
    if (!c->own_net) {
        lb_status st = lb_mlp_create(seed, &c->own_net);
        if (st != LB_OK) return st;
    }
    const long long n = (long long)npairs;
    const int batch = (int)std::min<long long>(4096, n / LB_MLP_TILE * LB_MLP_TILE);
    lb_status st = lb_mlp_train(c->own_net, pre, post, n, epochs, batch, 1e-3f, seed, nullptr, c->stream);
    if (st != LB_OK) return st;
    return lb_set_collide_learned(c, c->own_net, 1e-4, 1);
}

namespace {
constexpr char MLP_MAGIC[8] = {'L', 'B', 'M', 'L', 'P', '3', '7', '\0'};
constexpr uint32_t MLP_FILE_VERSION = 1;
constexpr uint32_t MLP_NNORM = 4 * 37;
}  // namespace

lb_status lb_collide_save(lb_ctx* c, const char* path) {
    if (!c || !path) return LB_ERR_ARG;
    const lb_mlp* net = nullptr;
    double bound = 0.0;
    int check_every = 1;
    lb_status st = learned_info(c->learned, &net, &bound, &check_every);
    if (st != LB_OK) return st;
    std::vector<float> params(LB_MLP_NPARAM), norm(MLP_NNORM);
    st = lb_mlp_get_params(net, params.data(), norm.data());
    if (st != LB_OK) return st;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return LB_ERR_ARG;
    const uint32_t head[3] = {MLP_FILE_VERSION, (uint32_t)LB_MLP_NPARAM, MLP_NNORM};
    const int32_t ce = check_every;
    bool ok = std::fwrite(MLP_MAGIC, 1, 8, fp) == 8 && std::fwrite(head, 4, 3, fp) == 3 &&
              std::fwrite(&ce, 4, 1, fp) == 1 && std::fwrite(&bound, 8, 1, fp) == 1 &&
              std::fwrite(params.data(), 4, params.size(), fp) == params.size() &&
              std::fwrite(norm.data(), 4, norm.size(), fp) == norm.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LB_OK : LB_ERR_ARG;
}

lb_status lb_collide_load(lb_ctx* c, const char* path) {
    if (!c || !path) return LB_ERR_ARG;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LB_ERR_ARG;
    char magic[8];
    uint32_t head[3];
    int32_t ce = 0;
    double bound = 0.0;
    std::vector<float> params(LB_MLP_NPARAM), norm(MLP_NNORM);
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, MLP_MAGIC, 8) == 0 &&
              std::fread(head, 4, 3, fp) == 3 && head[0] == MLP_FILE_VERSION &&
              head[1] == (uint32_t)LB_MLP_NPARAM && head[2] == MLP_NNORM && std::fread(&ce, 4, 1, fp) == 1 &&
              std::fread(&bound, 8, 1, fp) == 1 &&
              std::fread(params.data(), 4, params.size(), fp) == params.size() &&
              std::fread(norm.data(), 4, norm.size(), fp) == norm.size();
    std::fclose(fp);
    if (!ok || ce < 1 || !(bound >= 0.0)) return LB_ERR_ARG;
    if (!c->own_net) {
        lb_status st = lb_mlp_create(0, &c->own_net);
        if (st != LB_OK) return st;
    }
    lb_status st = lb_mlp_set_params(c->own_net, params.data(), norm.data());
    if (st != LB_OK) return st;
    return lb_set_collide_learned(c, c->own_net, bound, ce);
}

lb_status lb_set_collide_plain(lb_ctx* c) {
    if (!c) return LB_ERR_ARG;
    LB_CUDA(cudaStreamSynchronize(c->stream));
    learned_destroy(c->learned);
    c->learned = nullptr;
    return LB_OK;
}

lb_status lb_learned_stats(lb_ctx* c, long long* checked, long long* fallback, double* max_residual) {
    if (!c) return LB_ERR_ARG;
    if (!c->learned) return LB_ERR_STATE;
    return learned_stats(c->learned, checked, fallback, max_residual, c->stream);
}

lb_status lb_learned_tiles(lb_ctx* c, unsigned char* modes, int n) {
    if (!c || !modes) return LB_ERR_ARG;
    if (!c->learned) return LB_ERR_STATE;
    const int ntiles = (c->p.Lx / 32) * (c->p.Ly / 32);
    if (n != ntiles) return LB_ERR_ARG;
    return learned_tiles(c->learned, ntiles, modes, c->stream);
}

lb_status lb_steps_done(const lb_ctx* c, long long* n) {
    if (!c || !n) return LB_ERR_ARG;
    *n = c->steps;
    return LB_OK;
}

// ---- slabs of a lattice cut along y (include/lb_slab.h) ----

lb_status lb_init_slab(const lb_params* p, int cuts, const double* rho, const double* ux, const double* uy,
                       const double* T, lb_ctx** out) {
    lbg::NvtxRange nvtx_("lb_init_slab");
    if (!p || cuts < 0 || cuts > 3 || (cuts && p->y_periodic)) return LB_ERR_ARG;
    if (cuts && p->Ly < 2 * HALO) return LB_ERR_ARG;
    lb_status st = init_ctx(p, cuts, rho, ux, uy, T, out);
    if (st != LB_OK) return st;
    cudaError_t e = cudaEventCreateWithFlags(&(*out)->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lb_free(*out);
        *out = nullptr;
        return cuda_fail(e, "cudaEventCreateWithFlags");
    }
    return LB_OK;
}

lb_status lb_slab_step(lb_ctx* c, int part) {
    lbg::NvtxRange nvtx_("lb_slab_step");
    if (!c || part < 0 || part > 2) return LB_ERR_ARG;
    if (c->learned || c->use_tma) return LB_ERR_STATE;
    if (part == 0) {
        if (c->band_done) return LB_ERR_STATE;
        return launch_one_step(c);
    }
    if ((part == 1) == c->band_done) return LB_ERR_STATE;  // bands first, then the rest
    const int Ly = c->p.Ly;
    const int lo = (c->sp.cut & 1) ? HALO : 0, hi = (c->sp.cut & 2) ? Ly - HALO : Ly;
    auto rows = [&](int r0, int r1) -> cudaError_t {
        if (c->p.precision == LB_FP64)
            return launch_step_fp64_rows((const double*)c->buf[c->cur], (double*)c->buf[c->cur ^ 1], c->sp,
                                         c->flag, r0, r1, c->stream);
        return launch_step_fp32_rows(c->p.precision == LB_FP32SPLIT, (const float*)c->buf[c->cur],
                                     (float*)c->buf[c->cur ^ 1], c->sp, c->flag, r0, r1, c->stream);
    };
    cudaError_t e;
    if (part == 1) {
        e = rows(0, lo);
        if (e == cudaSuccess) e = rows(hi, Ly);
        if (e != cudaSuccess) return cuda_fail(e, "slab band launch");
        c->band_done = true;
        return LB_OK;
    }
    e = rows(lo, hi);
    if (e != cudaSuccess) return cuda_fail(e, "slab interior launch");
    c->band_done = false;
    c->cur ^= 1;
    c->steps += 1;
    return LB_OK;
}

namespace {
// The copy holding the newest state: the one being written while a split step is half done.
void* newest(lb_ctx* c) { return c->buf[c->band_done ? c->cur ^ 1 : c->cur]; }
size_t elem_bytes(const lb_ctx* c) { return c->p.precision == LB_FP64 ? 8 : 4; }
}  // namespace

lb_status lb_slab_pack(lb_ctx* c, int side, void* buf) {
    if (!c || !buf || side < 0 || side > 1) return LB_ERR_ARG;
    cudaError_t e = launch_slab_pack(elem_bytes(c), newest(c), buf, c->sp, side, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab pack launch");
    return LB_OK;
}

lb_status lb_slab_unpack(lb_ctx* c, int side, const void* buf) {
    if (!c || !buf || side < 0 || side > 1) return LB_ERR_ARG;
    if (!(c->sp.cut & (1 << side))) return LB_ERR_ARG;  // a wall side has no ghost rows
    cudaError_t e = launch_slab_unpack(elem_bytes(c), buf, newest(c), c->sp, side, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab unpack launch");
    return LB_OK;
}

lb_status lb_slab_exchange(lb_ctx* lo, lb_ctx* hi) {
    lbg::NvtxRange nvtx_("lb_slab_exchange");
    if (!lo || !hi || lo == hi) return LB_ERR_ARG;
    if (!(lo->sp.cut & 2) || !(hi->sp.cut & 1) || lo->p.Lx != hi->p.Lx || lo->p.precision != hi->p.precision)
        return LB_ERR_ARG;
    if (lo->band_done || hi->band_done || !lo->ev || !hi->ev) return LB_ERR_STATE;
    if (hi->stream != lo->stream) {
        LB_CUDA(cudaEventRecord(hi->ev, hi->stream));
        LB_CUDA(cudaStreamWaitEvent(lo->stream, hi->ev, 0));
    }
    cudaError_t e = launch_slab_exchange(elem_bytes(lo), lo->buf[lo->cur], lo->sp, hi->buf[hi->cur], hi->sp,
                                         lo->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab exchange launch");
    if (hi->stream != lo->stream) {
        LB_CUDA(cudaEventRecord(lo->ev, lo->stream));
        LB_CUDA(cudaStreamWaitEvent(hi->stream, lo->ev, 0));
    }
    return LB_OK;
}

}  // extern "C"
