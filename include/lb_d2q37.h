/*
 * lb_d2q37.h -- C ABI of the GB300 (sm_103a) D2Q37 lattice-Boltzmann time step.
 *
 * The method (arXiv 1804.01918, Sec. 3): each site of a regular 2-D lattice holds 37
 * populations; one time step first propagates them (each population hops up to three sites,
 * Sec. 3 and Fig. 1) and then collides them (mixing that conserves mass, momentum and energy;
 * the model obeys the perfect-gas law p = rho T). Propagate is a pull (Sec. 4, Fig. 3 listing):
 * each population of the new lattice is read from the old lattice at the site displaced by a
 * per-population offset. The full code also applies the boundary conditions (Table 1, "Global").
 *
 * Readings of what the paper leaves to its references (same for every entry point):
 *   - thermal velocities xi_i = r c_i, r = 1.19697977..., over the 37 lattice vectors with
 *     |c_x|, |c_y| <= 3 listed by lb_velocity_set();
 *   - equilibrium: 4th-order Hermite expansion of the Maxwellian in (rho, u, T);
 *   - collide: BGK with relaxation time tau; gravity g by evaluating the equilibrium at
 *     u + tau g and T + tau (1 - tau) |g|^2 / 2;
 *   - x is periodic; below row 0 and above row Ly-1 sit walls: three halo rows per wall hold the
 *     rest equilibrium at the wall temperature with the density of the mirror interior row
 *     (LB_WALL_REST), or, as an alternative closure, the equilibrium at the mirror row's
 *     density, opposite velocity and temperature reflected about the wall value (LB_WALL_MIRROR);
 *   - macroscopic output: rho = sum f, rho u = sum f xi, rho (u^2 + 2 T) = sum f xi^2; optionally
 *     the half-step fields that average the pre- and post-collision momentum and energy.
 *
 * Conventions:
 *   - Host fields are row-major [Ly][Lx] float64 (x fastest). Populations exchanged with the
 *     host are plane-major [37][Ly][Lx] float64 in the order of lb_velocity_set().
 *   - Every function returns an lb_status and never aborts; a NULL pointer, a non-positive size
 *     or tau <= 0.5 gives LB_ERR_ARG. After LB_ERR_CUDA, lb_last_error() holds the CUDA message.
 *   - Device memory: either the library allocates it (params.workspace == NULL) or the caller
 *     passes one block of at least lb_workspace_bytes() bytes, 256-byte aligned, that it owns and
 *     keeps alive until lb_free() (e.g. a PyTorch tensor). All work is queued on params.stream
 *     (a cudaStream_t; NULL makes the library create and own a non-blocking stream).
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef LB_D2Q37_H
#define LB_D2Q37_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_NPOP 37

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,       /* invalid argument (NULL, size, tau, workspace too small ...) */
    LB_ERR_ALLOC = 2,     /* device or host allocation failed */
    LB_ERR_CUDA = 3,      /* a CUDA call failed; see lb_last_error() */
    LB_ERR_NONFINITE = 4, /* a site produced a non-finite or non-positive density or temperature */
    LB_ERR_STATE = 5,     /* call not valid in the context's current state */
    LB_ERR_RANGE = 6      /* a population outside the exact-accumulation range: LB_FP32SPLIT, a
                             deviation |f - w| reached 1; LB_FP64, a finite |f| reached 16 (the
                             moment sums are exact 96-bit fixed-point sums with quantum 2^-80) */
} lb_status;

typedef enum {
    LB_FP64 = 0,   /* populations stored and collided in FP64; the moment sums are accumulated
                      exactly in 96-bit fixed point on the integer pipe and correctly rounded to
                      FP64 once (at least as accurate as any FP64 summation order; GB300's FP64
                      pipe binds the step) */
    LB_FP32DEV = 1,  /* populations stored as FP32 deviations f - w; FP32 collide, FP64 moment
                        accumulation and FP64 conservation projection */
    LB_FP32SPLIT = 2 /* same storage and FP32 collide; the moment sums and the projection residual
                        are accumulated by an exact error-free split of each FP32 value into an
                        integer multiple of 2^-22 (summed exactly in 32-bit integers) and a residual
                        below 2^-23 (summed in FP32, error ~1e-10) instead of in FP64, whose rate on
                        GB300 is 1/64 of FP32 */
} lb_precision;

/* Wall closure (the paper defers boundary conditions to its references; Table 1 counts them in
 * the "Global" time). Halo row y = -1 - k mirrors interior row k and y = Ly + k mirrors row
 * Ly - 1 - k (k = 0, 1, 2); the fields of a mirror site are the moments of its current populations
 * (after a step: the post-collision ones, rho, u + g, T). */
typedef enum {
    LB_WALL_REST = 0,  /* f_eq(rho_mirror, 0, T_wall): a rest gas at the wall temperature */
    LB_WALL_MIRROR = 1 /* f_eq(rho_mirror, -u_mirror, 2 T_wall - T_mirror): linear interpolation
                          between a row and its halo row gives u = 0 and T = T_wall half a site
                          outside the last interior row (no-slip isothermal wall). A non-positive
                          reflected temperature sets the LB_ERR_NONFINITE flag and that halo site
                          gets the LB_WALL_REST value instead */
} lb_wall_mode;

typedef struct {
    int Lx, Ly;           /* lattice size; 4 <= Lx, 4 <= Ly, Lx * Ly < 2^31 */
    double tau;           /* BGK relaxation time, > 0.5 */
    double gx, gy;        /* gravity (lattice units, per step) */
    double T_top;         /* wall temperature above row Ly-1 */
    double T_bottom;      /* wall temperature below row 0 */
    int y_periodic;       /* 0: walls at top/bottom; 1: periodic in y (no walls) */
    int precision;        /* lb_precision */
    int wall_mode;        /* lb_wall_mode (ignored when y_periodic) */
    void* stream;         /* cudaStream_t or NULL */
    void* workspace;      /* caller-owned device memory or NULL */
    size_t workspace_bytes;
} lb_params;

/* Human-readable name of a status code (static string). */
const char* lb_status_str(lb_status s);

/* Last CUDA error message recorded by this thread (static per thread; "" if none). */
const char* lb_last_error(void);

/* The library's population order: cx[37], cy[37] lattice vectors, w[37] weights and the thermal
 * scale r (xi = r c). Any argument may be NULL. Pure host call. Order: 0 = rest; 1..18 one
 * vector of each opposite pair; 18 + k is the opposite of k. */
lb_status lb_velocity_set(int* cx, int* cy, double* w, double* r);

/* Device bytes a context with these parameters needs (both population copies, the host-exchange
 * staging area and status words). Pure host call; fields other than Lx, Ly, precision ignored.
 * The two population copies are the double buffer of the Fig. 3 listing (prv/nxt). */
lb_status lb_workspace_bytes(const lb_params* p, size_t* bytes);

/* Create a context: copy the host fields rho, ux, uy, T ([Ly][Lx] float64, caller-owned) to the
 * device, set every population to the equilibrium of its site (Sec. 3 model) and write the wall
 * halos. Synchronous: the host arrays may be reused on return. */
lb_status lb_init(const lb_params* p, const double* rho, const double* ux, const double* uy,
                  const double* T, lb_ctx** out);

/* Seeded Rayleigh-Taylor initial fields (the paper's application, Sec. 3; the recipe is a reading,
 * the paper prints none): walls top and bottom, periodic x; T_top = 2 / (1 + R),
 * T_bottom = 2 R / (1 + R) with R = T_bottom / T_top > 0 the temperature ratio (for an Atwood
 * number A use R = (1 + A) / (1 - A)); interface y_i(x) = Ly/2 + Ly sum_{k=1..8} a_k
 * cos(2 pi k x / Lx + phi_k) with a_1..a_8 uniform draws scaled to sum 1e-3 and phi_1..phi_8
 * uniform in [0, 2 pi), drawn in that order from SplitMix64 seeded with `seed` (u = (next >> 11)
 * 2^-53); T = 1 + (T_bottom - T_top)/2 tanh((y_i - y)/2); u = 0; rho = exp(-g (y - y_i)/T)/T;
 * gravity g = 0.1 T_top / Ly downward. Writes host arrays rho, ux, uy, T ([Ly][Lx] float64,
 * caller-owned) and, if not NULL, *T_top, *T_bottom and *gy (= -g). Pure host call (no GPU);
 * LB_ERR_ARG for non-positive sizes or R. */
lb_status lb_rt_fields(int Lx, int Ly, double R, uint64_t seed, double* rho, double* ux, double* uy,
                       double* T, double* T_top, double* T_bottom, double* gy);

/* lb_init with the fields of lb_rt_fields(p->Lx, p->Ly, R, seed): p's T_top, T_bottom and gy are
 * replaced by the recipe's; every other field of p is used as given. Synchronous. */
lb_status lb_init_rt(const lb_params* p, double R, uint64_t seed, lb_ctx** out);

/* Advance n >= 0 fused time steps: pull propagate (Fig. 3 listing) + collide (Sec. 3) + wall halo
 * write, one kernel per step, CUDA-graph launched. Asynchronous on the context's stream; a
 * non-finite state is reported by the next lb_sync / lb_moments / lb_get_populations. */
lb_status lb_step(lb_ctx* c, int n);

/* Propagate only (no collide): the pull of the Fig. 3 listing, new_i(x, y) =
 * old_i((x - c_ix) mod Lx, y - c_iy), reading wall halos (or wrapping in y when y_periodic);
 * halo rows are carried over unchanged. A pure copy: bit-exact. Asynchronous. */
lb_status lb_propagate(lb_ctx* c);

/* Choose how an LB_FP32SPLIT step reads its populations: use_tma = 1 (available when Lx is a
 * multiple of 4) stages the 37 shifted rows of each 32 x 4-site tile into a two-stage shared-memory
 * ring with TMA bulk-tensor copies, one tile ahead of the computation; 0 (the default) reads them
 * with plain coalesced loads, which measured faster on GB300 (20.0 vs 13.6 G site updates/s at
 * 2304 x 8192): the shared-memory reads replace the global loads one for one, and the per-tile
 * barrier costs more than the load latency it hides. Results are identical bit for bit.
 * LB_ERR_STATE if TMA staging is unavailable. Synchronous. */
lb_status lb_set_staging(lb_ctx* c, int use_tma);

/* Collide only, in place on the current populations (LB_FP64 contexts): the paper's separate
 * collide kernel (Sec. 3; timed on its own in Table 1). Moments, shifted equilibrium and BGK as in
 * lb_step, then the wall halo rows. lb_propagate followed by lb_collide equals one lb_step bit for
 * bit. Asynchronous; LB_ERR_STATE for FP32 contexts or while the learned collide is set. */
lb_status lb_collide(lb_ctx* c);

/* Wait for queued work; returns LB_ERR_NONFINITE (once) if any step since the last check saw a
 * non-finite or non-positive density/temperature, else LB_OK. */
lb_status lb_sync(lb_ctx* c);

/* Macroscopic fields of the current populations into caller-owned host arrays [Ly][Lx] float64
 * (any may be NULL). Synchronous. */
lb_status lb_moments(lb_ctx* c, double* rho, double* ux, double* uy, double* T);

/* Same into caller-owned device arrays of Lx*Ly float64 (any may be NULL). Asynchronous. */
lb_status lb_moments_device(lb_ctx* c, double* rho, double* ux, double* uy, double* T);

/* Half-step ("physical") fields of the current populations, taken as the post-collision state a
 * step leaves: with the shifted-equilibrium forcing a collision adds rho g to the momentum and
 * rho (u.g + |g|^2 / 2) to the kinetic energy sum f xi^2 / 2 and keeps rho and T, so averaging
 * the pre- and post-collision momentum and energy gives u_h = u - g / 2 and
 * T_h = T + |g|^2 / (4 D) (D = 2) from the stored moments (rho, u, T); rho is unchanged. The
 * paper reports no fields (the cited D2Q37 works use these); with g = 0 they equal lb_moments.
 * Caller-owned host arrays [Ly][Lx] float64 (any may be NULL). Synchronous. */
lb_status lb_moments_half_step(lb_ctx* c, double* rho, double* ux, double* uy, double* T);

/* Copy the current interior populations to host f[37][Ly][Lx] float64 (FP32DEV contexts return
 * w + deviation). Synchronous. */
lb_status lb_get_populations(lb_ctx* c, double* f);

/* Replace the current populations by host f[37][Ly][Lx] float64 and rewrite the wall halos from
 * them (checkpoint restore). Synchronous. */
lb_status lb_set_populations(lb_ctx* c, const double* f);

/* Steps taken since lb_init (lb_propagate counts as one). */
lb_status lb_steps_done(const lb_ctx* c, long long* n);

/* Release the context and, if the library allocated it, its device memory. NULL-safe. */
void lb_free(lb_ctx* c);

/* ---- Allocation-free macroscopic fields (the paper has no counterpart to this call) ----
 *
 * For callers that cannot allocate device memory -- code whose device memory belongs to a host
 * framework's own allocator, or that runs where cudaMalloc/cudaFree are not allowed -- this call
 * computes rho, ux, uy, T of one caller-owned population copy without allocating anything: no
 * cudaMalloc, cudaFree or allocating library routine. Its device staging area is a static array of
 * 4 x LB_NOALLOC_MAX_SITES doubles (2 MiB) that every GPU which loads the library holds until the
 * process exits.
 *
 *   p:  Lx, Ly, precision and stream are read (other fields ignored); p->stream is a cudaStream_t
 *       or NULL (legacy default stream). Lx * Ly must not exceed LB_NOALLOC_MAX_SITES, else
 *       LB_ERR_ARG with the reason in lb_last_error().
 *   f:  device pointer to one population copy in the library layout: 37 planes of (Ly + 6) x Lx
 *       elements (3 halo rows each side, x fastest), double for LB_FP64 or FP32 deviations f - w
 *       for LB_FP32DEV and LB_FP32SPLIT. A context's workspace holds copy A at offset 0 and copy B right after it
 *       (offset rounded up to 256 bytes); the current copy is A after an even number of steps.
 *   rho, ux, uy, T: caller-owned host arrays [Ly][Lx] (any may be NULL).
 * Synchronous (returns after the host arrays are written). The first call on a device looks up
 * the static array's device address with that device current; make that first call before any
 * stream capture. All calls share the one array and nothing in it needs clearing (every element
 * read is written first by the same call), so calls whose GPU work overlaps (other host threads,
 * other streams) race on it: serialise them. */
#define LB_NOALLOC_MAX_SITES 65536
lb_status lb_moments_noalloc(const lb_params* p, const void* f, double* rho, double* ux, double* uy,
                             double* T);

#ifdef __cplusplus
}
#endif

#endif /* LB_D2Q37_H */
