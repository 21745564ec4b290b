/*
 * lb_ensemble.h -- batched ensemble of independent D2Q37 lattices of uneven sizes.
 *
 * The paper notes that sites carry no data dependency on each other within propagate or collide,
 * so any schedule is valid (Sec. 3), and parallelises by handing tiles of the lattice to threads
 * (Sec. 1, Sec. 4 listing). The ensemble extends the same idea across many independent lattices:
 * one kernel launch per time step covers a global list of (lattice, tile) work items over every
 * member (one block per item), so lattices of very different sizes share the GPU without one
 * launch per lattice. Step sequences are captured into CUDA graphs; the tile shape is chosen by a
 * timing autotuner.
 *
 * Each member is the same time step as lb_step (include/lb_d2q37.h: pull propagate, collide with
 * gravity, wall halos), with its own size, relaxation time, gravity and wall temperatures.
 * Storage: FP32 deviations (LB_FP32SPLIT, default, or LB_FP32DEV).
 *
 * Conventions as in lb_d2q37.h (status codes, host field layout, caller- or library-owned device
 * memory, stream). An ensemble is not thread-safe.
 */
#ifndef LB_ENSEMBLE_H
#define LB_ENSEMBLE_H

#include "lb_d2q37.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ensemble lb_ensemble;

typedef struct {
    int tile_x, tile_y;  /* sites per work item; 0, 0 = 64 x 4 until lb_ensemble_autotune. A
                            member whose Lx is not a multiple of tile_x gets tiles of the widest
                            power of two >= 32 dividing its Lx (same site count), when there is one */
    int graph_steps;     /* steps per captured CUDA graph; even, 0 = 100 */
    int precision;       /* LB_FP32SPLIT (0 is read as this) or LB_FP32DEV */
    void* stream;        /* cudaStream_t or NULL (library-owned non-blocking stream) */
    void* workspace;     /* caller-owned device memory or NULL */
    size_t workspace_bytes;
    int per_item;        /* 0 (default): one persistent launch per step, a grid of the
                            co-resident blocks (occupancy x SMs) that take the work items in
                            list order from a counter; 1: one block per work item. Same results
                            either way. */
} lb_ensemble_opts;

/* Device bytes needed by n members (members[k].Lx, .Ly used). */
lb_status lb_ensemble_workspace_bytes(int n, const lb_params* members, const lb_ensemble_opts* o,
                                      size_t* bytes);

/* Create an ensemble of n >= 1 members. members[k]: Lx, Ly, tau, gx, gy, T_top, T_bottom,
 * y_periodic of member k (its precision, stream and workspace fields are ignored; wall_mode must
 * be LB_WALL_REST -- the ensemble kernel is built with the rest closure only -- else LB_ERR_ARG;
 * as for lb_init, tau must be finite and > 0.5, the wall temperatures finite and > 0 and the
 * gravity finite, else LB_ERR_ARG).
 * rho[k], ux[k],
 * uy[k], T[k]: host fields [Ly][Lx] float64 of member k. Populations start at equilibrium with
 * wall halos written. Synchronous. */
lb_status lb_ensemble_init(int n, const lb_params* members, const double* const* rho,
                           const double* const* ux, const double* const* uy,
                           const double* const* T, const lb_ensemble_opts* opts,
                           lb_ensemble** out);

/* lb_ensemble_init with member k's fields from lb_rt_fields(members[k].Lx, members[k].Ly, R[k],
 * seeds[k]) (its T_top, T_bottom and gy replaced by the recipe's). Synchronous. */
lb_status lb_ensemble_init_rt(int n, const lb_params* members, const double* R, const uint64_t* seeds,
                              const lb_ensemble_opts* opts, lb_ensemble** out);

/* Advance every member by n steps: one launch per step over all members (graph-replayed). Async. */
lb_status lb_ensemble_step(lb_ensemble* e, int n);

/* Wait; LB_ERR_NONFINITE / LB_ERR_RANGE (once) if any member's step flagged its state. */
lb_status lb_ensemble_sync(lb_ensemble* e);

/* Time every candidate tile shape (tile_x in 32..256, tile_y in 1..16, 128..2048 sites) for
 * `steps` launches each and keep the fastest. Trial launches read the current populations and
 * write the other copy without swapping, so the ensemble's state is unchanged. Synchronous.
 * Writes the chosen shape and its MLUPS (any output may be NULL). */
lb_status lb_ensemble_autotune(lb_ensemble* e, int steps, int* tile_x, int* tile_y, double* mlups);

/* Current tile shape, number of work items and total sites (any output may be NULL). */
lb_status lb_ensemble_info(const lb_ensemble* e, int* tile_x, int* tile_y, int* ntiles,
                           long long* sites);

/* Macroscopic fields of member k into host arrays [Ly][Lx] (any may be NULL). Synchronous. */
lb_status lb_ensemble_moments(lb_ensemble* e, int k, double* rho, double* ux, double* uy,
                              double* T);

/* Populations of member k into host f[37][Ly][Lx] float64 (w + deviation). Synchronous. */
lb_status lb_ensemble_get_populations(lb_ensemble* e, int k, double* f);

/* Release the ensemble (and its device memory if the library allocated it). NULL-safe. */
void lb_ensemble_free(lb_ensemble* e);

#ifdef __cplusplus
}
#endif

#endif /* LB_ENSEMBLE_H */
