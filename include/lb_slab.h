/*
 * lb_slab.h -- one D2Q37 lattice cut into horizontal slabs: the domain decomposition that spreads
 * a lattice over several GPUs (one slab per GPU) or several slabs over one GPU.
 *
 * The paper runs on one KNL socket and names a hybrid MPI + OpenMP code for clusters as future
 * work (Sec. 5). A time step of a site reads only sites at most three rows away (the D2Q37 pull,
 * |c_y| <= 3, Sec. 3), so a lattice cut along y needs, per step and per cut, only the populations
 * that cross the cut: below a slab's row 0, ghost row k (k = 1, 2, 3) is read only for populations
 * with c_y >= k (15, 8 and 3 of them), above its last row only for c_y <= -k. These 26
 * population-rows per cut and direction are all that travels between slabs. x stays periodic in
 * every slab; the global walls stay on the outer sides of the first and last slab.
 *
 * A slab is an lb_ctx (include/lb_d2q37.h) whose lattice is rows [y0, y0 + Ly) of the global
 * lattice; its fields, lb_moments, lb_get_populations etc. cover those rows. After every step the
 * ghost rows of each cut side must be refilled from the neighbour before the next step: in one
 * process with lb_slab_exchange, across processes with lb_slab_pack, a transport of the caller's
 * choice (NCCL send/receive, peer copies) and lb_slab_unpack. Per step, a split launch lets the
 * transport overlap the step: lb_slab_step(c, LB_SLAB_BANDS) writes the rows within three rows of
 * each cut (the only rows a neighbour reads), the caller packs and sends them, and
 * lb_slab_step(c, LB_SLAB_INTERIOR) writes the rest while they travel (interior rows never read a
 * ghost row). Results are the same, bit for bit, as one lattice of all the rows.
 *
 * Packed layout (lb_slab_pack / lb_slab_unpack): LB_SLAB_GHOST_ROWS rows of Lx elements (double
 * for LB_FP64, float deviations f - w for the FP32 forms), for k = 1, 2, 3 outward from the cut and,
 * for each k, the populations in lb_velocity_set() order whose velocity crosses the cut by at least
 * k rows. Buffers are caller-owned device memory.
 */
#ifndef LB_SLAB_H
#define LB_SLAB_H

#include "lb_d2q37.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LB_SLAB_GHOST_ROWS 26

typedef enum { LB_SLAB_WHOLE = 0, LB_SLAB_BANDS = 1, LB_SLAB_INTERIOR = 2 } lb_slab_part;

/* A slab context: as lb_init, for the slab's own rows (p->Ly = its row count, p->T_top/T_bottom
 * and the wall closure apply to the sides that are global walls). cuts: bit 0 = the side below row
 * 0 is cut (a neighbour slab lies below), bit 1 = the side above row Ly - 1 is cut. A cut side gets
 * no wall rows; its ghost rows are undefined until the first exchange or unpack, which must come
 * before the first step. LB_ERR_ARG for cuts outside 0..3, a cut slab with y_periodic or with
 * Ly < 6. Slabs take neither the learned collide nor TMA staging (LB_ERR_STATE). */
lb_status lb_init_slab(const lb_params* p, int cuts, const double* rho, const double* ux, const double* uy,
                       const double* T, lb_ctx** out);

/* One step of a slab, or half of one: LB_SLAB_WHOLE = all rows (then swap), LB_SLAB_BANDS = the
 * rows within three rows of a cut side (no swap yet), LB_SLAB_INTERIOR = the other rows (then swap).
 * BANDS must come before INTERIOR (LB_ERR_STATE otherwise). lb_step(c, 1) on a slab is
 * LB_SLAB_WHOLE; lb_step with n > 1 on a cut slab is LB_ERR_STATE (exchanges must come between
 * steps). Async on the context's stream. */
lb_status lb_slab_step(lb_ctx* c, int part);

/* Pack the rows c sends across its side `side` (0 = below row 0, 1 = above row Ly - 1) from its
 * newest state (after a whole step, or after the BANDS part of a split step) into buf
 * [LB_SLAB_GHOST_ROWS][Lx]. Async on the context's stream. */
lb_status lb_slab_pack(lb_ctx* c, int side, void* buf);

/* Write what the neighbour across cut side `side` packed (its opposite side) into c's ghost rows
 * there, in the newest state. LB_ERR_ARG if that side is not cut. Async on the context's stream. */
lb_status lb_slab_unpack(lb_ctx* c, int side, const void* buf);

/* Exchange across the cut between slab lo (its side above cut) and slab hi (its side below cut),
 * lattice to lattice without a buffer: lo's top rows fill hi's ghost rows below, hi's bottom rows
 * fill lo's ghost rows above. Both must have the same Lx and precision, be at a whole step, and
 * live on one device (or on devices with peer access enabled). The copy runs on lo's stream after
 * the work queued on hi's stream, and hi's stream waits for it. Async. */
lb_status lb_slab_exchange(lb_ctx* lo, lb_ctx* hi);

#ifdef __cplusplus
}
#endif

#endif /* LB_SLAB_H */
