/*
 * lb_learned.h -- learned collide for the D2Q37 step (GB300 tensor cores).
 *
 * A small MLP (37 -> 128 -> 128 -> 37, GELU) replaces the collide of Sec. 3: it maps the 37
 * pre-collision FP32 deviations of a site to the collision change, which is added to them and
 * projected exactly onto the conserved moments (mass, momentum, energy; gravity included). Its
 * forward and backward products run on tcgen05 tensor cores (BF16 operands, FP32 accumulation)
 * in hand-written kernels; it is trained on the GPU (Adam) on (pre, post) pairs that the plain
 * collide of this library produces. In a lattice step, every 32 x 32-site tile whose result
 * differs from the plain collide by more than bound x max|f_plain| (checked every check_every
 * steps) is replaced by the plain collide and stays on it until the next check.
 *
 * Layouts: sample arrays are [n][37] float32 in the order of lb_velocity_set() (device memory,
 * caller-owned). Parameters are packed W1[128][37] b1[128] W2[128][128] b2[128] W3[37][128]
 * b3[37] (float32); normalisation is [4][37]: mean and standard deviation of the inputs, then of
 * the targets (post - pre).
 * Conventions as in lb_d2q37.h. Learned steps need an LB_FP32SPLIT context with Lx and Ly
 * multiples of 32.
 */
#ifndef LB_LEARNED_H
#define LB_LEARNED_H

#include "lb_d2q37.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_mlp lb_mlp;

#define LB_MLP_NPARAM 26149
#define LB_MLP_TILE 128

/* New network on the current device: weights and biases uniform in +-1/sqrt(fan_in) from a
 * SplitMix64 stream seeded with `seed`, identity normalisation. The library allocates its memory. */
lb_status lb_mlp_create(uint64_t seed, lb_mlp** out);
void lb_mlp_free(lb_mlp* net); /* NULL-safe; waits for the device's queued work first, since the
                                  network may be in use on any stream */

/* Host copies of the FP32 parameters (LB_MLP_NPARAM floats) and normalisation (148 floats). */
lb_status lb_mlp_get_params(const lb_mlp* net, float* params, float* norm);
/* Replace parameters (and normalisation unless norm is NULL); resets the optimizer state. */
lb_status lb_mlp_set_params(lb_mlp* net, const float* params, const float* norm);

/* y[n][37] = network(x[n][37]) on normalised inputs (device arrays, n a multiple of 128). */
lb_status lb_mlp_eval(lb_mlp* net, const float* x, float* y, int n, void* stream);

/* Mean squared error over n samples x 37 outputs of network(x) against normalised targets t, and
 * its gradient with respect to the packed parameters (host array of LB_MLP_NPARAM floats). */
lb_status lb_mlp_loss_grad(lb_mlp* net, const float* x, const float* t, int n, double* loss,
                           float* grad, void* stream);

/* FP32 debug mode of lb_mlp_loss_grad: the same loss and gradient computed in plain FP32 on the
 * CUDA cores (no BF16 rounding; GELU from the CUDA math library's erff), gradients summed over the
 * samples in FP64. For checking against an FP64 reference (agreement ~1e-6 relative); slow, and
 * allocates temporary device memory. Any n > 0. Synchronous. The paper has no counterpart (its
 * method has no learned part). */
lb_status lb_mlp_loss_grad_fp32(lb_mlp* net, const float* x, const float* t, int n, double* loss,
                                float* grad, void* stream);

/* Train on n (pre, post) pairs: sets the normalisation from the data, then `epochs` passes of
 * shuffled mini-batches (batch a multiple of 128) with Adam (beta 0.9 / 0.999, eps 1e-8, rate lr).
 * One cooperative launch per epoch when a batch's CTAs (batch / 128) fit on the GPU at once, else
 * one launch per batch and its Adam step; the same arithmetic either way, and bit-reproducible.
 * The per-epoch launch works on the epoch's samples laid out in batch order in temporary device
 * memory (244 bytes per sample: the BF16 inputs and the FP32 targets, normalised).
 * epoch_loss (host, may be NULL) receives each epoch's mean loss. Synchronous. */
lb_status lb_mlp_train(lb_mlp* net, const float* pre, const float* post, long long n, int epochs,
                       int batch, float lr, uint64_t seed, float* epoch_loss, void* stream);

/* Training pairs from a context's current state (LB_FP32SPLIT): for each of the n site indices
 * (y * Lx + x, device array) pre = the pulled deviations, post = their plain collide. Async. */
lb_status lb_collect_pairs(lb_ctx* c, const int* sites, int n, float* pre, float* post);

/* Context-owned learned collide. lb_collide_train: the context creates (once) its own network
 * (seeded with `seed`), trains it on npairs device pairs pre/post [npairs][37] float32 (as
 * lb_mlp_train: `epochs` passes, batch min(4096, npairs rounded down to a multiple of 128), rate
 * 1e-3, Adam) and switches the context to the learned collide with bound 1e-4 checked every
 * step. Needs an LB_FP32SPLIT context with Lx, Ly multiples of 32 (else LB_ERR_STATE) and
 * npairs >= 128. Synchronous.
 * lb_collide_save: write the context's current learned collide (network parameters,
 * normalisation, bound, check interval) to a file: 8-byte magic "LBMLP37", uint32 version 1,
 * uint32 LB_MLP_NPARAM, uint32 148, int32 check_every, float64 bound, then the float32 parameters
 * and normalisation, all little-endian. LB_ERR_STATE without a learned collide, LB_ERR_ARG if the
 * file cannot be written.
 * lb_collide_load: read such a file into the context's own network and switch the context to it
 * with the stored bound and interval. LB_ERR_ARG for a missing, short or foreign file. */
lb_status lb_collide_train(lb_ctx* c, const float* pre, const float* post, size_t npairs, int epochs,
                           uint64_t seed);
lb_status lb_collide_save(lb_ctx* c, const char* path);
lb_status lb_collide_load(lb_ctx* c, const char* path);

/* Switch the context's collide to the learned one (net must outlive the setting), or back.
 * Setting it allocates the tile decisions, the statistics and a scratch area for the plain result
 * of the tiles in flight (three 32 x 32 tiles per SM, ~150 KB each). */
lb_status lb_set_collide_learned(lb_ctx* c, const lb_mlp* net, double bound, int check_every);
lb_status lb_set_collide_plain(lb_ctx* c);

/* Tiles checked and tiles that fell back since the learned collide was set, and the largest
 * tile residual seen. Synchronous. */
lb_status lb_learned_stats(lb_ctx* c, long long* checked, long long* fallback, double* max_residual);

/* The current decision of every 32 x 32-site tile (the per-tile fallback above): modes[t] = 1 if
 * tile t (row-major over tiles, t = (y / 32) * (Lx / 32) + x / 32) was rewritten with the plain
 * collide at its last check, 0 if it keeps the network's result. n must equal the number of
 * tiles (LB_ERR_ARG otherwise); modes is caller-owned host memory. LB_ERR_STATE without a learned
 * collide. Synchronous. */
lb_status lb_learned_tiles(lb_ctx* c, unsigned char* modes, int n);

#ifdef __cplusplus
}
#endif

#endif /* LB_LEARNED_H */
