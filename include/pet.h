/*
 * pet.h -- C ABI of penalised PET image reconstruction by MM in libnmf.so.
 *
 * The method: Zhou, Lange & Suchard, "Graphics Processing Units and
 * High-Dimensional Optimization", Section 3.2 and Algorithm 2.  Estimate the
 * Poisson emission intensities lambda (p pixels) from coincidence counts y
 * (d lines of flight) with geometry constants E (d x p, e_ij >= 0) by
 * maximising the penalised loglikelihood (Eq. (PET-objpen))
 *
 *     f(lambda) = sum_i [ y_i ln (E lambda)_i - (E lambda)_i ]
 *                 - mu/2 sum_{{j,k} in N} (lambda_j - lambda_k)^2 ,
 *
 * N the pairs of adjacent pixels.  Algorithm 2 scales E to unit column
 * sums, starts from lambda = 1 and repeats, for every pixel j in parallel,
 *
 *     c_j = sum_i y_i e_ij lambda_j / (E lambda)_i
 *     b_j = mu (|N_j| lambda_j + sum_{k in N_j} lambda_k) - 1 ,  a_j = -2 mu |N_j|
 *     lambda_j <- the positive root of a_j x^2 + b_j x + c_j = 0
 *
 * (mu = 0 gives the EM update lambda_j <- c_j).  The library never forms
 * the scaled E: it keeps the column sums sigma_j and works with lambda_j /
 * sigma_j, which gives the same products.
 *
 * Several images are reconstructed together, one per penalty constant
 * mu_k (the paper's table sweeps mu): they share E, y and N, so every pass
 * over E serves all of them.
 *
 * Conventions (as in nmf.h): float32 row-major dense arrays; "device" means
 * memory of the current CUDA device; the caller owns E, y and lambda, and E
 * and y must stay alive and unchanged for the life of a context; errors
 * only through the return code (nmf_status, see nmf.h) and
 * pet_last_error(); one context per stream; deterministic results (no
 * floating-point atomics, fixed reduction orders).
 */
#ifndef PET_H_
#define PET_H_

#include <stdint.h>

#include "nmf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pet_ctx pet_ctx;

/* Create a reconstruction context.
 *   d, p      lines of flight and pixels (d >= 1, p >= 1)
 *   E         device, d x p float32 row-major (ld = p): the raw geometry,
 *             e_ij >= 0 and finite; every column must have a positive sum
 *             (every pixel seen by some line), else NMF_EINVAL
 *   y         device, d float32 counts, >= 0 and finite
 *   nbr_ptr,  host CSR of the neighbourhood system N: the neighbours of
 *   nbr_idx   pixel j are nbr_idx[nbr_ptr[j] .. nbr_ptr[j+1]-1]; nbr_ptr has
 *             p + 1 entries from 0; each index in [0, p), never j itself,
 *             and the system symmetric (k in N_j exactly when j in N_k);
 *             copied at init
 *   nimg      images reconstructed together, 1..8
 *   mu        host, nimg penalty constants, each >= 0 and finite
 *   lambda    device, nimg x p float32 (image k is row k): the intensities,
 *             updated in place; with init_ones != 0 set to 1 (Algorithm 2's
 *             start), else read as the start (>= 0 and finite)
 *   stream    cudaStream_t (NULL: the legacy default stream)
 * Allocates the workspaces (column sums, the scaled intensities, a second
 * intensity buffer, per-line ratios, back-projection partials: about
 * (3 nimg + 2) p + 2 nimg d floats plus nimg * p * segments floats) and
 * checks E, y and lambda on the device (synchronises once).  On failure
 * *out is NULL and nothing is leaked.                                       */
nmf_status pet_init(int64_t d, int64_t p, const float* E, const float* y,
                    const int32_t* nbr_ptr, const int32_t* nbr_idx, int32_t nimg,
                    const double* mu, float* lambda, int32_t init_ones, void* stream,
                    pet_ctx** out);

/* Run `iters` >= 0 iterations of Algorithm 2's loop body on every image.
 * Each iteration is two kernel launches: the forward projection (E lambda)
 * with the per-line ratios y_i / (E lambda)_i (a y_i = 0 line gives 0), and
 * the back projection sum_i e_ij y_i / (E lambda)_i, whose last block per
 * column block forms c_j, b_j and the positive root in float64.  lambda
 * holds the result when the call returns (asynchronous on the stream).    */
nmf_status pet_step(pet_ctx* ctx, int iters);

/* Restart from Algorithm 2's start, lambda = 1 for every image, on the same
 * E, y and neighbourhood system (no allocation, no check).  Asynchronous. */
nmf_status pet_restart(pet_ctx* ctx);

/* f(lambda) of Eq. (PET-objpen) for every image at the current lambda, in
 * float64 (the projections summed in float64, a y_i = 0 line contributing
 * -(E lambda)_i only, each pair of N once), into f_out (host, nimg
 * doubles).  Synchronises.                                                 */
nmf_status pet_objective(pet_ctx* ctx, double* f_out);

/* Algorithm 2 with Section 3's stopping rule: iterate until every image's
 * |f_n - f_{n-1}| / (|f_{n-1}| + 1) < tol or max_iters iterations, testing
 * every `check_every` >= 1 iterations (all images run the same count).
 * *iters_done (host) and f_out (host, nimg doubles; may be NULL) receive the
 * count and the last objectives.  Synchronises.                           */
nmf_status pet_run(pet_ctx* ctx, int max_iters, double tol, int check_every, int* iters_done,
                   double* f_out);

/* CUDA-event timing of the context's kernels by kind (0 = forward
 * projection, 1 = back projection with the update, 2 = objective): enable
 * (on != 0, clearing the totals) or disable, and read the total
 * milliseconds and launch count of one kind (synchronises).              */
nmf_status pet_profile_enable(pet_ctx* ctx, int on);
nmf_status pet_profile_read(pet_ctx* ctx, int kind, double* ms, int64_t* count);

void pet_destroy(pet_ctx* ctx);

/* Reason for the last failure on ctx (ctx == NULL: the last failure of any
 * call on this thread).  Never NULL.                                      */
const char* pet_last_error(const pet_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PET_H_ */
