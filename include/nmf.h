/*
 * nmf.h -- C ABI of the GB300 multiplicative-update NMF library (libnmf.so).
 *
 * The method: Zhou, Lange & Suchard, "Graphics Processing Units and
 * High-Dimensional Optimization", Section 3.1.  Given a nonnegative data
 * matrix V (p x n), find nonnegative W (p x r) and H (r x n) minimising the
 * Frobenius objective f = ||V - W H||_F^2 (Eq. (3.1); Algorithm 1 states the
 * problem).  The paper's letters X, V, W are this library's V, W, H.
 *
 * One iteration (Algorithm 1's loop body; Eqs. (3.3) and (3.4)), with eps
 * added to the denominators only:
 *     H <- H .* (W^T V) ./ ((W^T W) H + eps)       right-factor update
 *     W <- W .* (V H^T) ./ (W (H H^T) + eps)       left-factor update
 * Default order: H first, then W (NMF_ORDER_H_FIRST).  NMF_ORDER_W_FIRST
 * is Algorithm 1's own order.  Both are MM block-relaxation steps with the
 * descent property (Section 2, Eq. (3.2)).
 *
 * Conventions for every entry point:
 *   - Matrices are float32, row-major, densely packed (leading dimension =
 *     number of columns): V is p x n, W is p x r, H is r x n.
 *   - Pointers marked "device" must be CUDA device (or managed) memory of
 *     the current device; "host" means ordinary or pinned host memory.
 *   - The caller owns V, W and H.  V must stay alive and unchanged for the
 *     life of a context; W and H are read and updated in place.
 *   - The library owns its workspaces (operand copies of V in the layout and
 *     precision of the chosen arithmetic, factor operand planes, Gram
 *     matrices and their partials, objective partials) and frees them in
 *     nmf_destroy.
 *   - Errors are reported only through the return code (never by exception,
 *     abort or device trap).  nmf_last_error() gives a one-line reason.
 *   - A context is bound to one CUDA stream and is not thread-safe; use one
 *     context per stream.  Asynchronous calls enqueue work on that stream.
 *   - Results are deterministic: no floating-point atomics; every reduction
 *     runs in a fixed order, so repeated runs are bitwise identical.
 */
#ifndef NMF_H_
#define NMF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NMF_OK = 0,
  NMF_EINVAL = 1,        /* bad argument: null pointer, size, rank, eps, enum  */
  NMF_ENOMEM = 2,        /* device or host allocation failed                   */
  NMF_ECUDA = 3,         /* a CUDA runtime/driver call or launch failed        */
  NMF_ETIMEOUT = 4,      /* a bounded device-side wait ran out (no hang)       */
  NMF_ENONFINITE = 5,    /* V holds a negative, NaN or infinite entry          */
  NMF_EUNSUPPORTED = 6   /* valid request this build or device cannot serve    */
} nmf_status;

/* Arithmetic of the two V-streaming products W^T V and V H^T.  All forms
 * accumulate in float32; the element-wise update, the Gram matrices and the
 * objective are float32/float64 in every form.
 *   NMF_FP32   : float32 FMA on the SM cores (the plain reference form)
 *   NMF_TF32   : tcgen05 tensor cores, TF32 operands
 *   NMF_BF16X3 : tcgen05, each operand split x = hi + lo (both bf16);
 *                products hi*hi + hi*lo + lo*hi
 *   NMF_BF16   : tcgen05, operands rounded to bf16 (half the bytes of V)    */
typedef enum {
  NMF_FP32 = 0,
  NMF_TF32 = 1,
  NMF_BF16X3 = 2,
  NMF_BF16 = 3
} nmf_precision;

typedef enum {
  NMF_ORDER_H_FIRST = 0, /* H then W                                        */
  NMF_ORDER_W_FIRST = 1  /* W then H: Algorithm 1's order                   */
} nmf_order;

/* The model the factors are fitted under (Section 3.1).
 *   NMF_MODEL_GAUSSIAN : minimise ||V - W H||_F^2 by Algorithm 1 (the
 *                        alternating updates above); every precision.
 *   NMF_MODEL_POISSON  : maximise the Poisson loglikelihood
 *                        L = sum_ij [v_ij ln (WH)_ij - (WH)_ij] by the
 *                        paper's simultaneous square-root MM update
 *                          W_ik <- W_ik sqrt((sum_j v_ij H_kj / b_ij) / sum_j H_kj)
 *                          H_kj <- H_kj sqrt((sum_i v_ij W_ik / b_ij) / sum_i W_ik)
 *                        with b = W H from the same iteration (eps guards
 *                        the divisions; a term with v_ij = 0 is zero).
 *                        r <= 64, NMF_FP32 (float32 FMA passes) or
 *                        NMF_BF16X3 (the products W H, q H^T and W^T q of
 *                        both passes on the tensor cores, split hi + lo with
 *                        float32 accumulation; nmf_init makes a tile-blocked
 *                        float32 copy of V, about p n 4 bytes), else
 *                        NMF_EUNSUPPORTED.  NMF_FP32 sums the denominators
 *                        and the numerators' segment partials in float64,
 *                        NMF_BF16X3 in compensated float32; the final
 *                        ratio, square root and product are float32.
 *                        `order` is ignored; nmf_objective returns L;
 *                        nmf_half_step and nmf_read_gram are not served.  */
typedef enum {
  NMF_MODEL_GAUSSIAN = 0,
  NMF_MODEL_POISSON = 1
} nmf_model;

typedef struct {
  int64_t p;             /* rows of V and W                                 */
  int64_t n;             /* columns of V and H                              */
  int32_t r;             /* rank: 1 <= r <= 128, r <= min(p, n)             */
  float eps;             /* >= 0, added to every update denominator         */
  nmf_precision prec;
  nmf_order order;
  uint64_t seed;         /* used when init_from_seed != 0                   */
  int32_t init_from_seed;/* 1: nmf_init overwrites W, H with iid uniform(0,1)
                            draws (Algorithm 1's start; counter-based
                            SplitMix64, W on stream 1, H on stream 2)        */
  int32_t validate;      /* 1: nmf_init rejects V with a negative or
                            non-finite entry (NMF_ENONFINITE)               */
  int32_t split_k;       /* 0: automatic; otherwise the number of K-splits
                            per output tile of each product (tuning knob)   */
  int32_t model;         /* nmf_model (0: Gaussian, the default)           */
} nmf_config;

typedef struct nmf_ctx nmf_ctx;
typedef struct nmf_batch nmf_batch;

/* Fill *cfg with defaults for a p x n problem of rank r: eps = 1e-10,
 * NMF_FP32, NMF_ORDER_H_FIRST, seed 0, no seeded init, no validation,
 * automatic split.  Returns NMF_EINVAL if cfg is null.                      */
nmf_status nmf_config_default(nmf_config* cfg, int64_t p, int64_t n, int32_t r);

/* Create a context for V (device, p x n), W (device, p x r), H (device,
 * r x n) on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Allocates the workspaces, builds V's operand copies for the chosen
 * precision (one pass over V), optionally seeds W and H, and forms the Gram
 * matrices W^T W and H H^T of the starting factors.  Asynchronous on the
 * stream except for allocation.  On failure *out is NULL and nothing is
 * leaked.                                                                    */
nmf_status nmf_init(const nmf_config* cfg, const float* V, float* W, float* H,
                    void* stream, nmf_ctx** out);

/* Run `iters` >= 0 MM iterations (Algorithm 1's loop body, in cfg.order;
 * for NMF_MODEL_POISSON the simultaneous square-root update), updating W
 * and H in place.  Asynchronous on the context's stream.                   */
nmf_status nmf_step(nmf_ctx* ctx, int iters);

/* One block update only: which = 0 updates H (Eq. (3.4) in the paper's
 * letters), which = 1 updates W (Eq. (3.3)).  nmf_step(ctx, 1) equals the
 * two half steps in cfg.order.  Asynchronous.  NMF_EUNSUPPORTED for the
 * Poisson model (its update has no half steps).                            */
nmf_status nmf_half_step(nmf_ctx* ctx, int which);

/* f = ||V - W H||_F^2 (Eq. (3.1)) at the current W, H, as a direct residual
 * summed in float64 in a fixed order; for NMF_MODEL_POISSON the
 * loglikelihood L = sum_ij [v_ij ln (WH)_ij - (WH)_ij] (0 ln 0 = 0) instead,
 * (WH)_ij by a compensated float32 dot product, the rest in float64.
 * *f_out is host memory.  Synchronises the stream.                          */
nmf_status nmf_objective(nmf_ctx* ctx, double* f_out);

/* Algorithm 1 with Section 3's stopping rule (f is the model's objective:
 * the Frobenius residual, or L for the Poisson model): iterate until
 * |f_k - f_{k-1}| / (|f_{k-1}| + 1) < tol or max_iters iterations, testing
 * the objective every `check_every` >= 1 iterations.  *iters_done and *f_out
 * (host) receive the count and the last objective.  Synchronises.          */
nmf_status nmf_run(nmf_ctx* ctx, int max_iters, double tol, int check_every,
                   int* iters_done, double* f_out);

/* nmf_run with the loop on the device: one CUDA graph whose while-node runs
 * `check_every` iterations, the objective and the stopping test per round;
 * the test kernel decides whether another round runs, so the host waits
 * once for the whole run instead of once per test.  Same arguments, same
 * iterates, *iters_done and *f_out as nmf_run (the tests take the same
 * float64 operations).  The graph is built on the first call for a given
 * check_every and kept with the context (captured on a private stream of
 * the context; the launch and the final copies use the context's stream).
 * Synchronises.  NMF_ECUDA if the driver cannot build the graph.           */
nmf_status nmf_converge(nmf_ctx* ctx, int max_iters, double tol, int check_every,
                        int* iters_done, double* f_out);

/* nmf_converge with every iteration in ONE persistent launch, for problems
 * that are launch-bound rather than HBM-bound (the faces matrix of the
 * paper's Table 2, 361 x 2429): Algorithm 1 (Eqs. (3.3)-(3.4)) in cfg.order
 * and Section 3's stopping rule on Eq. (3.1)'s objective, with the same
 * arguments, rounds of `check_every` iterations, remainder and results
 * (*iters_done, *f_out) as nmf_converge.  One cooperative launch of one block
 * per SM: each block keeps a column slice of V and a row slice of V in shared
 * memory for the whole run, updates its columns of H and its rows of W
 * (reading the whole other factor each half step), and the blocks meet at a
 * grid-wide barrier after every half step; the objective of a round is a
 * float64 sum of per-block partials in block order, so every block takes the
 * same stopping decision.  Arithmetic: float32 products with fixed reduction
 * trees, each Gram the float32 sum in block order of the blocks' partial
 * Grams of their own slices, IEEE division, compensated float32 residuals
 * summed in float64; the iterates agree with nmf_converge's to float32
 * rounding, not bitwise.  Needs NMF_MODEL_GAUSSIAN and NMF_FP32 (else
 * NMF_EUNSUPPORTED), r <= 16, and V's two slices plus the larger factor
 * within one block's shared memory (else NMF_EUNSUPPORTED; 361 x 2429 fits
 * up to r = 12).  A workspace of (p + n) * ceil4(r) + sms * r * (r + 1)
 * floats is allocated on the first call.  A grid-wide barrier that waits
 * longer than about a second makes the call return NMF_ETIMEOUT.
 * Afterwards the other entry points continue from the new W and H.
 * Synchronises.                                                             */
nmf_status nmf_converge_resident(nmf_ctx* ctx, int max_iters, double tol, int check_every,
                                 int* iters_done, double* f_out);

/* Quasi-Newton acceleration of the MM map (the scheme the paper names in
 * Section 4; Zhou, Alexander & Lange).  Each iteration evaluates
 * x1 = F(x_n) and x2 = F(x1) by two MM iterations (F = nmf_step(ctx, 1); x
 * stacks W and H), keeps the secant pairs (x1 - x_n, x2 - x1) of the last q
 * iterations as the columns of U and V (float32, on the device), forms
 * U^T U and U^T V from float64 inner products in a fixed order, and takes
 *     x_{n+1} = x1 + V (U^T U - U^T V)^-1 U^T (x1 - x_n)
 * when all its entries are nonnegative and its objective is no worse than
 * x2's, and x2 otherwise (also when the q x q system is singular), so an
 * iteration never ends worse than two MM iterations.  Runs max_iters
 * iterations or until Section 3's rule holds for tol on the model's
 * objective (the Frobenius objective; L for the Poisson model, maximised).
 * *iters_done, *f_out (the last objective) and *qn_taken (quasi-Newton
 * points taken) are host memory; each may be NULL.  The workspace,
 * (3 + 2q) (p + n) r floats, is allocated by the first call and sized for
 * its q; later calls take any q up to that (NMF_EINVAL above it).
 * 1 <= q <= 32.  Synchronises (three times per iteration).                  */
nmf_status nmf_qn_run(nmf_ctx* ctx, int q, int max_iters, double tol, int* iters_done,
                      double* f_out, int* qn_taken);

/* Restart from Algorithm 1's seeded start on the same V (multiple random
 * starts): rebuild V's operand copies (one pass over V), draw W and H iid
 * uniform(0,1) from `seed` exactly as init_from_seed does, and re-form the
 * Gram matrices.  No allocation.  Asynchronous.                            */
nmf_status nmf_restart(nmf_ctx* ctx, uint64_t seed);

/* Copy the current Gram matrix (which = 0: W^T W, which = 1: H H^T) into
 * host memory `out` (r*r doubles, row-major).  Synchronises.
 * NMF_EUNSUPPORTED for the Poisson model (it forms no Gram matrices).     */
nmf_status nmf_read_gram(nmf_ctx* ctx, int which, double* out);

/* One-call solve: V, W, H may each be host or device pointers (detected per
 * pointer).  Host inputs are copied in, `iters` iterations run, W and H are
 * copied back to host outputs and, if f_out is not NULL, the final objective
 * is written there (host).  Synchronises; uses `stream` for all work.      */
nmf_status nmf_solve(const nmf_config* cfg, const float* V, float* W, float* H,
                     int iters, double* f_out, void* stream);

void nmf_destroy(nmf_ctx* ctx);

/* ---- Batched form: many independent problems in one grouped launch -------
 * Instance b has its own cfgs[b] (p, n, r, eps; precision must be the same
 * for all, order is H first), V[b] (device), W[b], H[b] (device, updated in
 * place).  Every iteration of every instance runs inside one persistent
 * grouped kernel per iteration, replayed from a CUDA graph.  The pointer
 * arrays are host memory and are copied at init.                            */
nmf_status nmf_batched_init(int count, const nmf_config* cfgs,
                            const float* const* V, float* const* W,
                            float* const* H, void* stream, nmf_batch** out);
nmf_status nmf_batched_step(nmf_batch* b, int iters);
/* f_out: host array of `count` doubles.  Synchronises.  NMF_ETIMEOUT if a
 * bounded device wait of an earlier step ran out (the error is then
 * cleared).                                                                */
nmf_status nmf_batched_objective(nmf_batch* b, double* f_out);
/* The schedule the autotuner chose at nmf_batched_init ("policy/grid":
 * lpt, glpt or rr over `grid` persistent blocks).  No counterpart in the
 * paper.  The environment variable NMF_BATCHED_SCHEDULE, read at init,
 * forces one candidate by that name (NMF_EINVAL if it names none), and
 * NMF_TUNE_CACHE (a file path) caches the choice per batch signature.
 * Never NULL; "" for b == NULL.                                            */
const char* nmf_batched_schedule(const nmf_batch* b);
/* Failure-detection test hook (no counterpart in the paper): the next
 * nmf_batched_step iteration is launched outside its graph with every
 * block's first pipeline stage armed for 16 bytes more than its copies
 * bring, so that every bounded wait on it runs out (about 3 s per half
 * step) without a fault: the blocks stop before updating any factor, the
 * next nmf_batched_objective reports NMF_ETIMEOUT, and later steps run
 * normally.  NMF_EINVAL for b == NULL.                                      */
nmf_status nmf_batched_test_expire_next_wait(nmf_batch* b);
void nmf_batched_destroy(nmf_batch* b);

/* ---- Gram matrix without allocation --------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc -- programs whose device memory belongs to
 * another allocator (a framework's caching allocator or a fixed arena), and
 * latency-critical code where cudaMalloc may synchronise the device.
 * Computes, on `stream`, the r x r Gram matrix of a factor F with the same
 * kernels nmf_init uses, writing float64 G_out (device, r*r, row-major):
 *   layout 0: F is M x r row-major (ldf must equal r), G = F^T F   (like W)
 *   layout 1: F is r x M with row pitch ldf >= M,      G = F F^T   (like H)
 * It allocates nothing: its scratch is a static 8 MiB device array inside
 * the library, held by every GPU that loads the library until exit.  The
 * first call on a device (with that device current) looks the array's
 * device address up; under CUDA's lazy module loading that lookup may load
 * the library's device code on the device, which can allocate and
 * synchronise inside the driver, so make the first call per device at
 * start-up, off any latency-critical path and before any stream capture.
 * A failed lookup (NMF_ECUDA) is not remembered: the next call retries.
 * Sizes needing more than 2^21 floats of scratch (ceil(M/128)*r*r + r*r)
 * are rejected with NMF_EINVAL and a message in nmf_last_error(NULL).  All
 * calls share the scratch: calls that overlap on the GPU race and must not
 * be issued concurrently.  Asynchronous.                                    */
nmf_status nmf_gram_noalloc(const float* F, int32_t layout, int64_t M, int64_t ldf, int32_t r,
                            double* G_out, void* stream);

/* ---- Failure-detection test hook ------------------------------------------
 * No counterpart in the paper.  Every device-side wait of the library is
 * bounded (about 1.5 s); when one expires the kernel records NMF_ETIMEOUT in
 * the context's error word, skips the rest of its work (the factors keep
 * their previous values) and returns, and the next synchronising call
 * (nmf_objective, nmf_run, nmf_read_gram, nmf_solve) reports NMF_ETIMEOUT.
 * This hook makes that happen on purpose for the next half step: it gives
 * the launch's grid-wide publication waits a target the device counter
 * never reaches, so that every block's wait runs out (about 3 s in all).
 * For the NMF_BF16X3 Poisson model it acts on the next iteration run by
 * nmf_step: the first pass's first V stage waits for 16 bytes more than its
 * copies bring, every block gives up (a few seconds), and the update leaves
 * W and H unchanged.  The context stays usable afterwards.  NMF_EINVAL for
 * ctx == NULL; NMF_EUNSUPPORTED for the NMF_FP32 Poisson model (its kernels
 * have no waits).                                                          */
nmf_status nmf_test_expire_next_wait(nmf_ctx* ctx);

/* ---- Self-check of the update's division ----------------------------------
 * No counterpart in the paper.  The update new = (old * num) / (den + eps)
 * (Eqs. (3.3)-(3.4)) divides with IEEE round-to-nearest; the kernels do so by
 * Markstein's quotient correction where its conditions hold and by the IEEE
 * division elsewhere.  This runs `count` divisions on the current device
 * (the first 64 * 2^23 sweep every significand of the divisor against 64
 * dividends; the rest are random operand pairs drawn from `seed`) and
 * reports how many differ bit for bit from the IEEE division
 * (*mismatches) and how many took the quick form (*quick).  Synchronous;
 * allocates 16 bytes.  NMF_EINVAL for count < 0 or null outputs.           */
nmf_status nmf_selfcheck_div(int64_t count, uint64_t seed, uint64_t* mismatches,
                             uint64_t* quick);

/* ---- Instrumentation ---------------------------------------------------
 * Number of kernels this library has launched in this process (all
 * contexts), for launch accounting.                                         */
uint64_t nmf_kernel_launches(void);
/* Enable (on != 0) or disable CUDA-event timing of the context's kernels by
 * kind; enabling clears the totals.  Kinds: 0 = the V-streaming products
 * with their fused epilogues, 1 = Gram reductions, 2 = objective,
 * 3 = operand copies / seeding / starting Grams.                           */
nmf_status nmf_profile_enable(nmf_ctx* ctx, int on);
/* Total milliseconds and launch count recorded for `kind` since enabling.
 * Synchronises the stream.                                                 */
nmf_status nmf_profile_read(nmf_ctx* ctx, int kind, double* ms, int64_t* count);

const char* nmf_status_str(nmf_status s);
/* Reason for the last failure on ctx (or, with ctx == NULL, the last failure
 * of any call on this thread).  Never NULL.                                */
const char* nmf_last_error(const nmf_ctx* ctx);
/* Library version string.                                                  */
const char* nmf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NMF_H_ */
