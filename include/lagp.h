/*
 * lagp.h -- C ABI of the GB300 (sm_103a) library for local approximate
 * Gaussian process regression with ALC local design search
 * (Gramacy, Niemi & Weiss, "Massively parallel approximate Gaussian process
 * regression", arXiv:1310.5182).
 *
 * Notation follows the paper: X is the N x p design, Y the N responses, Xref
 * the M reference (predictive) locations x; every location gets its own local
 * design X_n(x) grown greedily from the n0 nearest neighbours to n rows, the
 * search restricted to the N' nearest neighbours of x (Sec. 3.1).  The
 * correlation is the isotropic Gaussian K(x,x') = exp(-||x - x'||^2 / d)
 * (Sec. 2.1) with lengthscale d and nugget g: design matrices carry g on the
 * diagonal, cross covariances carry none, and a candidate's self covariance
 * is 1 + g.
 *
 * Conventions for every entry point below:
 *  - Array arguments are DEVICE pointers owned by the caller (for example the
 *    storage of PyTorch CUDA tensors), row-major and densely packed, except
 *    in lagp_agp, whose arrays are HOST pointers.  The library never frees or
 *    retains caller memory.
 *  - Work is enqueued on the context's stream and is asynchronous with respect
 *    to the host, except lagp_agp, which returns after its results are in host
 *    memory.  The context owns a device workspace that grows on demand;
 *    growing it synchronises the device.
 *  - The return value reports argument and CUDA errors: LAGP_EINVAL for an
 *    inconsistent size or parameter (nothing is launched), LAGP_ECUDA for a
 *    failed CUDA call, LAGP_ENOMEM when the workspace cannot grow.  The text
 *    of the last error is available from lagp_last_error().
 *  - Numerical failures of single locations do not fail the call: the call
 *    returns LAGP_OK, status[m] receives LAGP_ENOTPD (a local covariance
 *    matrix that is not positive definite in floating point) and that
 *    location's floating outputs are NaN (its index outputs -1).
 *  - M = 0 is a no-op that returns LAGP_OK; M must be below 2^30 (the
 *    persistent kernels count locations with a 32-bit atomic counter).
 *  - A context must not be used from two host threads at once.
 */
#ifndef LAGP_H
#define LAGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LAGP_OK = 0,
    LAGP_EINVAL = 1,   /* invalid argument: nothing was launched */
    LAGP_ENOTPD = 2,   /* per-location: local matrix not positive definite */
    LAGP_ECUDA = 3,    /* a CUDA runtime call failed */
    LAGP_ETIMEOUT = 4, /* per-location: a bounded device-side wait gave up */
    LAGP_ENOMEM = 5    /* workspace could not be allocated, or a bounded
                          candidate buffer overflowed (lagp_knn) */
} lagp_status;

/* element type of X, Y and Xref */
typedef enum { LAGP_F64 = 0, LAGP_F32 = 1 } lagp_dtype;

/* arithmetic of the ALC search (lagp_alc_select)
 *  LAGP_PREC_F64     the plain form: every candidate's criterion evaluated
 *                    with Eq. (dxy) in FP64, O(j^2) per candidate per step.
 *  LAGP_PREC_F32BULK candidates screened in FP32 through the Schur-complement
 *                    form of the same criterion (O(j) per candidate per
 *                    step); every contender (FP32 score within the
 *                    contender margin of the FP32 maximum) is re-scored with
 *                    Eq. (dxy) in double-float arithmetic (FP32 hi/lo pairs,
 *                    ~48 significant bits) in the Cholesky basis of K_j,
 *                    whose inverse factor grows by the partitioned inverse
 *                    of the bordered factor; the argmax is taken on those
 *                    values.  No FP64 instruction is used (this GPU runs
 *                    FP64 at 1/64 of the FP32 rate); the double-float
 *                    Cholesky basis keeps the decisions' and predictions'
 *                    errors at ~sqrt(cond(K_j)) 2^-48.  A location where
 *                    the FP32 screen breaks down (near-singular local
 *                    matrices: no contender with m_j^{-1} > 0 in
 *                    double-float) is redone in the same call by the
 *                    LAGP_PREC_F64SCHUR form; status LAGP_ENOTPD only if
 *                    that fails too.
 *  LAGP_PREC_F64SCHUR the same Schur-complement form with the candidate
 *                    state in FP64 (the incremental O(j) form of the
 *                    criterion, exact to FP64 rounding); the contenders
 *                    within a margin of 1e-5 of the best score are
 *                    re-scored with Eq. (dxy) as above.
 *  LAGP_PREC_F32BULK_F64 the FP32 screen of LAGP_PREC_F32BULK with its
 *                    contenders re-scored by Eq. (dxy) in FP64 against
 *                    K_j^{-1}, grown by the FP64 partitioned inverse (the
 *                    FP32-bulk form with an FP64 update); faster than
 *                    LAGP_PREC_F32BULK where many contenders a step are
 *                    re-scored, its decisions carrying the K^{-1} basis's
 *                    ~cond(K_j) 2^-53 error.  Breakdowns are redone by
 *                    LAGP_PREC_F64SCHUR like LAGP_PREC_F32BULK's. */
typedef enum {
    LAGP_PREC_F64 = 0,
    LAGP_PREC_F32BULK = 1,
    LAGP_PREC_F64SCHUR = 2,
    LAGP_PREC_F32BULK_F64 = 3
} lagp_precision;

typedef struct lagp_ctx lagp_ctx;

/* Tunables of the persistent kernels.  Zero fields mean "choose
 * automatically" (a per-shape choice made by the built-in tuner). */
typedef struct {
    int32_t ctas_per_sm;    /* resident CTAs per SM of the ALC kernels */
    int32_t block_threads;  /* threads per CTA of the ALC kernels */
    int32_t rescore_max;    /* F32BULK: contenders re-scored together in one
                               batch, 1..32, used up to 16; 0 = automatic (the
                               autotuner's choice for the shape, else 8).
                               More contenders take further batches, none is
                               dropped.  (F64SCHUR and F32BULK_F64: the
                               contenders re-scored, 0 = 8; beyond it those
                               with the lowest FP32 scores are not re-scored,
                               a bound on the work those forms accept.) */
    double rescore_rel;     /* F32BULK: cap of the contender margin (default
                               0.5; a higher cap trades speed for fewer
                               decisions missed where the FP32 state is poor).
                               A candidate is a contender when its FP32
                               score is within the margin of the FP32 maximum;
                               the margin is 8x the largest relative
                               FP32-vs-double-float score error observed on
                               earlier re-scores (decaying 0.75x per step), at
                               least 0.02 and at most rescore_rel */
    int32_t knn_path;       /* kNN collection pass (lagp_knn): 0 = automatic
                               (tcgen05 tensor cores, FP16 split products,
                               for p <= 20; CUDA cores otherwise), 1 = CUDA
                               cores (FP32) always */
} lagp_tuning;

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle.  Returns LAGP_EINVAL for a bad device, LAGP_ECUDA on failure. */
lagp_status lagp_create(lagp_ctx **ctx, int device, void *cuda_stream);

/* Release the context and its workspace (synchronises its stream).  NULL is
 * accepted. */
lagp_status lagp_destroy(lagp_ctx *ctx);

/* Switch the stream later calls enqueue on. */
lagp_status lagp_set_stream(lagp_ctx *ctx, void *cuda_stream);

/* Text of the last error on this context ("" if none); valid until the next
 * call on the context. */
const char *lagp_last_error(const lagp_ctx *ctx);

/* Name of a status code. */
const char *lagp_status_string(lagp_status s);

lagp_status lagp_get_tuning(const lagp_ctx *ctx, lagp_tuning *out);
lagp_status lagp_set_tuning(lagp_ctx *ctx, const lagp_tuning *in);

/* Number of kernels this context has launched since creation (all entry
 * points), for launch accounting. */
int64_t lagp_launch_count(const lagp_ctx *ctx);

/* Work counters of the FP32-bulk ALC search (not part of the paper's method;
 * they measure the double-float re-score that the FP32 screen leaves, Eq. dxy):
 *   out[0]  locations searched
 *   out[1]  sum over steps of the contenders re-scored (n_c)
 *   out[2]  sum over steps of n_c * j   (j = design size at the step)
 *   out[3]  sum over steps of n_c * j^2
 * summed over every F32BULK search launched on this context since it was
 * created or last read.  Reading synchronises the context's stream and
 * resets the counters to zero. */
lagp_status lagp_alc_work(lagp_ctx *ctx, uint64_t out[4]);

/* Work counters of the Newton MLE of d (lagp_mle_step; not part of the
 * paper's method, they give its FP64 operation count, Eq. gpk):
 *   out[0]  sum over likelihood evaluations of n^3 (each factorises K_n:
 *           ~n^3/3 flops)
 *   out[1]  sum over derivative evaluations of n^3 (L^{-1}, K^{-1} and
 *           L^{-1} K' L^{-T}: ~2 n^3 flops)
 * summed over every lagp_mle_step launched on this context since it was
 * created or last read.  Reading synchronises the context's stream and
 * resets the counters to zero. */
lagp_status lagp_mle_work(lagp_ctx *ctx, uint64_t out[2]);

/* Diagnostic: the library's own FP64 exponential (Tang's table-driven
 * method, used for the kernel values of the FP64 kernels) and the CUDA
 * library's exp, both evaluated at the n device values a[] into the device
 * arrays out_tang[] and out_lib[] (enqueued on the context's stream). */
lagp_status lagp_exp64_check(lagp_ctx *ctx, const double *a, int64_t n, double *out_tang,
                             double *out_lib);

/* Diagnostic of the double-float arithmetic of the FP32-bulk search: for
 * each of the n device doubles a[i], split[2i] and split[2i+1] (device
 * floats) receive its double-float split hi + lo (hi rounded to nearest, the
 * split done on the integer pipe), and ex[2i], ex[2i+1] the double-float
 * exponential of hi + lo (Tang's method in double-float arithmetic).
 * Enqueued on the context's stream. */
lagp_status lagp_df_check(lagp_ctx *ctx, const double *a, int64_t n, float *split, float *ex);

/* Autotuner.  Times the ALC search (a2..a6, or a2..a7 when Y is not NULL) on
 * a sample of the given problem (its first min(M, 16 x SMs) locations) for
 * every admissible number of resident CTAs per SM of the persistent kernel
 * and, for F32BULK with tuning.rescore_max == 0, for double-float re-score
 * batches of 16, 8 and 4 contenders, and records the fastest for problems of
 * this shape (precision, N' capacity, n_max, p, with or without prediction)
 * on this context; later calls with tuning.ctas_per_sm == 0 (and
 * rescore_max == 0) use it.  Results do not depend on either choice.
 * Synchronises the stream.  Arguments as lagp_alc_predict;
 * *best_ctas_per_sm and *best_rescore_max (either may be NULL) receive the
 * choices. */
lagp_status lagp_autotune(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                          const void *Xref, int64_t M, const int32_t *idx, const int32_t *Nprime,
                          int32_t Nprime_max, int32_t n0, const int32_t *n, int32_t n_max,
                          const double *d, double g, lagp_precision prec, const void *Y,
                          int32_t *best_ctas_per_sm, int32_t *best_rescore_max);

/* ---------------------------------------------------------------- a1: kNN
 * Exact N'-nearest-neighbour candidate sets (Sec. 3.1: the ALC search is
 * restricted to the N' nearest neighbours of x; Fig. 1 step 2(a) takes the
 * first n0 of them as the initial design).
 *   X       N x p design (dtype)            Xref  M x p locations (dtype)
 *   Nprime  M per-location N' values, or NULL (all = Nprime_max)
 *   idx     M x Nprime_max int32 output: design rows sorted by ascending
 *           (d2, row), where d2 = sum_i (x_i - X_{r,i})^2 is accumulated in
 *           FP64 in coordinate order without fused multiply-add; entries past
 *           Nprime[m] are -1.  The result is bit-exact and deterministic.
 *   status  M int32 output or NULL: LAGP_OK; LAGP_EINVAL (Nprime[m] outside
 *           [1, Nprime_max], or non-finite distances); LAGP_ENOMEM (more
 *           design rows than the candidate capacity, at least
 *           min(2 Nprime_max + 1024, 8192), lie within FP32 screening
 *           resolution of the N'-th distance, i.e. massively duplicated
 *           rows).  A failed location's idx row is -1.
 * Requires 1 <= Nprime_max <= min(N, 4096), N < 2^31 and 1 <= p <= 64. */
lagp_status lagp_knn(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                     const void *Xref, int64_t M, const int32_t *Nprime, int32_t Nprime_max,
                     int32_t *idx, int32_t *status);

/* Diagnostic of the kNN screen's collection pass on the tensor cores (used
 * by lagp_knn for p <= 20 unless tuning.knn_path = 1): out (device, M x N
 * floats) receives, for every location m and design row r, the value
 *   s = |y_m|^2 + |y_r|^2 - 2 y_m . y_r
 * that the pass computes with FP16 split products and FP32 accumulation,
 * where y = fl32(x - c) are the coordinates centred at the midrange c of
 * each coordinate over X and Xref.  It differs from |y_m - y_r|^2 by at most
 * the pass's error bound.  Requires 1 <= p <= 20; other arguments as lagp_knn. */
lagp_status lagp_knn_tc_dist(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                             const void *Xref, int64_t M, float *out);

/* Diagnostic of the last lagp_knn call on this context: *n_retry receives
 * the number of locations that the exact (CUDA-core, direct-form) retry of
 * the screen recomputed, *tc_failed 1 if the tensor-core pass gave up on a
 * bounded wait (its locations then went to the retry).  Synchronises. */
lagp_status lagp_knn_stats(lagp_ctx *ctx, int64_t *n_retry, int32_t *tc_failed);

/* Test hook for failure detection: the next tensor-core pass of lagp_knn on
 * this context stops feeding its pipeline after the first design block, so
 * that its bounded waits (2 s each) run out.  The pass then reports the
 * failure (lagp_knn_stats: tc_failed = 1) and the exact CUDA-core retry
 * recomputes all its locations: the call's results are unchanged, only
 * slower.  No GPU fault is involved. */
lagp_status lagp_knn_tc_stall(lagp_ctx *ctx);

/* ---------------------------------------------- a2..a6: greedy ALC search
 * Local designs by the greedy ALC search of Fig. 1 step 2: the first n0
 * candidates of idx form X_{n0}(x); for j = n0..n[m]-1 the candidate that
 * maximises the reduction in variance v_j(x) - v_{j+1}(x) of Eq. (dxy)
 * (with g_j, m_j of Eq. (piedef)) joins the design and K_j^{-1} grows by the
 * partitioned inverse (Sec. 2.2).  Exact ties go to the lower design row.
 *   X, Xref     as lagp_knn;  idx, Nprime, Nprime_max  as produced by lagp_knn
 *               (Nprime_max <= 4096); a location whose idx row holds a row
 *               outside [0, N), or whose n[m] / Nprime[m] are inconsistent,
 *               gets status LAGP_EINVAL
 *   n0          initial nearest-neighbour design size, >= 1
 *   n           M final design sizes (n0 <= n[m] <= Nprime[m]), or NULL
 *               (all = n_max)
 *   d           M lengthscales (> 0);  g  nugget (>= 0)
 *   prec        LAGP_PREC_F64, LAGP_PREC_F32BULK, LAGP_PREC_F64SCHUR or LAGP_PREC_F32BULK_F64
 *               (see lagp_precision)
 *   sel         M x n_max int32 output: the chosen design rows in the order
 *               chosen (the n0 seeds first); -1 past n[m]
 *   alc         M x n_max FP64 output or NULL: raw Delta of Eq. (dxy) of the
 *               row chosen at step j (NaN for the seeds and past n[m]);
 *               multiplying by psi_j / (j - 2) gives the normalised value of
 *               the paper's step 9
 *   status      M int32 output: LAGP_OK / LAGP_ENOTPD / LAGP_EINVAL per
 *               location
 * Requires n_max <= 128 (K_j^{-1} is kept in shared memory). */
lagp_status lagp_alc_select(lagp_ctx *ctx, const void *X, int64_t N, int32_t p,
                            lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *idx,
                            const int32_t *Nprime, int32_t Nprime_max, int32_t n0,
                            const int32_t *n, int32_t n_max, const double *d, double g,
                            lagp_precision prec, int32_t *sel, double *alc, int32_t *status);

/* ---------------------------------------- a2..a7: search + local predict
 * lagp_alc_select followed by the predictive equations of a7 on each chosen
 * design, fused into the same kernel: the FP64 partitioned inverse that
 * grows K_j^{-1} (Sec. 2.2) also grows alpha_j = K_j^{-1} Y_j,
 * psi_j = Y_j^T K_j^{-1} Y_j and k_j(x)^T K_j^{-1} k_j(x) in O(j) per step:
 * with b* = K_j^{-1} k_j(x*), mu = 1/(1 + g - k_j(x*)^T b*) and
 * r_y = y* - Y_j^T b*,  alpha_{j+1} = [alpha_j - mu r_y b*; mu r_y],
 * psi_{j+1} = psi_j + mu r_y^2,  and likewise for k(x)^T K^{-1} k(x).
 * Outputs mean, s2, df (M each, FP64) equal those of lagp_predict on sel up
 * to rounding (here K_n^{-1} comes from the partitioned inverse, there from a
 * fresh Cholesky factorisation).  Other arguments as lagp_alc_select. */
lagp_status lagp_alc_predict(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                             lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *idx,
                             const int32_t *Nprime, int32_t Nprime_max, int32_t n0,
                             const int32_t *n, int32_t n_max, const double *d, double g,
                             lagp_precision prec, int32_t *sel, double *alc, double *mean,
                             double *s2, double *df, int32_t *status);

/* ------------------------------------------------------ a7: local predict
 * Predictive equations (Eqs. predgp, preds2) on each location's local design:
 *   mean = k^T K^{-1} Y_n,   psi = Y_n^T K^{-1} Y_n,
 *   s2   = psi (1 + g - k^T K^{-1} k) / n,   df = n,
 * with K_n factorised by FP64 Cholesky.  The predictive variance is
 * s2 * df / (df - 2).
 *   Y      N responses (dtype);  sel  M x n_max design rows (from
 *          lagp_alc_select);  n  M sizes or NULL (= n_max);  d  M lengthscales
 *          (a location whose sel row holds a row outside [0, N), n[m] outside
 *          [1, n_max] or d[m] <= 0 gets status LAGP_EINVAL, NaN outputs)
 *   mean, s2, df   M FP64 outputs;  status  M int32 outputs */
lagp_status lagp_predict(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                         lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *sel,
                         const int32_t *n, int32_t n_max, const double *d, double g,
                         double *mean, double *s2, double *df, int32_t *status);

/* ------------------------------- a4/a5 for one location and a fixed design
 * The ALC criterion of Eq. (dxy) for Nc candidates at one reference location
 * x and a given design of n rows — the computation Sec. 4.1 times (one x,
 * N' = 60,000 candidates, n = 16..512).  Per candidate, with K_n = L L^T
 * (FP64 Cholesky of the design's covariance, nugget g on the diagonal):
 *   u_c = L^{-1} k_n(x_c),  s_c = |u_c|^2,  q_c = (L^{-1} k_n(x))^T u_c,
 *   delta[c] = (K(x_c, x) - q_c)^2 / (1 + g - s_c)
 * (Eq. (dxy) with Eq. (piedef), simplified), FP64 throughout.
 *   X        N x p design (dtype), device
 *   x        p FP64 coordinates of the location, device
 *   design   n design rows (int32, device), 1 <= n <= 1024
 *   cands    Nc candidate rows (int32, device)
 *   delta    Nc FP64 outputs (NaN for every candidate when K_n is not
 *            positive definite)
 *   status   1 int32 output: LAGP_OK or LAGP_ENOTPD (K_n not positive definite)
 * Two kernels: the factorisation of K_n (one CTA) and the candidates'
 * triangular solves (one thread per candidate). */
lagp_status lagp_alc_eval(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                          const double *x, const int32_t *design, int32_t n, const int32_t *cands,
                          int64_t Nc, double d, double g, double *delta, int32_t *status);

/* --------------------------------------------- separable lengthscales
 * Sec. 3.1 notes the separable correlation, a vector theta of lengthscales:
 * K(x,x') = exp(-sum_i (x_i - x'_i)^2 / theta_i).  It equals the isotropic
 * correlation with d = 1 of the inputs scaled column by column,
 * x_i / sqrt(theta_i).  This call writes that scaling (FP64, N x p, device):
 * the search (lagp_alc_select, lagp_alc_predict, lagp_alc_eval) and the
 * prediction (lagp_predict) called on scaled design and locations with
 * d = 1 evaluate the separable correlation.  The candidate sets keep coming
 * from lagp_knn on the unscaled inputs (the N' nearest neighbours in the
 * input space; calling it on scaled inputs gives the neighbours in the
 * theta-scaled metric instead).  The likelihood, MLE and adjoint entry
 * points estimate a single (isotropic) d.
 *   X      N x p inputs (dtype), device;  theta  p lengthscales > 0, device
 *   Xs     N x p FP64 outputs, device */
lagp_status lagp_scale_inputs(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                              const double *theta, double *Xs);

/* ------------------------------------------------------- a8: local MLE
 * Per-location Newton maximisation in d of the concentrated log-likelihood
 * of Eq. (gpk), log p(Y_n | d) = log Gamma(n/2) - (n/2) log(2 pi)
 *   - (1/2) log|K_n| - (n/2) log(psi/2), on the local design (Fig. 1 step 3),
 * with analytic first and second derivatives in d, all in FP64.  Step rule:
 * Newton step -l'/l'' when l'' < 0, else doubling/halving in the gradient's
 * direction; proposals are clipped to [dmin, dmax]; a Newton step no longer
 * than 1e-3 d is taken as it is (near the maximiser the rise in l it brings
 * is below the FP64 resolution of l), any other proposal is halved (at most
 * 20 times) until l does not decrease; stop when the step is below 1e-10 d,
 * when no halving recovers an increase, or after max_iter iterations.
 *   d       M lengthscales, in: starting values, out: estimates
 *   llik, dllik, d2llik   M FP64 outputs at the final d (any may be NULL)
 *   iters   M int32 iterations taken (may be NULL);  status  M int32
 * max_iter = 0 evaluates the likelihood and its derivatives at d only. */
lagp_status lagp_mle_step(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                          lagp_dtype dtype, int64_t M, const int32_t *sel, const int32_t *n,
                          int32_t n_max, double *d, double g, double dmin, double dmax,
                          int32_t max_iter, double *llik, double *dllik, double *d2llik,
                          int32_t *iters, int32_t *status);

/* ------------------------------------------- adjoint of a7 / a8 in (d, g)
 * Analytic derivatives of the local predictive mean and scale (Eqs. predgp,
 * preds2) and of the log-likelihood (Eq. gpk) with respect to the
 * lengthscale d and the nugget g, per location, FP64:
 *   dK/dd = (D/d^2) o exp(-D/d),   dK/dg = I,   d(K^{-1}) = -K^{-1} dK K^{-1}.
 * Outputs are M-vectors (any may be NULL except status). */
lagp_status lagp_predict_grad(lagp_ctx *ctx, const void *X, const void *Y, int64_t N,
                              int32_t p, lagp_dtype dtype, const void *Xref, int64_t M,
                              const int32_t *sel, const int32_t *n, int32_t n_max,
                              const double *d, double g, double *dmean_dd, double *dmean_dg,
                              double *ds2_dd, double *ds2_dg, double *dllik_dd,
                              double *dllik_dg, int32_t *status);

/* ----------------------------------------- a7 without device allocation
 * The paper has no counterpart to this entry point.  It computes exactly what
 * lagp_predict computes, for callers that cannot allocate device memory:
 * applications whose own allocator owns all device memory after start-up,
 * services under a device-memory budget fixed when they start, and
 * latency-critical paths that cannot afford cudaMalloc's implicit device
 * synchronisation.  Its scratch is a fixed array inside the library (2 MiB
 * plus 256 bytes of device memory, held by every GPU that loads the library
 * until the process exits), so the call itself calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *   Arguments, outputs and per-location status are those of lagp_predict.
 *   Limit: n_max <= 64 (LAGP_EINVAL with an explanatory message otherwise).
 *   All calls share the scratch: calls that overlap on the GPU (different
 *   streams, or different contexts on one device) race, so order them.
 *   The first call on a device looks up the scratch's device address, with
 *   that device current; make this first call before any stream capture. */
lagp_status lagp_predict_noalloc(lagp_ctx *ctx, const void *X, const void *Y, int64_t N,
                                 int32_t p, lagp_dtype dtype, const void *Xref, int64_t M,
                                 const int32_t *sel, const int32_t *n, int32_t n_max,
                                 const double *d, double g, double *mean, double *s2, double *df,
                                 int32_t *status);

/* --------------------------------------------- whole method, host buffers
 * The multi-stage algorithm of Fig. 1 for every reference location:
 * kNN (a1) -> greedy ALC design at lengthscale d0 (a2..a6) -> local MLE of d
 * on that design (a8) -> ... -> prediction (a7).  mle_rounds = 0 predicts on
 * the design at d0 (no MLE; the prediction is carried by the search itself).
 * mle_rounds = r >= 1 runs Fig. 1 steps 2-3 r times (step 4: "repeat as
 * desired"): each round searches the designs at the current per-location d
 * and then moves d to the MLE on that design, starting from the current d;
 * the prediction (step 5) uses the last design and estimate.  r = 2 is the
 * two-stage scheme of Sec. 2.2 (designs re-searched with the local
 * estimates).  All array arguments are HOST pointers; the inputs are copied
 * to the device, and the outputs copied back, inside the call, which returns
 * after the outputs are in host memory.
 *   Nprime, n   M per-location values or NULL (all = Nprime_max / n_max)
 *   mle_rounds  0 .. LAGP_MAX_MLE_ROUNDS; dmin, dmax, max_iter as in
 *               lagp_mle_step (ignored when mle_rounds = 0)
 *   mean, s2, df, status   M outputs (status: the first failing stage, in
 *               the order kNN, each round's search and MLE, prediction)
 *   d_out  M final lengthscales or NULL */
#define LAGP_MAX_MLE_ROUNDS 16
lagp_status lagp_agp(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                     lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *Nprime,
                     int32_t Nprime_max, int32_t n0, const int32_t *n, int32_t n_max,
                     double d0, double g, lagp_precision prec, int32_t mle_rounds, double dmin,
                     double dmax, int32_t max_iter, double *mean, double *s2, double *df,
                     double *d_out, int32_t *status);

#ifdef __cplusplus
}
#endif
#endif /* LAGP_H */
