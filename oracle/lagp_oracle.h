/*
 * lagp_oracle.h -- plain, slow FP64 reference for local approximate GP
 * regression (Gramacy, Niemi & Weiss, "Massively parallel approximate
 * Gaussian process regression").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the correctness yardstick for the
 * CUDA library in paper_1310_5182_gb300/; it shares no code, header, table or
 * helper with it.  Only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py may load it.  The product path never calls it.
 *
 * Conventions shared with the paper (Sec. 2.1, Sec. 2.2):
 *   K(x,x') = exp(-||x-x'||^2 / d)   isotropic Gaussian correlation, d = theta
 *   design matrices carry the nugget g on their diagonal; cross covariances
 *   (to the reference location x, or between distinct rows) carry none; the
 *   self-covariance of a candidate is K(x_c,x_c) = 1 + g.
 * All arrays are row-major host arrays; all arithmetic is IEEE FP64 with no
 * contraction of multiply-add (the library is compiled -ffp-contract=off).
 */
#ifndef LAGP_ORACLE_H
#define LAGP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOTPD = 2 };

/* Separable lengthscales theta[0..p-1] for the correlations of the search
 * and the prediction (orc_alc_select, orc_alc_scores, orc_partitioned_inverse,
 * orc_predict): K(x,x') = exp(-(sum_i (x_i - x'_i)^2 / theta_i) / d).
 * theta = NULL returns to the isotropic form.  The kNN stays Euclidean; the
 * likelihood, MLE and adjoint functions are isotropic only. */
int orc_set_separable(const double *theta, int p);

/* Number of OpenMP threads used by the per-location loops (1 = serial).
 * Returns the value actually in effect (1 when built without OpenMP). */
int orc_set_threads(int nthreads);

/* Exact N'-nearest-neighbour candidate set (Sec. 3.1: the search is
 * restricted to the N' nearest neighbours of x; Fig. 1 step 2(a) takes the
 * first n0 of them as the initial design).
 * d2 = sum_i (x_i - X_{r,i})^2 accumulated in coordinate order; rows sorted by
 * (d2, r) ascending.  idx is M x Npmax, padded with -1 past Np[m]. */
int orc_knn(const double *X, int64_t N, int p, const double *Xref, int64_t M,
            const int32_t *Np, int32_t Npmax, int32_t *idx);

/* Greedy ALC local design search (Fig. 1 steps 2(a)-2(b); Eq. (dxy) with
 * g_j, m_j from Eq. (piedef); partitioned inverse update of Sec. 2.2).
 *   idx     M x Npmax candidate rows (from orc_knn), first n0 = NN seed
 *   n       per-location final design size, n0 <= n[m] <= Np[m]
 *   d       per-location lengthscale
 *   sel     M x nmax selected design rows in the order chosen (-1 padded)
 *   alc     M x nmax or NULL: raw Delta of the row chosen at step j
 *           (NaN for the n0 seed rows and past n[m])
 *   topk>0: top_idx/top_val (M x nmax x topk) receive, for every step j, the
 *           topk best candidates (design row, Delta) in decreasing Delta order,
 *           ties to the lower design row; -1/NaN padded.
 *   status  per location: ORC_OK or ORC_ENOTPD (a non-positive m_j^{-1}). */
int orc_alc_select(const double *X, int64_t N, int p, const double *Xref, int64_t M,
                   const int32_t *idx, const int32_t *Np, int32_t Npmax, int32_t n0,
                   const int32_t *n, int32_t nmax, const double *d, double g,
                   int32_t *sel, double *alc, int32_t topk, int32_t *top_idx,
                   double *top_val, int32_t *status);

/* ALC of every candidate at one step of one location, both in the paper's
 * three-term form (Eq. dxy) and in the simplified form m_j (kappa - q)^2.
 * design: the j chosen rows; cands: nc candidate rows.  For tests. */
int orc_alc_scores(const double *X, int64_t N, int p, const double *x,
                   const int32_t *design, int32_t j, const int32_t *cands, int32_t nc,
                   double d, double g, double *delta3, double *delta_simple);

/* Partitioned-inverse growth of K^{-1} along a given design order (Sec. 2.2):
 * starts from the direct inverse of the first n0 rows, then adds rows one at a
 * time.  Kinv receives the n x n result.  For tests. */
int orc_partitioned_inverse(const double *X, int64_t N, int p, const int32_t *design,
                            int32_t n0, int32_t n, double d, double g, double *Kinv);

/* Local predictive equations (Eqs. predgp, preds2) on the selected design,
 * with K_n^{-1} formed directly by Cholesky:
 *   mean = k^T K^{-1} Y,  psi = Y^T K^{-1} Y,
 *   s2 = psi (1 + g - k^T K^{-1} k) / n,  df = n.  */
int orc_predict(const double *X, const double *Y, int64_t N, int p, const double *Xref,
                int64_t M, const int32_t *sel, const int32_t *n, int32_t nmax,
                const double *d, double g, double *mean, double *s2, double *df,
                int32_t *status);

/* Concentrated log-likelihood of Eq. (gpk) on the selected design and its
 * first two derivatives in d.  Any of the outputs may be NULL. */
int orc_llik(const double *X, const double *Y, int64_t N, int p, int64_t M,
             const int32_t *sel, const int32_t *n, int32_t nmax, const double *d,
             double g, double *llik, double *dllik, double *d2llik, int32_t *status);

/* Per-location Newton maximisation of the log-likelihood in d (Fig. 1 step 3)
 * within [dmin, dmax], at most max_iter iterations.  d is updated in place. */
int orc_mle(const double *X, const double *Y, int64_t N, int p, int64_t M,
            const int32_t *sel, const int32_t *n, int32_t nmax, double *d, double g,
            double dmin, double dmax, int32_t max_iter, double *llik, double *dllik,
            double *d2llik, int32_t *iters, int32_t *status);

/* Derivatives of the predictive mean and scale with respect to d and g,
 * analytic (differentiating Eqs. predgp/preds2).  For the adjoint tests. */
int orc_predict_grad(const double *X, const double *Y, int64_t N, int p,
                     const double *Xref, int64_t M, const int32_t *sel, const int32_t *n,
                     int32_t nmax, const double *d, double g, double *dmean_dd,
                     double *dmean_dg, double *ds2_dd, double *ds2_dg, double *dllik_dg,
                     int32_t *status);

#ifdef __cplusplus
}
#endif
#endif
