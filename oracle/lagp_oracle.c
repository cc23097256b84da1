/*
 * lagp_oracle.c -- plain FP64 reference implementation of local approximate
 * GP regression with ALC local design search (Gramacy, Niemi & Weiss,
 * "Massively parallel approximate Gaussian process regression").
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py.  It is deliberately slow and literal: every
 * function follows the paper's equations in the paper's order and notation,
 * with no blocking, fusion or reordering.  It shares no code with the CUDA
 * library.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *  - design matrices K_j carry the nugget g on the diagonal; cross
 *    covariances carry none; a candidate's self covariance K_j(x',x') = 1+g
 *    (Fig. 3 step 5 uses 1 + eta).
 *  - g_j carries the minus sign of Eq. (piedef) (Fig. 3 step 5 drops it).
 *  - the candidate pool at step j is the N' nearest neighbours minus the j
 *    rows already chosen (Sec. 3.1), the loop runs j = n0..n-1 (Fig. 1).
 *  - ties: kNN by (d2, row); ALC argmax to the lower design row.
 *  - K(x,x) in the predictive scale is 1+g (a noisy response).
 */
#include "lagp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

int orc_set_threads(int nthreads) {
#ifdef _OPENMP
    g_threads = nthreads < 1 ? 1 : nthreads;
    return g_threads;
#else
    (void)nthreads;
    g_threads = 1;
    return 1;
#endif
}

/* ---------------------------------------------------------------- basics */

/* squared Euclidean distance, coordinates summed in order 0..p-1, each term
 * formed as a separate subtract, multiply and add (no fused multiply-add). */
static double sqdist(const double *a, const double *b, int p) {
    double s = 0.0;
    for (int i = 0; i < p; i++) {
        double diff = a[i] - b[i];
        double sq = diff * diff;
        s = s + sq;
    }
    return s;
}

/* Separable lengthscales theta_1..theta_p (Sec. 3.1 notes the separable
 * version of the correlation as a simple modification): when set, the
 * correlations used by the search and the prediction are
 *   K(x,x') = exp(-(sum_i (x_i - x'_i)^2 / theta_i) / d). */
static int g_sep = 0;
static double g_theta[64];

int orc_set_separable(const double *theta, int p) {
    if (!theta) {
        g_sep = 0;
        return ORC_OK;
    }
    if (p < 1 || p > 64) return ORC_EINVAL;
    for (int i = 0; i < p; i++)
        if (!(theta[i] > 0.0)) return ORC_EINVAL;
    for (int i = 0; i < p; i++) g_theta[i] = theta[i];
    g_sep = 1;
    return ORC_OK;
}

/* Gaussian correlation: isotropic K(x,x') = exp(-||x-x'||^2 / d) (Sec. 2.1),
 * or the separable form above */
static double kern(const double *a, const double *b, int p, double d) {
    if (g_sep) {
        double s = 0.0;
        for (int i = 0; i < p; i++) {
            double diff = a[i] - b[i];
            double sq = diff * diff;
            s = s + sq / g_theta[i];
        }
        return exp(-s / d);
    }
    return exp(-sqdist(a, b, p) / d);
}

/* Cholesky factorisation A = L L^T of an n x n SPD matrix (row-major, lower
 * triangle of L written into L, upper part zeroed).  Returns 0 on success,
 * -1 if a pivot is not positive. */
static int cholesky(const double *A, int n, double *L) {
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int k = 0; k < j; k++) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int k = 0; k < j; k++) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / ljj;
        }
    }
    return 0;
}

/* A^{-1} = L^{-T} L^{-1} from the Cholesky factor, by solving A x = e_c for
 * every unit vector.  Returns 0 / -1 like cholesky(). */
static int spd_inverse(const double *A, int n, double *Ainv) {
    double *L = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = cholesky(A, n, L);
    if (rc == 0) {
        for (int c = 0; c < n; c++) {
            for (int i = 0; i < n; i++) { /* forward: L y = e_c */
                double t = (i == c) ? 1.0 : 0.0;
                for (int k = 0; k < i; k++) t -= L[i * n + k] * y[k];
                y[i] = t / L[i * n + i];
            }
            for (int i = n - 1; i >= 0; i--) { /* backward: L^T x = y */
                double t = y[i];
                for (int k = i + 1; k < n; k++) t -= L[k * n + i] * Ainv[k * n + c];
                Ainv[i * n + c] = t / L[i * n + i];
            }
        }
    }
    free(L);
    free(y);
    return rc;
}

/* log|A| from the Cholesky factor (sum of 2 log L_ii). */
static double logdet_from_chol(const double *L, int n) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += 2.0 * log(L[i * n + i]);
    return s;
}

/* K_j over the design rows: exp(-D/d) + g I */
static void design_cov(const double *X, int p, const int32_t *rows, int j, double d, double g,
                       double *K) {
    for (int a = 0; a < j; a++)
        for (int b = 0; b < j; b++) {
            double v = kern(X + (size_t)rows[a] * p, X + (size_t)rows[b] * p, p, d);
            if (a == b) v += g;
            K[a * j + b] = v;
        }
}

/* --------------------------------------------------------------- kNN (a1) */

typedef struct {
    double d2;
    int32_t row;
} orc_pair;

static int pair_cmp(const void *pa, const void *pb) {
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->d2 < b->d2) return -1;
    if (a->d2 > b->d2) return 1;
    return (a->row > b->row) - (a->row < b->row);
}

int orc_knn(const double *X, int64_t N, int p, const double *Xref, int64_t M,
            const int32_t *Np, int32_t Npmax, int32_t *idx) {
    if (N < 1 || p < 1 || M < 0 || Npmax < 1 || Npmax > N || N > INT32_MAX) return ORC_EINVAL;
    for (int64_t m = 0; m < M; m++) {
        int32_t k = Np ? Np[m] : Npmax;
        if (k < 1 || k > Npmax) return ORC_EINVAL;
    }
    int rc = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int64_t m = 0; m < M; m++) {
        orc_pair *pr = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)N);
        const double *x = Xref + (size_t)m * p;
        for (int64_t r = 0; r < N; r++) {
            pr[r].d2 = sqdist(x, X + (size_t)r * p, p);
            pr[r].row = (int32_t)r;
        }
        qsort(pr, (size_t)N, sizeof(orc_pair), pair_cmp);
        int32_t k = Np ? Np[m] : Npmax;
        for (int32_t t = 0; t < Npmax; t++) idx[(size_t)m * Npmax + t] = (t < k) ? pr[t].row : -1;
        free(pr);
    }
    return rc;
}

/* ------------------------------------------------- ALC criterion (a4, a5) */

/* Eq. (piedef) and Eq. (dxy) for one candidate x' given the current design:
 *   m_j^{-1}(x') = K_j(x',x') - k_j(x')^T K_j^{-1} k_j(x')
 *   g_j(x')      = -m_j(x') K_j^{-1} k_j(x')
 *   Delta = k_j(x)^T G_j m_j^{-1} k_j(x) + 2 k_j(x)^T g_j K(x',x) + K(x',x)^2 m_j
 * with G_j = g_j g_j^T.  Work vectors kc, Kkc, gv have length j.
 * Returns the three-term value; *simple receives m_j (K(x',x) - q)^2 with
 * q = k_j(x)^T K_j^{-1} k_j(x'); *minv_out receives m_j^{-1}. */
static double alc_one(const double *X, int p, const double *x, const int32_t *design, int j,
                      const double *Kinv, const double *kx, int32_t cand, double d, double g,
                      double *kc, double *Kkc, double *gv, double *simple, double *minv_out) {
    const double *xc = X + (size_t)cand * p;
    for (int i = 0; i < j; i++) kc[i] = kern(xc, X + (size_t)design[i] * p, p, d);
    for (int i = 0; i < j; i++) {
        double t = 0.0;
        for (int k = 0; k < j; k++) t += Kinv[i * j + k] * kc[k];
        Kkc[i] = t;
    }
    double quad = 0.0;
    for (int i = 0; i < j; i++) quad += kc[i] * Kkc[i];
    double minv = (1.0 + g) - quad;
    double m = 1.0 / minv;
    for (int i = 0; i < j; i++) gv[i] = -m * Kkc[i];
    double kxg = 0.0;
    for (int i = 0; i < j; i++) kxg += kx[i] * gv[i];
    double kappa = kern(xc, x, p, d);
    double term1 = kxg * kxg * minv; /* k^T g g^T k * m^{-1} */
    double term2 = 2.0 * kxg * kappa;
    double term3 = kappa * kappa * m;
    double q = 0.0;
    for (int i = 0; i < j; i++) q += kx[i] * Kkc[i];
    if (simple) *simple = m * (kappa - q) * (kappa - q);
    if (minv_out) *minv_out = minv;
    return term1 + term2 + term3;
}

/* Partitioned inverse (Sec. 2.2, Eq. piedef): given K_j^{-1} (j x j) and a new
 * row x* with k* = k_j(x*), m = 1/(1+g - k*^T K^{-1} k*) and g = -m K^{-1} k*,
 *   K_{j+1}^{-1} = [ K^{-1} + g g^T / m , g ; g^T , m ].
 * Writes the (j+1) x (j+1) result into Knew.  Returns -1 if m^{-1} <= 0. */
static int grow_inverse(const double *Kinv, int j, const double *kstar, double g, double *Knew,
                        double *work) {
    for (int i = 0; i < j; i++) {
        double t = 0.0;
        for (int k = 0; k < j; k++) t += Kinv[i * j + k] * kstar[k];
        work[i] = t;
    }
    double quad = 0.0;
    for (int i = 0; i < j; i++) quad += kstar[i] * work[i];
    double minv = (1.0 + g) - quad;
    if (!(minv > 0.0)) return -1;
    double m = 1.0 / minv;
    int jn = j + 1;
    for (int i = 0; i < j; i++) work[i] = -m * work[i]; /* g vector */
    for (int a = 0; a < j; a++)
        for (int b = 0; b < j; b++) Knew[a * jn + b] = Kinv[a * j + b] + work[a] * work[b] / m;
    for (int a = 0; a < j; a++) {
        Knew[a * jn + j] = work[a];
        Knew[j * jn + a] = work[a];
    }
    Knew[j * jn + j] = m;
    return 0;
}

/* ---------------------------------------------- greedy search (a2 .. a6) */

static int select_one(const double *X, int p, const double *x, const int32_t *cands, int32_t Np,
                      int32_t n0, int32_t n, double d, double g, int32_t *sel, double *alc,
                      int32_t topk, int32_t *top_idx, double *top_val, int32_t nmax) {
    int32_t *design = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *Kinv = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *Knew = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *K0 = (double *)malloc(sizeof(double) * (size_t)n0 * n0);
    double *kx = (double *)malloc(sizeof(double) * (size_t)n);
    double *kc = (double *)malloc(sizeof(double) * (size_t)n);
    double *Kkc = (double *)malloc(sizeof(double) * (size_t)n);
    double *gv = (double *)malloc(sizeof(double) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)Np);
    unsigned char *chosen = (unsigned char *)calloc((size_t)Np, 1);
    int rc = ORC_OK;

    /* step 2(a): the n0 nearest neighbours, inverse formed directly */
    for (int i = 0; i < n0; i++) {
        design[i] = cands[i];
        chosen[i] = 1;
    }
    design_cov(X, p, design, n0, d, g, K0);
    if (spd_inverse(K0, n0, Kinv) != 0) rc = ORC_ENOTPD;

    /* step 2(b): j = n0 .. n-1 */
    for (int j = n0; j < n && rc == ORC_OK; j++) {
        for (int i = 0; i < j; i++) kx[i] = kern(x, X + (size_t)design[i] * p, p, d);
        int best = -1;
        for (int c = 0; c < Np; c++) {
            if (chosen[c]) continue;
            double minv;
            delta[c] = alc_one(X, p, x, design, j, Kinv, kx, cands[c], d, g, kc, Kkc, gv, NULL,
                               &minv);
            if (!(minv > 0.0)) {
                rc = ORC_ENOTPD;
                break;
            }
            if (best < 0 || delta[c] > delta[best] ||
                (delta[c] == delta[best] && cands[c] < cands[best]))
                best = c;
        }
        if (rc != ORC_OK || best < 0) {
            if (best < 0) rc = ORC_ENOTPD;
            break;
        }
        if (topk > 0 && top_idx && top_val) {
            /* the topk best candidates of this step, by repeated selection */
            unsigned char *taken = (unsigned char *)calloc((size_t)Np, 1);
            for (int t = 0; t < topk; t++) {
                int b = -1;
                for (int c = 0; c < Np; c++) {
                    if (chosen[c] || taken[c]) continue;
                    if (b < 0 || delta[c] > delta[b] ||
                        (delta[c] == delta[b] && cands[c] < cands[b]))
                        b = c;
                }
                size_t o = ((size_t)j * topk) + t;
                top_idx[o] = (b < 0) ? -1 : cands[b];
                top_val[o] = (b < 0) ? NAN : delta[b];
                if (b >= 0) taken[b] = 1;
            }
            free(taken);
        }
        /* augment the design and grow K^{-1} by the partitioned inverse */
        const double *xs = X + (size_t)cands[best] * p;
        for (int i = 0; i < j; i++) kc[i] = kern(xs, X + (size_t)design[i] * p, p, d);
        if (grow_inverse(Kinv, j, kc, g, Knew, Kkc) != 0) {
            rc = ORC_ENOTPD;
            break;
        }
        memcpy(Kinv, Knew, sizeof(double) * (size_t)(j + 1) * (j + 1));
        design[j] = cands[best];
        chosen[best] = 1;
        if (alc) alc[j] = delta[best];
    }
    (void)nmax;
    for (int i = 0; i < n; i++) sel[i] = (rc == ORC_OK) ? design[i] : -1;
    free(design);
    free(Kinv);
    free(Knew);
    free(K0);
    free(kx);
    free(kc);
    free(Kkc);
    free(gv);
    free(delta);
    free(chosen);
    return rc;
}

int orc_alc_select(const double *X, int64_t N, int p, const double *Xref, int64_t M,
                   const int32_t *idx, const int32_t *Np, int32_t Npmax, int32_t n0,
                   const int32_t *n, int32_t nmax, const double *d, double g,
                   int32_t *sel, double *alc, int32_t topk, int32_t *top_idx,
                   double *top_val, int32_t *status) {
    if (N < 1 || p < 1 || M < 0 || n0 < 1 || nmax < n0 || Npmax < 1 || !(g >= 0.0))
        return ORC_EINVAL;
    for (int64_t m = 0; m < M; m++) {
        int32_t k = Np ? Np[m] : Npmax;
        int32_t nm = n ? n[m] : nmax;
        if (k < 1 || k > Npmax || k > N || nm < n0 || nm > nmax || nm > k || !(d[m] > 0.0))
            return ORC_EINVAL;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int64_t m = 0; m < M; m++) {
        int32_t k = Np ? Np[m] : Npmax;
        int32_t nm = n ? n[m] : nmax;
        int32_t *s = sel + (size_t)m * nmax;
        double *a = alc ? alc + (size_t)m * nmax : NULL;
        int32_t *ti = (topk > 0 && top_idx) ? top_idx + (size_t)m * nmax * topk : NULL;
        double *tv = (topk > 0 && top_val) ? top_val + (size_t)m * nmax * topk : NULL;
        for (int t = 0; t < nmax; t++) {
            s[t] = -1;
            if (a) a[t] = NAN;
        }
        if (ti)
            for (size_t t = 0; t < (size_t)nmax * topk; t++) {
                ti[t] = -1;
                tv[t] = NAN;
            }
        int rc = select_one(X, p, Xref + (size_t)m * p, idx + (size_t)m * Npmax, k, n0, nm, d[m],
                            g, s, a, topk, ti, tv, nmax);
        status[m] = rc;
    }
    return ORC_OK;
}

int orc_alc_scores(const double *X, int64_t N, int p, const double *x,
                   const int32_t *design, int32_t j, const int32_t *cands, int32_t nc,
                   double d, double g, double *delta3, double *delta_simple) {
    if (N < 1 || p < 1 || j < 1 || nc < 0 || !(d > 0.0)) return ORC_EINVAL;
    double *K = (double *)malloc(sizeof(double) * (size_t)j * j);
    double *Kinv = (double *)malloc(sizeof(double) * (size_t)j * j);
    double *kx = (double *)malloc(sizeof(double) * (size_t)j);
    double *kc = (double *)malloc(sizeof(double) * (size_t)j);
    double *Kkc = (double *)malloc(sizeof(double) * (size_t)j);
    double *gv = (double *)malloc(sizeof(double) * (size_t)j);
    design_cov(X, p, design, j, d, g, K);
    int rc = spd_inverse(K, j, Kinv) == 0 ? ORC_OK : ORC_ENOTPD;
    if (rc == ORC_OK) {
        for (int i = 0; i < j; i++) kx[i] = kern(x, X + (size_t)design[i] * p, p, d);
        for (int c = 0; c < nc; c++)
            delta3[c] = alc_one(X, p, x, design, j, Kinv, kx, cands[c], d, g, kc, Kkc, gv,
                                &delta_simple[c], NULL);
    }
    free(K);
    free(Kinv);
    free(kx);
    free(kc);
    free(Kkc);
    free(gv);
    return rc;
}

int orc_partitioned_inverse(const double *X, int64_t N, int p, const int32_t *design,
                            int32_t n0, int32_t n, double d, double g, double *Kinv) {
    if (N < 1 || p < 1 || n0 < 1 || n < n0 || !(d > 0.0)) return ORC_EINVAL;
    double *K0 = (double *)malloc(sizeof(double) * (size_t)n0 * n0);
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *B = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *ks = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    design_cov(X, p, design, n0, d, g, K0);
    int rc = spd_inverse(K0, n0, A) == 0 ? ORC_OK : ORC_ENOTPD;
    for (int j = n0; j < n && rc == ORC_OK; j++) {
        const double *xs = X + (size_t)design[j] * p;
        for (int i = 0; i < j; i++) ks[i] = kern(xs, X + (size_t)design[i] * p, p, d);
        if (grow_inverse(A, j, ks, g, B, w) != 0) rc = ORC_ENOTPD;
        else memcpy(A, B, sizeof(double) * (size_t)(j + 1) * (j + 1));
    }
    if (rc == ORC_OK) memcpy(Kinv, A, sizeof(double) * (size_t)n * n);
    free(K0);
    free(A);
    free(B);
    free(ks);
    free(w);
    return rc;
}

/* ------------------------------------------------------- prediction (a7) */

static int predict_one(const double *X, const double *Y, int p, const double *x,
                       const int32_t *s, int nm, double d, double g, double *mean, double *s2,
                       double *df) {
    double *K = (double *)malloc(sizeof(double) * (size_t)nm * nm);
    double *Ki = (double *)malloc(sizeof(double) * (size_t)nm * nm);
    double *kx = (double *)malloc(sizeof(double) * (size_t)nm);
    double *y = (double *)malloc(sizeof(double) * (size_t)nm);
    design_cov(X, p, s, nm, d, g, K);
    int rc = spd_inverse(K, nm, Ki) == 0 ? ORC_OK : ORC_ENOTPD;
    if (rc == ORC_OK) {
        for (int i = 0; i < nm; i++) {
            kx[i] = kern(x, X + (size_t)s[i] * p, p, d);
            y[i] = Y[s[i]];
        }
        double mu = 0.0, psi = 0.0, kk = 0.0;
        for (int a = 0; a < nm; a++)
            for (int b = 0; b < nm; b++) {
                mu += kx[a] * Ki[a * nm + b] * y[b];
                psi += y[a] * Ki[a * nm + b] * y[b];
                kk += kx[a] * Ki[a * nm + b] * kx[b];
            }
        *mean = mu;
        *s2 = psi * ((1.0 + g) - kk) / (double)nm;
        *df = (double)nm;
    }
    free(K);
    free(Ki);
    free(kx);
    free(y);
    return rc;
}

int orc_predict(const double *X, const double *Y, int64_t N, int p, const double *Xref,
                int64_t M, const int32_t *sel, const int32_t *n, int32_t nmax,
                const double *d, double g, double *mean, double *s2, double *df,
                int32_t *status) {
    if (N < 1 || p < 1 || M < 0 || nmax < 1 || !(g >= 0.0)) return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int64_t m = 0; m < M; m++) {
        int32_t nm = n ? n[m] : nmax;
        mean[m] = s2[m] = df[m] = NAN;
        status[m] = predict_one(X, Y, p, Xref + (size_t)m * p, sel + (size_t)m * nmax, nm, d[m],
                                g, &mean[m], &s2[m], &df[m]);
    }
    return ORC_OK;
}

/* --------------------------------------------- likelihood and MLE (a8) */

/* Eq. (gpk): log p(Y|d) = log Gamma(n/2) - (n/2) log(2 pi) - (1/2) log|K|
 *                         - (n/2) log(psi/2),      psi = Y^T K^{-1} Y.
 * Derivatives in d, with D the squared distances, E = exp(-D/d),
 *   K'  = (D/d^2) o E,            K'' = (D^2/d^4 - 2 D/d^3) o E,
 *   l'  = -1/2 tr(K^{-1}K') + (n/2) phi/psi,  phi = a^T K' a,  a = K^{-1} Y,
 *   l'' = 1/2 tr(K^{-1}K'K^{-1}K') - 1/2 tr(K^{-1}K'')
 *         + (n/2) [ (a^T K'' a - 2 a^T K' K^{-1} K' a)/psi + phi^2/psi^2 ].
 * Derivative in g: dK/dg = I, so
 *   dl/dg = -1/2 tr(K^{-1}) + (n/2) a^T a / psi.  */
typedef struct {
    double l, dl, d2l, dldg;
} orc_lik;

static int llik_one(const double *X, const double *Y, int p, const int32_t *s, int nm, double d,
                    double g, orc_lik *out) {
    size_t nn = (size_t)nm * nm;
    double *K = (double *)malloc(sizeof(double) * nn);
    double *L = (double *)malloc(sizeof(double) * nn);
    double *Ki = (double *)malloc(sizeof(double) * nn);
    double *D = (double *)malloc(sizeof(double) * nn);
    double *K1 = (double *)malloc(sizeof(double) * nn);
    double *K2 = (double *)malloc(sizeof(double) * nn);
    double *A1 = (double *)malloc(sizeof(double) * nn); /* K^{-1} K' */
    double *a = (double *)malloc(sizeof(double) * (size_t)nm);
    double *y = (double *)malloc(sizeof(double) * (size_t)nm);
    double *t1 = (double *)malloc(sizeof(double) * (size_t)nm);
    int rc = ORC_OK;
    for (int i = 0; i < nm; i++) y[i] = Y[s[i]];
    for (int i = 0; i < nm; i++)
        for (int k = 0; k < nm; k++) {
            double dd = sqdist(X + (size_t)s[i] * p, X + (size_t)s[k] * p, p);
            double e = exp(-dd / d);
            D[i * nm + k] = dd;
            K[i * nm + k] = e + (i == k ? g : 0.0);
            K1[i * nm + k] = (dd / (d * d)) * e;
            K2[i * nm + k] = (dd * dd / (d * d * d * d) - 2.0 * dd / (d * d * d)) * e;
        }
    if (cholesky(K, nm, L) != 0 || spd_inverse(K, nm, Ki) != 0) {
        rc = ORC_ENOTPD;
    } else {
        double ldet = logdet_from_chol(L, nm);
        for (int i = 0; i < nm; i++) {
            double t = 0.0;
            for (int k = 0; k < nm; k++) t += Ki[i * nm + k] * y[k];
            a[i] = t;
        }
        double psi = 0.0;
        for (int i = 0; i < nm; i++) psi += y[i] * a[i];
        double hn = 0.5 * nm;
        out->l = lgamma(hn) - hn * log(2.0 * M_PI) - 0.5 * ldet - hn * log(psi / 2.0);
        /* A1 = K^{-1} K' */
        for (int i = 0; i < nm; i++)
            for (int k = 0; k < nm; k++) {
                double t = 0.0;
                for (int r = 0; r < nm; r++) t += Ki[i * nm + r] * K1[r * nm + k];
                A1[i * nm + k] = t;
            }
        double trA1 = 0.0, trA1A1 = 0.0, trKiK2 = 0.0;
        for (int i = 0; i < nm; i++) trA1 += A1[i * nm + i];
        for (int i = 0; i < nm; i++)
            for (int k = 0; k < nm; k++) trA1A1 += A1[i * nm + k] * A1[k * nm + i];
        for (int i = 0; i < nm; i++)
            for (int k = 0; k < nm; k++) trKiK2 += Ki[i * nm + k] * K2[k * nm + i];
        /* phi = a^T K' a ; t1 = K' a ; chi = (K'a)^T K^{-1} (K'a) ; a^T K'' a */
        double phi = 0.0, chi = 0.0, aK2a = 0.0;
        for (int i = 0; i < nm; i++) {
            double t = 0.0;
            for (int k = 0; k < nm; k++) t += K1[i * nm + k] * a[k];
            t1[i] = t;
        }
        for (int i = 0; i < nm; i++) phi += a[i] * t1[i];
        for (int i = 0; i < nm; i++)
            for (int k = 0; k < nm; k++) {
                chi += t1[i] * Ki[i * nm + k] * t1[k];
                aK2a += a[i] * K2[i * nm + k] * a[k];
            }
        out->dl = -0.5 * trA1 + hn * phi / psi;
        out->d2l = 0.5 * trA1A1 - 0.5 * trKiK2 + hn * ((aK2a - 2.0 * chi) / psi + phi * phi / (psi * psi));
        double trKi = 0.0, ata = 0.0;
        for (int i = 0; i < nm; i++) {
            trKi += Ki[i * nm + i];
            ata += a[i] * a[i];
        }
        out->dldg = -0.5 * trKi + hn * ata / psi;
        (void)D;
    }
    free(K);
    free(L);
    free(Ki);
    free(D);
    free(K1);
    free(K2);
    free(A1);
    free(a);
    free(y);
    free(t1);
    return rc;
}

int orc_llik(const double *X, const double *Y, int64_t N, int p, int64_t M,
             const int32_t *sel, const int32_t *n, int32_t nmax, const double *d,
             double g, double *llik, double *dllik, double *d2llik, int32_t *status) {
    if (N < 1 || p < 1 || M < 0 || nmax < 1 || !(g >= 0.0)) return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int64_t m = 0; m < M; m++) {
        int32_t nm = n ? n[m] : nmax;
        orc_lik r = {NAN, NAN, NAN, NAN};
        status[m] = llik_one(X, Y, p, sel + (size_t)m * nmax, nm, d[m], g, &r);
        if (llik) llik[m] = r.l;
        if (dllik) dllik[m] = r.dl;
        if (d2llik) d2llik[m] = r.d2l;
    }
    return ORC_OK;
}

/* Newton iteration on l(d) (Fig. 1 step 3).  The paper gives neither the step
 * rule nor the stopping rule; the reading taken is:
 *   proposal  d + delta with delta = -l'/l'' when l'' < 0, otherwise the
 *             sign-of-gradient step delta = +d (doubling) or -d/2 (halving);
 *   the proposal is clipped to [dmin, dmax] and delta is halved (at most 20
 *   times) until l does not decrease;
 *   stop when |d_new - d| < 1e-10 d, when no halving recovers an increase, or
 *   after max_iter iterations.  */
static int mle_one(const double *X, const double *Y, int p, const int32_t *s, int nm, double *d,
                   double g, double dmin, double dmax, int max_iter, orc_lik *res, int *iters) {
    orc_lik cur;
    int rc = llik_one(X, Y, p, s, nm, *d, g, &cur);
    int it = 0;
    while (rc == ORC_OK && it < max_iter) {
        it++;
        double delta;
        if (cur.d2l < 0.0) delta = -cur.dl / cur.d2l;
        else delta = (cur.dl > 0.0) ? *d : -0.5 * *d;
        double dn = 0.0;
        orc_lik nxt = cur;
        int accepted = 0;
        /* a short Newton step near the maximiser raises l by about
         * l'^2 / (2 |l''|), below the FP64 resolution of l there, so it is
         * taken without comparing l values; every other step must not lower
         * l, halving it at most 20 times */
        const int short_newton = cur.d2l < 0.0 && fabs(delta) <= 1e-3 * *d;
        for (int h = 0; h <= 20; h++) {
            dn = *d + delta;
            if (dn < dmin) dn = dmin;
            if (dn > dmax) dn = dmax;
            if (llik_one(X, Y, p, s, nm, dn, g, &nxt) == ORC_OK && (short_newton || nxt.l >= cur.l)) {
                accepted = 1;
                break;
            }
            delta *= 0.5;
        }
        if (!accepted) break;
        double step = fabs(dn - *d);
        *d = dn;
        cur = nxt;
        if (step < 1e-10 * *d) break;
    }
    *res = cur;
    *iters = it;
    return rc;
}

int orc_mle(const double *X, const double *Y, int64_t N, int p, int64_t M,
            const int32_t *sel, const int32_t *n, int32_t nmax, double *d, double g,
            double dmin, double dmax, int32_t max_iter, double *llik, double *dllik,
            double *d2llik, int32_t *iters, int32_t *status) {
    if (N < 1 || p < 1 || M < 0 || nmax < 1 || !(g >= 0.0) || !(dmin > 0.0) || !(dmax >= dmin) ||
        max_iter < 0)
        return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int64_t m = 0; m < M; m++) {
        int32_t nm = n ? n[m] : nmax;
        orc_lik r = {NAN, NAN, NAN, NAN};
        int it = 0;
        double dm = d[m];
        if (dm < dmin) dm = dmin;
        if (dm > dmax) dm = dmax;
        status[m] = mle_one(X, Y, p, sel + (size_t)m * nmax, nm, &dm, g, dmin, dmax, max_iter, &r,
                            &it);
        d[m] = dm;
        if (llik) llik[m] = r.l;
        if (dllik) dllik[m] = r.dl;
        if (d2llik) d2llik[m] = r.d2l;
        if (iters) iters[m] = it;
    }
    return ORC_OK;
}

/* --------------------------------------- predictive derivatives (adjoint) */

/* Differentiating Eqs. (predgp), (preds2) with t = d or g, dK/dt = Kt:
 *   d(K^{-1})/dt = -K^{-1} Kt K^{-1}
 *   mean  = kx^T K^{-1} y
 *   dmean = kx_t^T K^{-1} y - kx^T K^{-1} Kt K^{-1} y
 *   psi   = y^T K^{-1} y,         dpsi = -a^T Kt a,        a = K^{-1} y
 *   v     = 1 + g - kx^T K^{-1} kx
 *   dv    = [t==g] - 2 kx_t^T K^{-1} kx + kx^T K^{-1} Kt K^{-1} kx
 *   s2 = psi v / n,   ds2 = (dpsi v + psi dv) / n.
 * For t = d: Kt = K' (as in the likelihood), kx_t = (Dx/d^2) o kx;
 * for t = g: Kt = I, kx_t = 0. */
/* Triangular solves with the row-major lower Cholesky factor L (n x n):
 * x = L^{-1} r (forward) and x = L^{-T} r (backward). */
static void fwd_sub(const double *L, int n, const double *r, double *x) {
    for (int i = 0; i < n; i++) {
        double t = r[i];
        for (int k = 0; k < i; k++) t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
}

static void bwd_sub(const double *L, int n, const double *r, double *x) {
    for (int i = n - 1; i >= 0; i--) {
        double t = r[i];
        for (int k = i + 1; k < n; k++) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
}

/* a = K^{-1} y and b = K^{-1} kx are applied through the Cholesky factor
 * K = L L^T, and kx^T K^{-1} kx as |L^{-1} kx|^2: the explicit inverse and
 * the difference (1 + g) - kx^T b lose about eps cond(K) / v relative in v
 * (v ~ g near the design), which the g-derivative of s2 amplifies. */
static int pgrad_one(const double *X, const double *Y, int p, const double *x, const int32_t *s,
                     int nm, double d, double g, double out[5]) {
    size_t nn = (size_t)nm * nm;
    double *K = (double *)malloc(sizeof(double) * nn);
    double *Ki = (double *)malloc(sizeof(double) * nn);
    double *K1 = (double *)malloc(sizeof(double) * nn);
    double *kx = (double *)malloc(sizeof(double) * (size_t)nm);
    double *kxd = (double *)malloc(sizeof(double) * (size_t)nm);
    double *y = (double *)malloc(sizeof(double) * (size_t)nm);
    double *a = (double *)malloc(sizeof(double) * (size_t)nm);
    double *b = (double *)malloc(sizeof(double) * (size_t)nm); /* K^{-1} kx */
    int rc = ORC_OK;
    for (int i = 0; i < nm; i++) {
        y[i] = Y[s[i]];
        double dx = sqdist(x, X + (size_t)s[i] * p, p);
        kx[i] = exp(-dx / d);
        kxd[i] = (dx / (d * d)) * kx[i];
        for (int k = 0; k < nm; k++) {
            double dd = sqdist(X + (size_t)s[i] * p, X + (size_t)s[k] * p, p);
            double e = exp(-dd / d);
            K[i * nm + k] = e + (i == k ? g : 0.0);
            K1[i * nm + k] = (dd / (d * d)) * e;
        }
    }
    double *L = (double *)malloc(sizeof(double) * nn);
    double *w = (double *)malloc(sizeof(double) * (size_t)nm); /* L^{-1} kx, then L^{-1} y */
    if (cholesky(K, nm, L) != 0 || spd_inverse(K, nm, Ki) != 0) {
        rc = ORC_ENOTPD;
    } else {
        fwd_sub(L, nm, kx, w);
        double kk = 0.0;
        for (int i = 0; i < nm; i++) kk += w[i] * w[i];
        bwd_sub(L, nm, w, b);
        fwd_sub(L, nm, y, w);
        bwd_sub(L, nm, w, a);
        double psi = 0.0;
        for (int i = 0; i < nm; i++) psi += y[i] * a[i];
        double v = (1.0 + g) - kk;
        /* t = d */
        double kxd_a = 0.0, bK1a = 0.0, aK1a = 0.0, kxd_b = 0.0, bK1b = 0.0;
        for (int i = 0; i < nm; i++) {
            kxd_a += kxd[i] * a[i];
            kxd_b += kxd[i] * b[i];
            for (int k = 0; k < nm; k++) {
                bK1a += b[i] * K1[i * nm + k] * a[k];
                aK1a += a[i] * K1[i * nm + k] * a[k];
                bK1b += b[i] * K1[i * nm + k] * b[k];
            }
        }
        double dmean_dd = kxd_a - bK1a;
        double dpsi_dd = -aK1a;
        double dv_dd = -2.0 * kxd_b + bK1b;
        /* t = g */
        double ba = 0.0, aa = 0.0, bb = 0.0, trKi = 0.0;
        for (int i = 0; i < nm; i++) {
            ba += b[i] * a[i];
            aa += a[i] * a[i];
            bb += b[i] * b[i];
            trKi += Ki[i * nm + i];
        }
        double dmean_dg = -ba;
        double dpsi_dg = -aa;
        double dv_dg = 1.0 + bb;
        out[0] = dmean_dd;
        out[1] = dmean_dg;
        out[2] = (dpsi_dd * v + psi * dv_dd) / nm;
        out[3] = (dpsi_dg * v + psi * dv_dg) / nm;
        out[4] = -0.5 * trKi + 0.5 * nm * aa / psi;
    }
    free(K);
    free(Ki);
    free(K1);
    free(kx);
    free(kxd);
    free(y);
    free(a);
    free(b);
    free(L);
    free(w);
    return rc;
}

int orc_predict_grad(const double *X, const double *Y, int64_t N, int p,
                     const double *Xref, int64_t M, const int32_t *sel, const int32_t *n,
                     int32_t nmax, const double *d, double g, double *dmean_dd,
                     double *dmean_dg, double *ds2_dd, double *ds2_dg, double *dllik_dg,
                     int32_t *status) {
    if (N < 1 || p < 1 || M < 0 || nmax < 1 || !(g >= 0.0)) return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int64_t m = 0; m < M; m++) {
        int32_t nm = n ? n[m] : nmax;
        double o[5] = {NAN, NAN, NAN, NAN, NAN};
        status[m] = pgrad_one(X, Y, p, Xref + (size_t)m * p, sel + (size_t)m * nmax, nm, d[m], g, o);
        dmean_dd[m] = o[0];
        dmean_dg[m] = o[1];
        ds2_dd[m] = o[2];
        ds2_dg[m] = o[3];
        if (dllik_dg) dllik_dg[m] = o[4];
    }
    return ORC_OK;
}
