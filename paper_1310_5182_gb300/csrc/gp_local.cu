// a7 (local prediction), a8 (local Newton MLE of d) and the analytic adjoint
// of both in (d, g), on each location's selected design, all in FP64.
//
//   predict   Eqs. (predgp), (preds2): K_n = L L^T (Cholesky), z = L^{-1} Y_n,
//             w = L^{-1} k_n(x);  mean = w^T z,  psi = z^T z,
//             s2 = psi (1 + g - w^T w) / n,  df = n.
//   MLE       Eq. (gpk): l(d) = log Gamma(n/2) - (n/2) log 2pi - (1/2) log|K|
//             - (n/2) log(psi/2) with
//             l'  = -1/2 tr(K^{-1}K') + (n/2) phi/psi,  phi = a^T K' a, a = K^{-1}Y,
//             l'' = 1/2 tr(K^{-1}K'K^{-1}K') - 1/2 tr(K^{-1}K'')
//                   + (n/2) [(a^T K'' a - 2 (K'a)^T K^{-1} (K'a))/psi + phi^2/psi^2],
//             K' = (D/d^2) o E, K'' = (D^2/d^4 - 2D/d^3) o E, E = exp(-D/d);
//             Newton steps with the safeguards stated in lagp.h.
//   adjoint   d/dd and d/dg of mean and s2 through d(K^{-1}) = -K^{-1} dK K^{-1},
//             and dl/dg = -1/2 tr(K^{-1}) + (n/2) a^T a / psi.
// One CTA per location (persistent, atomic work counter); the n x n matrices
// live in a per-CTA global workspace (L2-resident), vectors in shared memory.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "exp64.cuh"
#include "lagp_internal.h"

namespace {

constexpr int GP_THREADS = 128;
constexpr int GP_WARPS = GP_THREADS / 32;

struct Blk {
    int tid, lane, warp;
};

__device__ double block_sum(double v, double *red, const Blk &b) {
    v = warp_sum(v);
    __syncthreads();
    if (b.lane == 0) red[b.warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < GP_WARPS; w++) s += red[w];
    return s;
}

// Block sums of NV values at once: warp sums, then one warp adds the warps'
// partials (not every thread); three barriers for all NV.
template <int NV>
__device__ void block_sums(double (&v)[NV], const Blk &b) {
    __shared__ double part[GP_WARPS * NV], tot[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) v[i] = warp_sum(v[i]);
    __syncthreads();  // earlier readers of part / tot are done
    if (b.lane == 0)
#pragma unroll
        for (int i = 0; i < NV; i++) part[b.warp * NV + i] = v[i];
    __syncthreads();
    if (b.warp == 0 && b.lane < NV) {
        double t = 0.0;
        for (int w = 0; w < GP_WARPS; w++) t += part[w * NV + b.lane];
        tot[b.lane] = t;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; i++) v[i] = tot[i];
}

// Lower Cholesky factor L of the symmetric n x n matrix A (lower triangle
// used), rd = 1 / diag(L), and in the same sweep the forward solves
// z_r = L^{-1} b_r of NR right-hand sides: each b_r^T is one more row of the
// factorised matrix (factorising [[A, B^T], [B, .]] gives the rows B L^{-T},
// that is z_r^T).  Left-looking by columns with one barrier per column: in
// the phase of column c every row i >= c (and every right-hand side) forms
//   s_i = A[i][c] - sum_{k<c} L[i][k] L[c][k];
// the pivot row takes L[c][c] = sqrt(s_c) and rd[c], the other rows keep s_i
// unscaled in a double buffer, and each row scales its own entry of column
// c by rd[c] in the next phase, whose sums take their term k = c from that
// buffer.  A phase therefore needs no second barrier, and no reduction: the
// pivot's sum is one lane's.  ub: 2 (n + NR) doubles of shared memory.
// Returns false (block-uniform) if a pivot is not positive.
// Entry r of a small array of pointers without indexing it at run time (no
// local-memory copy of the array).
template <int NR, typename P>
__device__ __forceinline__ P pick(P const (&v)[NR], int r) {
    P x = v[0];
#pragma unroll
    for (int q = 1; q < NR; q++)
        if (r == q) x = v[q];
    return x;
}

template <int NR>
__device__ bool block_cholesky(const double *A, double *L, double *rd, int n, int ld,
                               const double *const (&b)[NR], double *const (&z)[NR], double *ub,
                               int *flag, const Blk &bk) {
    const int rows = n + NR;
    if (bk.tid == 0) *flag = 1;
    for (int c = 0; c < n; c++) {
        const double *prev = ub + ((c + 1) & 1) * rows;  // column c - 1, unscaled
        double *cur = ub + (c & 1) * rows;
        const double rdp = c > 0 ? rd[c - 1] : 0.0;
        const double lcp = c > 0 ? prev[c] * rdp : 0.0;  // L[c][c-1]
        const double *Lc = L + (size_t)c * ld;
        for (int i = c + bk.tid; i < rows; i += GP_THREADS) {
            double *Lr = i < n ? L + (size_t)i * ld : pick(z, i - n);
            double s0 = i < n ? A[(size_t)i * ld + c] : pick(b, i - n)[c], s1 = 0.0;
            if (c > 0) {
                const double u = prev[i] * rdp;  // L[i][c-1]: scaled by its own row
                Lr[c - 1] = u;
                s0 = fma(-u, lcp, s0);
            }
            int k = 0;
            for (; k + 2 <= c - 1; k += 2) {  // two chains: half the dependent FMA latency
                s0 = fma(-Lr[k], Lc[k], s0);
                s1 = fma(-Lr[k + 1], Lc[k + 1], s1);
            }
            if (k < c - 1) s0 = fma(-Lr[k], Lc[k], s0);
            const double s = s0 + s1;
            if (i == c) {
                if (!(s > 0.0)) *flag = 0;
                const double r = s > 0.0 ? rsqrt(s) : 1.0;
                L[(size_t)c * ld + c] = s > 0.0 ? s * r : 1.0;
                rd[c] = r;
            } else {
                cur[i] = s;
            }
        }
        __syncthreads();
    }
    // the scaling of the last column: only the right-hand sides have entries
    // below its diagonal
    if (n > 0) {
        const double *last = ub + ((n - 1) & 1) * rows;
        if (bk.tid < NR) pick(z, bk.tid)[n - 1] = last[n + bk.tid] * rd[n - 1];
    }
    __syncthreads();
    return *flag != 0;
}

// x = L^{-1} rhs by forward substitution, one warp; rd = 1 / diag(L).
__device__ void warp_forward(const double *L, int ld, const double *rd, const double *rhs, double *x,
                             int n, int lane) {
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int k = lane; k < i; k += 32) s = fma(L[(size_t)i * ld + k], x[k], s);
        s = warp_sum(s);
        if (lane == 0) x[i] = (rhs[i] - s) * rd[i];
        __syncwarp();
    }
}

// x = L^{-T} rhs by backward substitution, one warp; rd = 1 / diag(L).
__device__ void warp_backward(const double *L, int ld, const double *rd, const double *rhs, double *x,
                              int n, int lane) {
    for (int i = n - 1; i >= 0; i--) {
        double s = 0.0;
        for (int k = i + 1 + lane; k < n; k += 32) s = fma(L[(size_t)k * ld + i], x[k], s);
        s = warp_sum(s);
        if (lane == 0) x[i] = (rhs[i] - s) * rd[i];
        __syncwarp();
    }
}

struct GpWork {
    double *D, *K, *L, *Li, *Ki, *A1;  // n x ld each
};

// Validate a location and load its design; returns the per-location status.
__device__ int load_design(const GpArgs &a, int64_t loc, int nm, const double *dptr, double *xd,
                           double *y, int *flag, const Blk &b) {
    if (b.tid == 0) *flag = LAGP_OK;
    __syncthreads();
    const double d = dptr ? dptr[loc] : 1.0;
    if (b.tid == 0 && (nm < 1 || nm > a.nmax || !(d > 0.0) || !isfinite(d))) *flag = LAGP_EINVAL;
    __syncthreads();
    if (*flag != LAGP_OK) return *flag;
    const int32_t *s = a.sel + loc * a.nmax;
    for (int t = b.tid; t < nm; t += GP_THREADS) {
        int32_t r = s[t];
        if (r < 0 || r >= a.N) *flag = LAGP_EINVAL;
    }
    __syncthreads();
    if (*flag != LAGP_OK) return *flag;
    for (int e = b.tid; e < nm * a.p; e += GP_THREADS) {
        int t = e / a.p, i = e - t * a.p;
        xd[e] = load_coord64(a.X, s[t], a.p, i, a.dtype);
    }
    for (int t = b.tid; t < nm; t += GP_THREADS)
        y[t] = a.dtype == LAGP_F64 ? static_cast<const double *>(a.Y)[s[t]]
                                   : (double)static_cast<const float *>(a.Y)[s[t]];
    __syncthreads();
    return LAGP_OK;
}

__device__ double sqd(const double *u, const double *v, int p) {
    double s = 0.0;
    for (int i = 0; i < p; i++) {
        double df = u[i] - v[i];
        s = fma(df, df, s);
    }
    return s;
}

// Row i and column k <= i of the e-th element of a lower triangle stored by rows.
__device__ __forceinline__ void tri_index(int e, int &i, int &k) {
    int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) r++;
    while (r * (r + 1) / 2 > e) r--;
    i = r;
    k = e - r * (r + 1) / 2;
}

// D (squared distances, lower triangle and diagonal) of the design.
__device__ void build_D(const double *xd, int nm, int p, double *D, int ld, const Blk &b) {
    for (int e = b.tid; e < nm * nm; e += GP_THREADS) {
        int i = e / nm, k = e - i * nm;
        if (k <= i) {
            double v = sqd(xd + (size_t)i * p, xd + (size_t)k * p, p);
            D[(size_t)i * ld + k] = v;
            D[(size_t)k * ld + i] = v;
        }
    }
    __syncthreads();
}

// K = exp(-D/d) + g I (full symmetric), over the lower triangle, with the
// table-driven exponential (etab: its table in shared memory).
__device__ void build_K(const double *D, int nm, int ld, double d, double g, double *K,
                        const double *etab, const Blk &b) {
    const double ninv_d = -1.0 / d;
    for (int e = b.tid; e < nm * (nm + 1) / 2; e += GP_THREADS) {
        int i, k;
        tri_index(e, i, k);
        const double v = exp64_tang(D[(size_t)i * ld + k] * ninv_d, etab) + (i == k ? g : 0.0);
        K[(size_t)i * ld + k] = v;
        K[(size_t)k * ld + i] = v;
    }
    __syncthreads();
}

// log-likelihood of Eq. (gpk) at d: needs K built; leaves L, rd and
// z = L^{-1} y (psi = y^T K^{-1} y = z^T z).  Returns false if K is not
// positive definite.
__device__ bool llik_value(const GpWork &W, int nm, int ld, const double *y, double *z, double *rd,
                           double *ub, int *flag, double *out_l, double *out_psi, const Blk &b) {
    const double *const rhs[1] = {y};
    double *const zs[1] = {z};
    if (!block_cholesky<1>(W.K, W.L, rd, nm, ld, rhs, zs, ub, flag, b)) return false;
    double v[2] = {0.0, 0.0};  // log|K|, psi
    for (int i = b.tid; i < nm; i += GP_THREADS) {
        v[0] += 2.0 * log(W.L[(size_t)i * ld + i]);
        v[1] = fma(z[i], z[i], v[1]);
    }
    block_sums<2>(v, b);
    // the constant and the logarithms on one thread (every thread evaluating
    // lgamma would hold the FP64 unit for nothing), then broadcast
    __shared__ double s_l;
    if (b.tid == 0) {
        const double hn = 0.5 * nm;
        s_l = lgamma(hn) - hn * log(2.0 * CUDART_PI) - 0.5 * v[0] - hn * log(v[1] / 2.0);
    }
    __syncthreads();
    *out_l = s_l;
    *out_psi = v[1];
    return true;
}

// K^{-1} and a = K^{-1} y from L (with rd = 1 / diag(L)) and z = L^{-1} y:
// Li = L^{-1} row by row, the columns of a row in parallel (full-lane FMAs,
// no reductions; the sums run down the rows, so that a warp's lanes read one
// row of Li at a time), then Ki = Li^T Li and a = Li^T z.
__device__ void inverse_from_L(const GpWork &W, int nm, int ld, const double *rd, const double *z,
                               double *a, const Blk &b) {
    for (int i = 0; i < nm; i++) {
        const double *Lr = W.L + (size_t)i * ld;
        // Li[i][c] = (delta_ic - sum_{k=c}^{i-1} L[i][k] Li[k][c]) / L[i][i]
        for (int c = b.tid; c <= i; c += GP_THREADS) {
            double s0 = (c == i) ? 1.0 : 0.0, s1 = 0.0;
            int k = i - 1;
            for (; k - 1 >= c; k -= 2) {
                s0 = fma(-Lr[k], W.Li[(size_t)k * ld + c], s0);
                s1 = fma(-Lr[k - 1], W.Li[(size_t)(k - 1) * ld + c], s1);
            }
            if (k >= c) s0 = fma(-Lr[k], W.Li[(size_t)k * ld + c], s0);
            W.Li[(size_t)i * ld + c] = (s0 + s1) * rd[i];
        }
        __syncthreads();
    }
    for (int e = b.tid; e < nm * (nm + 1) / 2; e += GP_THREADS) {  // lower triangle, mirrored
        int i, k;
        tri_index(e, i, k);
        double s0 = 0.0, s1 = 0.0;
        int r = i;
        for (; r + 2 <= nm; r += 2) {
            s0 = fma(W.Li[(size_t)r * ld + i], W.Li[(size_t)r * ld + k], s0);
            s1 = fma(W.Li[(size_t)(r + 1) * ld + i], W.Li[(size_t)(r + 1) * ld + k], s1);
        }
        if (r < nm) s0 = fma(W.Li[(size_t)r * ld + i], W.Li[(size_t)r * ld + k], s0);
        W.Ki[(size_t)i * ld + k] = s0 + s1;
        W.Ki[(size_t)k * ld + i] = s0 + s1;
    }
    for (int k = b.tid; k < nm; k += GP_THREADS) {  // a[k] = sum_{i >= k} Li[i][k] z[i]
        double s0 = 0.0, s1 = 0.0;
        int i = nm - 1;
        for (; i - 1 >= k; i -= 2) {
            s0 = fma(W.Li[(size_t)i * ld + k], z[i], s0);
            s1 = fma(W.Li[(size_t)(i - 1) * ld + k], z[i - 1], s1);
        }
        if (i >= k) s0 = fma(W.Li[(size_t)i * ld + k], z[i], s0);
        a[k] = s0 + s1;
    }
    __syncthreads();
}

struct Derivs {
    double dl, d2l, dldg, trKi;
};

// First and second d-derivatives of l (and dl/dg); needs K, L, rd, z = L^{-1} y
// and psi; leaves a = K^{-1} y.  The two traces with K' come from one of two
// products:
//   L_FREE (L is not needed afterwards): K' in A1's storage, C = L^{-1} K'
//     (n^3/2 FMAs) stored transposed in L's storage, and B = C L^{-T} =
//     L^{-1} K' L^{-T} (symmetric) over its lower triangle only (n^3/6),
//     column by column so that the lanes of a warp share the length of their
//     sums, never stored: tr(K^{-1} K') = tr(B), tr(K^{-1} K' K^{-1} K') =
//     |B|_F^2;
//   otherwise: K' in Li's storage once K^{-1} is built, A1 = K^{-1} K' (n^3).
// The symmetric matrices K', K'' and K^{-1} are read by columns where that
// makes a warp's loads contiguous, and the sums over them run over the lower
// triangle (off-diagonal entries twice).
template <bool L_FREE>
__device__ Derivs llik_derivs(const GpWork &W, int nm, int ld, double d, const double *z, double *a,
                              double psi, const double *rd, double *t1, double *t2, const Blk &b) {
    inverse_from_L(W, nm, ld, rd, z, a, b);
    const double id2 = 1.0 / (d * d), id3 = id2 / d, id4 = id2 * id2;
    double *Kp = L_FREE ? W.A1 : W.Li;
    for (int e = b.tid; e < nm * nm; e += GP_THREADS) {
        const int i = e / nm, k = e - i * nm;
        const double E = (i == k) ? 0.0 : W.K[(size_t)i * ld + k];
        Kp[(size_t)i * ld + k] = (W.D[(size_t)i * ld + k] * id2) * E;
    }
    __syncthreads();
    double trA1 = 0.0, trA1A1 = 0.0;
    if constexpr (L_FREE) {
        // C = L^{-1} K': C[i][k] = sum_{m <= i} Li[i][m] K'[m][k], into Ct[k][i]
        double *Ct = W.L;
        for (int e = b.tid; e < nm * nm; e += GP_THREADS) {
            const int i = e / nm, k = e - i * nm;
            const double *Lir = W.Li + (size_t)i * ld;
            double s0 = 0.0, s1 = 0.0;
            int m = 0;
            for (; m + 2 <= i + 1; m += 2) {
                s0 = fma(Lir[m], Kp[(size_t)m * ld + k], s0);
                s1 = fma(Lir[m + 1], Kp[(size_t)(m + 1) * ld + k], s1);
            }
            if (m <= i) s0 = fma(Lir[m], Kp[(size_t)m * ld + k], s0);
            Ct[(size_t)k * ld + i] = s0 + s1;
        }
        __syncthreads();
        // B[i][j] = sum_{k <= j} C[i][k] Li[j][k] for i >= j, by columns j (from
        // the last) and rows i (from the last) within a column
        for (int e = b.tid; e < nm * (nm + 1) / 2; e += GP_THREADS) {
            int r, q;
            tri_index(e, r, q);
            const int j = nm - 1 - r, i = nm - 1 - q;
            const double *Lj = W.Li + (size_t)j * ld;
            double s0 = 0.0, s1 = 0.0;
            int k = 0;
            for (; k + 2 <= j + 1; k += 2) {
                s0 = fma(Ct[(size_t)k * ld + i], Lj[k], s0);
                s1 = fma(Ct[(size_t)(k + 1) * ld + i], Lj[k + 1], s1);
            }
            if (k <= j) s0 = fma(Ct[(size_t)k * ld + i], Lj[k], s0);
            const double Bij = s0 + s1;
            if (i == j) {
                trA1 += Bij;
                trA1A1 = fma(Bij, Bij, trA1A1);
            } else {
                trA1A1 = fma(2.0 * Bij, Bij, trA1A1);
            }
        }
    } else {
        // A1 = K^{-1} K' (two accumulation chains per element)
        for (int e = b.tid; e < nm * nm; e += GP_THREADS) {
            const int i = e / nm, k = e - i * nm;
            const double *Kir = W.Ki + (size_t)i * ld;
            double s0 = 0.0, s1 = 0.0;
            int r = 0;
            for (; r + 2 <= nm; r += 2) {
                s0 = fma(Kir[r], Kp[(size_t)r * ld + k], s0);
                s1 = fma(Kir[r + 1], Kp[(size_t)(r + 1) * ld + k], s1);
            }
            if (r < nm) s0 = fma(Kir[r], Kp[(size_t)r * ld + k], s0);
            W.A1[(size_t)i * ld + k] = s0 + s1;
        }
    }
    // t1 = K' a (K' symmetric: read by columns)
    for (int i = b.tid; i < nm; i += GP_THREADS) {
        double s0 = 0.0, s1 = 0.0;
        int k = 0;
        for (; k + 2 <= nm; k += 2) {
            s0 = fma(Kp[(size_t)k * ld + i], a[k], s0);
            s1 = fma(Kp[(size_t)(k + 1) * ld + i], a[k + 1], s1);
        }
        if (k < nm) s0 = fma(Kp[(size_t)k * ld + i], a[k], s0);
        t1[i] = s0 + s1;
    }
    __syncthreads();
    // the lower triangle of K'' = (D^2/d^4 - 2D/d^3) o E with its off-diagonal
    // entries doubled (exact scalings by 2; its diagonal is zero)
    const double id4x2 = 2.0 * id4, id3x4 = 4.0 * id3;
    double trKiK2 = 0.0, aK2a = 0.0, trKi = 0.0, ata = 0.0;
    for (int e = b.tid; e < nm * (nm + 1) / 2; e += GP_THREADS) {
        int i, k;
        tri_index(e, i, k);
        if (i == k) {
            if (!L_FREE) trA1 += W.A1[(size_t)i * ld + i];
            if (!L_FREE) trA1A1 = fma(W.A1[(size_t)i * ld + i], W.A1[(size_t)i * ld + i], trA1A1);
            trKi += W.Ki[(size_t)i * ld + i];
            ata = fma(a[i], a[i], ata);
            continue;
        }
        if (!L_FREE) trA1A1 = fma(2.0 * W.A1[(size_t)i * ld + k], W.A1[(size_t)k * ld + i], trA1A1);
        const double Dik = W.D[(size_t)i * ld + k];
        const double K2w = (Dik * Dik * id4x2 - Dik * id3x4) * W.K[(size_t)i * ld + k];
        trKiK2 = fma(W.Ki[(size_t)i * ld + k], K2w, trKiK2);
        aK2a = fma(a[i] * K2w, a[k], aK2a);
    }
    // t2 = K^{-1} t1 (K^{-1} symmetric: read by columns)
    for (int i = b.tid; i < nm; i += GP_THREADS) {
        double s0 = 0.0, s1 = 0.0;
        int k = 0;
        for (; k + 2 <= nm; k += 2) {
            s0 = fma(W.Ki[(size_t)k * ld + i], t1[k], s0);
            s1 = fma(W.Ki[(size_t)(k + 1) * ld + i], t1[k + 1], s1);
        }
        if (k < nm) s0 = fma(W.Ki[(size_t)k * ld + i], t1[k], s0);
        t2[i] = s0 + s1;
    }
    __syncthreads();
    double phi_p = 0.0, chi_p = 0.0;
    for (int i = b.tid; i < nm; i += GP_THREADS) {
        phi_p = fma(a[i], t1[i], phi_p);
        chi_p = fma(t1[i], t2[i], chi_p);
    }
    double sums[8] = {trA1, trA1A1, trKiK2, aK2a, trKi, ata, phi_p, chi_p};
    block_sums<8>(sums, b);
    trA1 = sums[0];
    trA1A1 = sums[1];
    trKiK2 = sums[2];
    aK2a = sums[3];
    trKi = sums[4];
    ata = sums[5];
    const double phi = sums[6], chi = sums[7];
    // the scalars on one thread (divisions hold the FP64 unit), then broadcast
    __shared__ Derivs s_r;
    if (b.tid == 0) {
        const double hn = 0.5 * nm, ipsi = 1.0 / psi;
        s_r.dl = -0.5 * trA1 + hn * phi * ipsi;
        s_r.d2l = 0.5 * trA1A1 - 0.5 * trKiK2 + hn * ((aK2a - 2.0 * chi) * ipsi + phi * phi * (ipsi * ipsi));
        s_r.dldg = -0.5 * trKi + hn * ata * ipsi;
        s_r.trKi = trKi;
    }
    __syncthreads();
    return s_r;
}

struct GpShared {
    double *xd, *y, *a, *t1, *t2, *t3, *kx, *dx, *rd, *xq, *etab, *ub;
};

__device__ GpShared carve(unsigned char *raw, int nmax, int p) {
    GpShared S;
    double *base = reinterpret_cast<double *>(raw);
    S.xd = base;
    S.y = S.xd + (size_t)nmax * p;
    S.a = S.y + nmax;
    S.t1 = S.a + nmax;
    S.t2 = S.t1 + nmax;
    S.t3 = S.t2 + nmax;
    S.kx = S.t3 + nmax;
    S.dx = S.kx + nmax;
    S.rd = S.dx + nmax;  // 1 / diag of the current Cholesky factor
    S.xq = S.rd + nmax;
    S.etab = S.xq + p;  // EXP64_TABLE_SIZE: table of exp64_tang
    S.ub = S.etab + EXP64_TABLE_SIZE;  // 2 (nmax + 2): the Cholesky's column buffers
    return S;
}

__device__ GpWork work_for_block(double *ws, int nmax, int ld) {
    const size_t mat = (size_t)nmax * ld;
    double *w = ws + (size_t)blockIdx.x * 6 * mat;
    return GpWork{w, w + mat, w + 2 * mat, w + 3 * mat, w + 4 * mat, w + 5 * mat};
}

// ------------------------------------------------------------------ predict

__global__ void __launch_bounds__(GP_THREADS)
predict_kernel(GpArgs a, const double *__restrict__ dv, int *counter, double *ws, double *mean,
               double *s2, double *df, int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, ld = (nmax + 31) & ~31;
    GpShared S = carve(smem_raw, nmax, p);
    for (int i = threadIdx.x; i < EXP64_TABLE_SIZE; i += GP_THREADS) S.etab[i] = exp64_table_g[i];  // ordered by the loop's first barrier
    GpWork W = work_for_block(ws, nmax, ld);
    __shared__ int s_loc, s_flag, s_chol;
    Blk b{(int)threadIdx.x, (int)threadIdx.x & 31, (int)threadIdx.x >> 5};
    for (;;) {
        if (b.tid == 0) s_loc = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t loc = s_loc;
        __syncthreads();
        if (loc >= a.M) break;
        const int nm = a.n ? a.n[loc] : nmax;
        int st = load_design(a, loc, nm, dv, S.xd, S.y, &s_flag, b);
        double mu = CUDART_NAN, sv = CUDART_NAN, dfv = CUDART_NAN;
        if (st == LAGP_OK) {
            const double d = dv[loc], g = a.g;
            for (int i = b.tid; i < p; i += GP_THREADS) S.xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
            build_D(S.xd, nm, p, W.D, ld, b);
            build_K(W.D, nm, ld, d, g, W.K, S.etab, b);
            for (int t = b.tid; t < nm; t += GP_THREADS) S.kx[t] = exp(-sqd(S.xq, S.xd + (size_t)t * p, p) / d);
            __syncthreads();
            // z = L^{-1} Y_n (t1) and w = L^{-1} k_n(x) (t2) with the factorisation
            const double *const rhs[2] = {S.y, S.kx};
            double *const sol[2] = {S.t1, S.t2};
            if (!block_cholesky<2>(W.K, W.L, S.rd, nm, ld, rhs, sol, S.ub, &s_chol, b)) {
                st = LAGP_ENOTPD;
            } else {
                double m_p = 0.0, psi_p = 0.0, kk_p = 0.0;
                for (int i = b.tid; i < nm; i += GP_THREADS) {
                    m_p = fma(S.t2[i], S.t1[i], m_p);
                    psi_p = fma(S.t1[i], S.t1[i], psi_p);
                    kk_p = fma(S.t2[i], S.t2[i], kk_p);
                }
                double v[3] = {m_p, psi_p, kk_p};
                block_sums<3>(v, b);
                mu = v[0];
                const double psi = v[1], kk = v[2];
                sv = psi * ((1.0 + g) - kk) / nm;
                dfv = nm;
            }
        }
        if (b.tid == 0) {
            mean[loc] = mu;
            s2[loc] = sv;
            df[loc] = dfv;
            status[loc] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------- MLE

struct MleOut {
    double *llik, *dllik, *d2llik;
    int32_t *iters, *status;
};

__global__ void __launch_bounds__(GP_THREADS, 6)
mle_kernel(GpArgs a, double *dv, double dmin, double dmax, int max_iter, int *counter, double *ws,
           MleOut o, unsigned long long *work) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, ld = (nmax + 31) & ~31;
    GpShared S = carve(smem_raw, nmax, p);
    for (int i = threadIdx.x; i < EXP64_TABLE_SIZE; i += GP_THREADS) S.etab[i] = exp64_table_g[i];  // ordered by the loop's first barrier
    GpWork W = work_for_block(ws, nmax, ld);
    __shared__ int s_loc, s_flag, s_chol;
    Blk b{(int)threadIdx.x, (int)threadIdx.x & 31, (int)threadIdx.x >> 5};
    unsigned long long n_llik = 0, n_derivs = 0;  // evaluations x n^3 (thread 0's count)
    for (;;) {
        if (b.tid == 0) s_loc = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t loc = s_loc;
        __syncthreads();
        if (loc >= a.M) break;
        const int nm = a.n ? a.n[loc] : nmax;
        int st = load_design(a, loc, nm, dv, S.xd, S.y, &s_flag, b);
        const unsigned long long n3 = (unsigned long long)nm * nm * nm;
        double l = CUDART_NAN, psi = 0.0;
        Derivs dr{CUDART_NAN, CUDART_NAN, CUDART_NAN, CUDART_NAN};
        int it = 0;
        double d = dv[loc];
        if (st == LAGP_OK) {
            const double g = a.g;
            d = fmin(fmax(d, dmin), dmax);
            build_D(S.xd, nm, p, W.D, ld, b);
            build_K(W.D, nm, ld, d, g, W.K, S.etab, b);
            n_llik += n3;
            if (!llik_value(W, nm, ld, S.y, S.t3, S.rd, S.ub, &s_chol, &l, &psi, b)) {
                st = LAGP_ENOTPD;
            } else {
                dr = llik_derivs<true>(W, nm, ld, d, S.t3, S.a, psi, S.rd, S.t1, S.t2, b);
                n_derivs += n3;
                while (it < max_iter) {
                    it++;
                    double delta;
                    if (dr.d2l < 0.0) delta = -dr.dl / dr.d2l;
                    else delta = (dr.dl > 0.0) ? d : -0.5 * d;
                    bool accepted = false;
                    double dn = d, ln = l, psin = psi;
                    // a short Newton step near the maximiser raises l below the
                    // FP64 resolution of l: taken without comparing l values
                    const bool short_newton = dr.d2l < 0.0 && fabs(delta) <= 1e-3 * d;
                    for (int h = 0; h <= 20; h++) {
                        dn = fmin(fmax(d + delta, dmin), dmax);
                        build_K(W.D, nm, ld, dn, g, W.K, S.etab, b);
                        n_llik += n3;
                        if (llik_value(W, nm, ld, S.y, S.t3, S.rd, S.ub, &s_chol, &ln, &psin, b) &&
                            (short_newton || ln >= l)) {
                            accepted = true;
                            break;
                        }
                        delta *= 0.5;
                    }
                    if (!accepted) {
                        // restore K, L, a at the current d
                        build_K(W.D, nm, ld, d, g, W.K, S.etab, b);
                        llik_value(W, nm, ld, S.y, S.t3, S.rd, S.ub, &s_chol, &l, &psi, b);
                        n_llik += n3;
                        break;
                    }
                    const double step = fabs(dn - d);
                    d = dn;
                    l = ln;
                    psi = psin;
                    dr = llik_derivs<true>(W, nm, ld, d, S.t3, S.a, psi, S.rd, S.t1, S.t2, b);
                    n_derivs += n3;
                    if (step < 1e-10 * d) break;
                }
            }
        }
        if (b.tid == 0) {
            if (st == LAGP_OK) dv[loc] = d;
            if (o.llik) o.llik[loc] = st == LAGP_OK ? l : CUDART_NAN;
            if (o.dllik) o.dllik[loc] = st == LAGP_OK ? dr.dl : CUDART_NAN;
            if (o.d2llik) o.d2llik[loc] = st == LAGP_OK ? dr.d2l : CUDART_NAN;
            if (o.iters) o.iters[loc] = it;
            o.status[loc] = st;
        }
        __syncthreads();
    }
    if (b.tid == 0 && work) {
        atomicAdd(work, n_llik);
        atomicAdd(work + 1, n_derivs);
    }
}

// ------------------------------------------------------------------ adjoint

struct GradOut {
    double *dmean_dd, *dmean_dg, *ds2_dd, *ds2_dg, *dllik_dd, *dllik_dg;
    int32_t *status;
};

__global__ void __launch_bounds__(GP_THREADS)
grad_kernel(GpArgs a, const double *__restrict__ dv, int *counter, double *ws, GradOut o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, ld = (nmax + 31) & ~31;
    GpShared S = carve(smem_raw, nmax, p);
    for (int i = threadIdx.x; i < EXP64_TABLE_SIZE; i += GP_THREADS) S.etab[i] = exp64_table_g[i];  // ordered by the loop's first barrier
    GpWork W = work_for_block(ws, nmax, ld);
    __shared__ int s_loc, s_flag, s_chol;
    __shared__ double red[GP_WARPS];
    Blk b{(int)threadIdx.x, (int)threadIdx.x & 31, (int)threadIdx.x >> 5};
    for (;;) {
        if (b.tid == 0) s_loc = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t loc = s_loc;
        __syncthreads();
        if (loc >= a.M) break;
        const int nm = a.n ? a.n[loc] : nmax;
        int st = load_design(a, loc, nm, dv, S.xd, S.y, &s_flag, b);
        double r[6] = {CUDART_NAN, CUDART_NAN, CUDART_NAN, CUDART_NAN, CUDART_NAN, CUDART_NAN};
        if (st == LAGP_OK) {
            const double d = dv[loc], g = a.g, d2 = d * d;
            for (int i = b.tid; i < p; i += GP_THREADS) S.xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
            build_D(S.xd, nm, p, W.D, ld, b);
            build_K(W.D, nm, ld, d, g, W.K, S.etab, b);
            double l, psi;
            if (!llik_value(W, nm, ld, S.y, S.t3, S.rd, S.ub, &s_chol, &l, &psi, b)) {
                st = LAGP_ENOTPD;
            } else {
                Derivs dr = llik_derivs<false>(W, nm, ld, d, S.t3, S.a, psi, S.rd, S.t1, S.t2, b);
                // kx, kx_d = (Dx/d^2) kx ; b = K^{-1} kx (t1) by the two triangular
                // solves (w = L^{-1} kx in t3, v = 1 + g - w^T w: no explicit
                // inverse, no cancellation against k^T b), K'a (t2), K'b (t3)
                const double id2 = 1.0 / d2;
                for (int t = b.tid; t < nm; t += GP_THREADS) {
                    S.dx[t] = sqd(S.xq, S.xd + (size_t)t * p, p);
                    S.kx[t] = exp(-S.dx[t] / d);
                }
                __syncthreads();
                if (b.warp == 0) {
                    warp_forward(W.L, ld, S.rd, S.kx, S.t3, nm, b.lane);
                    warp_backward(W.L, ld, S.rd, S.t3, S.t1, nm, b.lane);
                }
                __syncthreads();
                double ww_p = 0.0;
                for (int i = b.tid; i < nm; i += GP_THREADS) ww_p = fma(S.t3[i], S.t3[i], ww_p);
                const double ww = block_sum(ww_p, red, b);
                for (int i = b.tid; i < nm; i += GP_THREADS) {
                    double sa = 0.0, sb = 0.0;
                    for (int k = 0; k < nm; k++) {
                        double E = (i == k) ? 0.0 : W.K[(size_t)i * ld + k];
                        double K1 = (W.D[(size_t)i * ld + k] * id2) * E;
                        sa = fma(K1, S.a[k], sa);
                        sb = fma(K1, S.t1[k], sb);
                    }
                    S.t2[i] = sa;
                    S.t3[i] = sb;
                }
                __syncthreads();
                double kxd_a = 0, bK1a = 0, aK1a = 0, kxd_b = 0, bK1b = 0, ba = 0, aa = 0, bb = 0;
                for (int i = b.tid; i < nm; i += GP_THREADS) {
                    const double kxi = S.kx[i];
                    const double kxdi = (S.dx[i] * id2) * kxi;
                    kxd_a = fma(kxdi, S.a[i], kxd_a);
                    kxd_b = fma(kxdi, S.t1[i], kxd_b);
                    bK1a = fma(S.t1[i], S.t2[i], bK1a);
                    aK1a = fma(S.a[i], S.t2[i], aK1a);
                    bK1b = fma(S.t1[i], S.t3[i], bK1b);
                    ba = fma(S.t1[i], S.a[i], ba);
                    aa = fma(S.a[i], S.a[i], aa);
                    bb = fma(S.t1[i], S.t1[i], bb);
                }
                kxd_a = block_sum(kxd_a, red, b);
                kxd_b = block_sum(kxd_b, red, b);
                bK1a = block_sum(bK1a, red, b);
                aK1a = block_sum(aK1a, red, b);
                bK1b = block_sum(bK1b, red, b);
                ba = block_sum(ba, red, b);
                aa = block_sum(aa, red, b);
                bb = block_sum(bb, red, b);
                const double v = (1.0 + g) - ww;  // = 1 + g - k^T K^{-1} k
                r[0] = kxd_a - bK1a;
                r[1] = -ba;
                r[2] = (-aK1a * v + psi * (-2.0 * kxd_b + bK1b)) / nm;
                r[3] = (-aa * v + psi * (1.0 + bb)) / nm;
                r[4] = dr.dl;
                r[5] = dr.dldg;
            }
        }
        if (b.tid == 0) {
            if (o.dmean_dd) o.dmean_dd[loc] = r[0];
            if (o.dmean_dg) o.dmean_dg[loc] = r[1];
            if (o.ds2_dd) o.ds2_dd[loc] = r[2];
            if (o.ds2_dg) o.ds2_dg[loc] = r[3];
            if (o.dllik_dd) o.dllik_dd[loc] = r[4];
            if (o.dllik_dg) o.dllik_dg[loc] = r[5];
            o.status[loc] = st;
        }
        __syncthreads();
    }
}

struct GpLaunch {
    int grid;
    size_t smem;
    double *ws;
    int *counter;
};

template <typename Kern>
lagp_status prepare(lagp_ctx *ctx, const GpArgs &a, Kern kern, GpLaunch &L) {
    const int ld = (a.nmax + 31) & ~31;
    L.smem = ((size_t)a.nmax * a.p + (size_t)a.nmax * 10 + (size_t)a.p + EXP64_TABLE_SIZE + 4) * 8 + 64;
    if (L.smem > ctx->smem_optin) return lagp_fail(ctx, LAGP_EINVAL, "n_max x p too large");
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, GP_THREADS, L.smem);
    const int per_sm = occ > 0 ? occ : 1;  // latency-bound FP64 phases: as many CTAs as fit
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    if (grid > a.M) grid = a.M;
    if (grid < 1) grid = 1;
    L.grid = (int)grid;
    L.ws = static_cast<double *>(lagp_ws(ctx, WS_GP_MAT, (size_t)grid * 6 * a.nmax * ld * 8 + 256));
    L.counter = static_cast<int *>(lagp_ws(ctx, WS_ALC_COUNTER, 256));
    if (!L.ws || !L.counter) return LAGP_ENOMEM;
    LAGP_CUDA(ctx, cudaMemsetAsync(L.counter + 1, 0, sizeof(int), ctx->stream));
    L.counter += 1;  // its own counter word
    return LAGP_OK;
}

}  // namespace

lagp_status launch_predict(lagp_ctx *ctx, const GpArgs &a, const double *d, double *mean,
                           double *s2, double *df, int32_t *status) {
    GpLaunch L;
    LAGP_TRY(prepare(ctx, a, predict_kernel, L));
    predict_kernel<<<L.grid, GP_THREADS, L.smem, ctx->stream>>>(a, d, L.counter, L.ws, mean, s2, df, status);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

lagp_status launch_mle(lagp_ctx *ctx, const GpArgs &a, double *d, double dmin, double dmax,
                       int32_t max_iter, double *llik, double *dllik, double *d2llik,
                       int32_t *iters, int32_t *status) {
    GpLaunch L;
    LAGP_TRY(prepare(ctx, a, mle_kernel, L));
    MleOut o{llik, dllik, d2llik, iters, status};
    int *ac = nullptr;
    unsigned long long *aw = nullptr;
    LAGP_TRY(alc_counters(ctx, &ac, &aw));  // (the MLE's words follow the ALC's)
    mle_kernel<<<L.grid, GP_THREADS, L.smem, ctx->stream>>>(a, d, dmin, dmax, max_iter, L.counter, L.ws, o,
                                                            aw + 8);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

lagp_status launch_predict_grad(lagp_ctx *ctx, const GpArgs &a, const double *d,
                                double *dmean_dd, double *dmean_dg, double *ds2_dd,
                                double *ds2_dg, double *dllik_dd, double *dllik_dg,
                                int32_t *status) {
    GpLaunch L;
    LAGP_TRY(prepare(ctx, a, grad_kernel, L));
    GradOut o{dmean_dd, dmean_dg, ds2_dd, ds2_dg, dllik_dd, dllik_dg, status};
    grad_kernel<<<L.grid, GP_THREADS, L.smem, ctx->stream>>>(a, d, L.counter, L.ws, o);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
