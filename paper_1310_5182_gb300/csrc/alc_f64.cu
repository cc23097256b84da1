// a2..a6, plain FP64 form: greedy ALC local design search (Fig. 1 step 2 of
// the paper) with every candidate's criterion evaluated by Eq. (dxy) in FP64.
//
// Layout: one persistent CTA works on one location at a time (locations are
// taken from an atomic counter).  Shared memory holds K_j^{-1} (FP64, leading
// dimension n_max) and the design's k_j(x); a per-CTA global panel holds
// K(x_c, x_i) for every candidate c and design row i, one column appended per
// step (the paper rebuilds these covariances every step; appending gives the
// same values for N' exponentials per step instead of N' j).
//
// Per step j, one warp per candidate (lane t owns design index t, t+32, ...):
//   b   = K_j^{-1} k_j(x_c)                 (the O(j^2) contraction, paper step 3)
//   m^-1 = 1 + g - k_j(x_c)^T b,  k_j(x)^T g_j = -m k_j(x)^T b   (steps 4-5, 7)
//   Delta = (k^T g)^2 m^-1 + 2 (k^T g) K(x_c,x) + K(x_c,x)^2 m      (Eq. dxy, step 8)
// then a block argmax (ties to the lower design row) and the partitioned
// inverse update of Sec. 2.2.  GB300 runs FP64 at 1/62 of the FP32 rate, so
// this form is bound by the FP64 pipe; it is the plain reference form.
//
// Few locations (at least two resident CTAs a location, as on the
// 100-location 2-d toy): one location per thread-block cluster of CS CTAs
// instead (CS up to 4, not necessarily a power of two).  CTA r of the
// cluster scores, and appends panel columns for, the candidates c with
// c mod CS = r; each step the CTAs exchange their best through distributed
// shared memory (one cluster barrier a step, the records double-buffered by
// the step's parity) and every CTA applies the same partitioned-inverse
// update to its own copy of K^{-1}, reading the winner's panel row from its
// owner's global panel after the barrier: the copies stay identical bit for
// bit, and so do the results whatever CS is.
#include <algorithm>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "lagp_internal.h"

namespace {

constexpr int F64_THREADS = 256;
constexpr int F64_WARPS = F64_THREADS / 32;
constexpr int NMAX_SMEM = 128;

struct F64Shared {
    double *Kinv;    // nmax x nmax
    double *kx;      // nmax: k_j(x)
    double *yd;      // nmax: responses of the design (fused prediction)
    double *alpha;   // nmax: K^{-1} Y_j (fused prediction)
    double *bstar;   // nmax: K^{-1} k*
    double *part;    // 4 x ld: partial sums of K^{-1} k*
    double *xd;      // nmax x p: design coordinates
    double *xq;      // p: reference location
    unsigned char *chosen;  // Npmax
};

// Contraction for one candidate (paper steps 3-4 and the k_j(x) dot product
// of step 7): lane t accumulates b_t = sum_k K^{-1}[k][t] kc[k] for its
// columns t = lane + 32 r, r < JQ; returns warp-uniform kc^T b and kx^T b.
// K^{-1} rows have leading dimension ld (a multiple of 32), so every read is
// inside the row; columns >= j are masked out of the sums.
template <int JQ>
__device__ __forceinline__ void contract_cand(const double *__restrict__ prow, const double *Kinv,
                                              int ld, const double *kx, int j, int lane,
                                              double &quad, double &kxb) {
    double kc[JQ], b[JQ];
#pragma unroll
    for (int r = 0; r < JQ; r++) {
        kc[r] = (lane + 32 * r < j) ? prow[lane + 32 * r] : 0.0;
        b[r] = 0.0;
    }
#pragma unroll
    for (int r = 0; r < JQ; r++) {
        const int kend = min(32, j - 32 * r);
        for (int kk = 0; kk < kend; kk++) {
            const double v = __shfl_sync(LAGP_FULL_MASK, kc[r], kk);
            const double *row = Kinv + (size_t)(32 * r + kk) * ld + lane;
#pragma unroll
            for (int r2 = 0; r2 < JQ; r2++) b[r2] = fma(row[32 * r2], v, b[r2]);
        }
    }
    double q = 0.0, x = 0.0;
#pragma unroll
    for (int r = 0; r < JQ; r++)
        if (lane + 32 * r < j) {
            q = fma(kc[r], b[r], q);
            x = fma(kx[lane + 32 * r], b[r], x);
        }
    quad = warp_sum(q);
    kxb = warp_sum(x);
}

__device__ __forceinline__ double kern64(const double *a, const void *X, int64_t r, int p,
                                         lagp_dtype dt, double d) {
    double s = 0.0;
    for (int i = 0; i < p; i++) {
        double diff = a[i] - load_coord64(X, r, p, i, dt);
        s += diff * diff;
    }
    return exp(-s / d);
}

namespace cg = cooperative_groups;

// CL: one location per cluster (candidates split over its CTAs)
template <bool CL>
__global__ void __launch_bounds__(F64_THREADS)
alc_f64_kernel(AlcArgs a, int *__restrict__ counter, double *__restrict__ panel_ws,
               double *__restrict__ kappa_ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, Npmax = a.Npmax;
    const int ld = (nmax + 31) & ~31;  // K^{-1} leading dimension
    F64Shared S;
    S.Kinv = reinterpret_cast<double *>(smem_raw);
    S.kx = S.Kinv + (size_t)(nmax + 1) * ld;
    S.yd = S.kx + ld;
    S.alpha = S.yd + ld;
    S.bstar = S.alpha + ld;
    S.part = S.bstar + nmax;
    S.xd = S.part + 4 * (size_t)ld;
    S.xq = S.xd + (size_t)nmax * p;
    S.chosen = reinterpret_cast<unsigned char *>(S.xq + p);
    __shared__ int s_loc, s_bad, s_cstar;
    __shared__ double w_v[F64_WARPS];
    __shared__ int w_row[F64_WARPS], w_slot[F64_WARPS];
    __shared__ double s_delta, s_mu, s_ry, s_cx, s_psi, s_qx, s_ystar;
    // the cluster's exchange of the step's best (by the step's parity)
    __shared__ double x_v[2];
    __shared__ int x_row[2], x_slot[2], x_bad[2];
    const bool fused = a.mean != nullptr;

    double *panel = panel_ws + (size_t)blockIdx.x * Npmax * nmax;  // [c][i], ld nmax
    double *kappa = kappa_ws + (size_t)blockIdx.x * Npmax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // cluster rank and size (1 and 0 without clusters); candidates c with
    // c mod CS = rank are this CTA's
    const int CS = CL ? (int)cg::this_cluster().num_blocks() : 1;
    const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
    int64_t next_loc = CL ? blockIdx.x / CS : 0;

    for (;;) {
        int64_t loc;
        if constexpr (CL) {
            loc = next_loc;  // a static share of the locations per cluster
            next_loc += gridDim.x / CS;
        } else {
            if (tid == 0) s_loc = atomicAdd(counter, 1);
            __syncthreads();
            loc = s_loc;
            __syncthreads();
        }
        if (loc >= a.M) break;

        const int k = a.Np ? a.Np[loc] : Npmax;
        const int nm = a.n ? a.n[loc] : nmax;
        const double d = a.d[loc], g = a.g;
        const int32_t *cands = a.idx + loc * Npmax;
        int32_t *sel = a.sel + loc * nmax;
        double *alc = a.alc ? a.alc + loc * nmax : nullptr;

        // per-location validation
        if (tid == 0) s_bad = (k < 1 || k > Npmax || nm < a.n0 || nm > nmax || nm > k || !(d > 0.0) ||
                               !isfinite(d)) ? LAGP_EINVAL : LAGP_OK;
        __syncthreads();
        if (s_bad == LAGP_OK)
            for (int c = tid; c < k; c += F64_THREADS) {
                int32_t r = cands[c];
                if (r < 0 || r >= a.N) s_bad = LAGP_EINVAL;
            }
        __syncthreads();
        // (outputs: the cluster's rank 0 alone writes them)
        if (rank == 0)
            for (int t = tid; t < nmax; t += F64_THREADS) {
                sel[t] = -1;
                if (alc) alc[t] = CUDART_NAN;
            }
        if (s_bad != LAGP_OK) {
            if (tid == 0 && rank == 0) {
                a.status[loc] = s_bad;
                if (fused) a.mean[loc] = a.s2[loc] = a.df[loc] = CUDART_NAN;
            }
            __syncthreads();
            continue;  // next location
        }

        // reference location, chosen flags, K(x_c, x) for every candidate
        for (int i = tid; i < p; i += F64_THREADS) S.xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
        for (int c = tid; c < k; c += F64_THREADS) S.chosen[c] = 0;
        __syncthreads();
        for (int c = tid; c < k; c += F64_THREADS) kappa[c] = kern64(S.xq, a.X, cands[c], p, a.dtype, d);
        __syncthreads();

        int status = LAGP_OK;
        if (tid == 0) s_psi = s_qx = 0.0;
        for (int j = 0; j < nm; j++) {
            int cstar;
            double delta = CUDART_NAN;
            if (j < a.n0) {
                cstar = j;  // Fig. 1 step 2(a): the nearest neighbours, in order
                // (the owner's panel row of the seed is read after the barrier)
                if constexpr (CL) cg::this_cluster().sync();
            } else {
                // ---- score every unchosen candidate (this CTA's share), one
                // warp per candidate
                ArgBest best{0.0, -1, -1};
                for (int c = rank + CS * warp; c < k; c += CS * F64_WARPS) {
                    if (S.chosen[c]) continue;
                    const double *prow = panel + (size_t)c * nmax;
                    double quad, kxb;
                    switch ((j + 31) >> 5) {
                        case 1: contract_cand<1>(prow, S.Kinv, ld, S.kx, j, lane, quad, kxb); break;
                        case 2: contract_cand<2>(prow, S.Kinv, ld, S.kx, j, lane, quad, kxb); break;
                        case 3: contract_cand<3>(prow, S.Kinv, ld, S.kx, j, lane, quad, kxb); break;
                        default: contract_cand<4>(prow, S.Kinv, ld, S.kx, j, lane, quad, kxb); break;
                    }
                    const double minv = (1.0 + g) - quad;  // m_j^{-1}(x_c), Eq. (piedef)
                    const double m = 1.0 / minv;
                    const double kxg = -m * kxb;           // k_j(x)^T g_j(x_c)
                    const double kap = kappa[c];
                    double dl = kxg * kxg * minv + 2.0 * kxg * kap + kap * kap * m;
                    if (!(minv > 0.0)) dl = -CUDART_INF;  // breakdown, flagged below
                    if (!(minv > 0.0) && lane == 0) s_bad = LAGP_ENOTPD;
                    if (better(dl, cands[c], best.v, best.row)) best = ArgBest{dl, cands[c], c};
                }
                if (lane == 0) {
                    w_v[warp] = best.v;
                    w_row[warp] = best.row;
                    w_slot[warp] = best.slot;
                }
                __syncthreads();
                if (tid == 0) {
                    ArgBest b0{w_v[0], w_row[0], w_slot[0]};
                    for (int w = 1; w < F64_WARPS; w++)
                        if (better(w_v[w], w_row[w], b0.v, b0.row)) b0 = ArgBest{w_v[w], w_row[w], w_slot[w]};
                    s_cstar = b0.slot;
                    s_delta = b0.v;
                    if constexpr (CL) {
                        x_v[j & 1] = b0.v;
                        x_row[j & 1] = b0.row;
                        x_slot[j & 1] = b0.slot;
                        x_bad[j & 1] = s_bad;
                    } else if (b0.slot < 0) {
                        s_bad = LAGP_ENOTPD;
                    }
                }
                if constexpr (CL) {
                    // the cluster's best (ties to the lower row), the same in every CTA
                    cg::cluster_group cl = cg::this_cluster();
                    cl.sync();
                    if (tid == 0) {
                        ArgBest b0{-CUDART_INF, INT32_MAX, -1};
                        int bad = LAGP_OK;
                        for (int r = 0; r < CS; r++) {
                            const double v = *cl.map_shared_rank(&x_v[j & 1], r);
                            const int row = *cl.map_shared_rank(&x_row[j & 1], r);
                            const int slot = *cl.map_shared_rank(&x_slot[j & 1], r);
                            const int rb = *cl.map_shared_rank(&x_bad[j & 1], r);
                            if (rb != LAGP_OK) bad = rb;
                            if (slot >= 0 && (b0.slot < 0 || better(v, row, b0.v, b0.row))) b0 = ArgBest{v, row, slot};
                        }
                        s_cstar = b0.slot;
                        s_delta = b0.v;
                        s_bad = bad != LAGP_OK ? bad : (b0.slot < 0 ? LAGP_ENOTPD : LAGP_OK);
                    }
                }
                __syncthreads();
                if (s_bad != LAGP_OK) {
                    status = s_bad;
                    break;
                }
                cstar = s_cstar;
                delta = s_delta;
            }
            // ---- partitioned inverse update with x* = candidate cstar (Sec. 2.2);
            // its panel row from the CTA that owns it
            const double *kst =
                (CL ? panel_ws + (size_t)(blockIdx.x - rank + cstar % CS) * Npmax * nmax : panel) +
                (size_t)cstar * nmax;
            // b* = K^{-1} k*: each output summed by QS threads over a share of
            // the rows, two chains each (short dependent FP64 chains)
            {
                const int QS = j * 4 <= F64_THREADS ? 4 : (j * 2 <= F64_THREADS ? 2 : 1);
                for (int e = tid; e < j * QS; e += F64_THREADS) {
                    const int t = e % j, q = e / j, k0 = q * j / QS, k1 = (q + 1) * j / QS;
                    double s0 = 0.0, s1 = 0.0;
                    int kk = k0;
                    for (; kk + 1 < k1; kk += 2) {
                        s0 = fma(S.Kinv[(size_t)kk * ld + t], kst[kk], s0);
                        s1 = fma(S.Kinv[(size_t)(kk + 1) * ld + t], kst[kk + 1], s1);
                    }
                    if (kk < k1) s0 = fma(S.Kinv[(size_t)kk * ld + t], kst[kk], s0);
                    S.part[(size_t)q * ld + t] = s0 + s1;
                }
                __syncthreads();
                for (int t = tid; t < j; t += F64_THREADS) {
                    double s = S.part[t];
                    for (int q = 1; q < QS; q++) s += S.part[(size_t)q * ld + t];
                    S.bstar[t] = s;
                }
            }
            __syncthreads();
            if (tid < 32) {
                double q = 0.0, xb = 0.0, yb = 0.0;
                for (int t = lane; t < j; t += 32) {
                    q = fma(kst[t], S.bstar[t], q);
                    if (fused) {
                        xb = fma(S.kx[t], S.bstar[t], xb);
                        yb = fma(S.yd[t], S.bstar[t], yb);
                    }
                }
                q = warp_sum(q);
                if (fused) {
                    xb = warp_sum(xb);
                    yb = warp_sum(yb);
                }
                if (lane == 0) {
                    double minv = (1.0 + g) - q;
                    s_mu = 1.0 / minv;
                    if (!(minv > 0.0)) s_bad = LAGP_ENOTPD;
                    if (fused) {
                        const int32_t row = cands[cstar];
                        s_ystar = a.dtype == LAGP_F64 ? static_cast<const double *>(a.Y)[row]
                                                      : (double)static_cast<const float *>(a.Y)[row];
                        s_ry = s_ystar - yb;          // y* - Y_j^T K^{-1} k*
                        s_cx = kappa[cstar] - xb;     // K(x*,x) - k_j(x)^T K^{-1} k*
                    }
                }
            }
            __syncthreads();
            if (s_bad != LAGP_OK) {
                status = s_bad;
                break;
            }
            const double mu = s_mu;
            // K^{-1} + g g^T / m with g = -mu b*:  += mu b* b*^T (lower triangle
            // and its mirror) ; border = -mu b*
            for (int e = tid; e < j * (j + 1) / 2; e += F64_THREADS) {
                int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
                while ((r + 1) * (r + 2) / 2 <= e) r++;
                while (r * (r + 1) / 2 > e) r--;
                const int c = e - r * (r + 1) / 2;
                const double val = fma(mu * S.bstar[r], S.bstar[c], S.Kinv[(size_t)r * ld + c]);
                S.Kinv[(size_t)r * ld + c] = val;
                S.Kinv[(size_t)c * ld + r] = val;
            }
            const double ry = fused ? s_ry : 0.0;
            for (int t = tid; t < j; t += F64_THREADS) {
                double gt = -mu * S.bstar[t];
                S.Kinv[(size_t)t * ld + j] = gt;
                S.Kinv[(size_t)j * ld + t] = gt;
                if (fused) S.alpha[t] = fma(-mu * ry, S.bstar[t], S.alpha[t]);
            }
            if (tid == 0) {
                if (fused) {
                    // Eqs. (predgp), (preds2) carried by the partitioned inverse
                    S.alpha[j] = mu * ry;
                    S.yd[j] = s_ystar;
                    s_psi = fma(mu * ry, ry, s_psi);
                    s_qx = fma(mu * s_cx, s_cx, s_qx);
                }
                S.Kinv[(size_t)j * ld + j] = mu;
                S.kx[j] = kappa[cstar];
                S.chosen[cstar] = 1;
                if (rank == 0) {
                    sel[j] = cands[cstar];
                    if (alc) alc[j] = delta;
                }
            }
            for (int i = tid; i < p; i += F64_THREADS)
                S.xd[(size_t)j * p + i] = load_coord64(a.X, cands[cstar], p, i, a.dtype);
            __syncthreads();
            // ---- append panel column j: K(x_c, x*) for every candidate (no nugget)
            if (j + 1 < nm) {
                const double *xs = S.xd + (size_t)j * p;
                for (int c = rank + CS * tid; c < k; c += CS * F64_THREADS)
                    panel[(size_t)c * nmax + j] = kern64(xs, a.X, cands[c], p, a.dtype, d);
            }
            __syncthreads();
        }
        if (status != LAGP_OK && rank == 0) {
            for (int t = tid; t < nmax; t += F64_THREADS) {
                sel[t] = -1;
                if (alc) alc[t] = CUDART_NAN;
            }
        }
        if (fused) {
            __syncthreads();
            if (warp == 0 && rank == 0) {
                double m = 0.0;
                for (int t = lane; t < nm; t += 32) m = fma(S.kx[t], S.alpha[t], m);
                m = warp_sum(m);
                if (lane == 0) {
                    const bool ok = status == LAGP_OK;
                    a.mean[loc] = ok ? m : CUDART_NAN;
                    a.s2[loc] = ok ? s_psi * ((1.0 + g) - s_qx) / nm : CUDART_NAN;
                    a.df[loc] = ok ? (double)nm : CUDART_NAN;
                }
            }
        }
        if (tid == 0 && rank == 0) a.status[loc] = status;
        __syncthreads();
    }
    // no CTA leaves while another may still read its exchange records
    if constexpr (CL) cg::this_cluster().sync();
}

}  // namespace

lagp_status launch_alc_f64(lagp_ctx *ctx, const AlcArgs &a) {
    if (a.nmax > NMAX_SMEM)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: n_max above 128 is not supported");
    cudaStream_t st = ctx->stream;
    const size_t ld = (size_t)((a.nmax + 31) & ~31);
    // K^{-1} (n_max x ld, plus one spare row so masked reads stay inside), kx, b*,
    // design coordinates, reference location, chosen flags
    size_t smem = ((size_t)a.nmax + 1) * ld * 8 + ld * 8 * 4 + 4 * ld * 8 + (size_t)a.nmax * a.p * 8 +
                  (size_t)a.p * 8 + (size_t)a.Npmax + 16;
    if (smem > ctx->smem_optin) return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: shared memory");
    // cluster size: with few locations, the CTAs of a cluster share one
    // location's candidates, as many as keep every cluster resident at once
    // (at most 4; 1 = no clusters, and whenever the user fixes the CTAs per SM)
    int cs = 1;
    if (ctx->tuning.ctas_per_sm == 0 && ctx->tune_override == 0) {
        cudaFuncSetAttribute(alc_f64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alc_f64_kernel<true>, F64_THREADS, smem);
        const int64_t fit = (int64_t)ctx->num_sms * std::max(occ, 1) / std::max<int64_t>(a.M, 1);
        cs = (int)std::min<int64_t>(4, fit);  // (4 measured faster than 6 on the 2-d toy)
        if (cs < 2) cs = 1;
    }
    int64_t grid;
    if (cs > 1) {
        ctx->last_alc_key = alc_shape_key("alc_f64", 0, a.nmax, a.p, a.mean != nullptr);
        grid = a.M * cs;
    } else {
        cudaFuncSetAttribute(alc_f64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alc_f64_kernel<false>, F64_THREADS, smem);
        int per_sm = alc_ctas_per_sm(ctx, alc_shape_key("alc_f64", 0, a.nmax, a.p, a.mean != nullptr), 2);
        if (occ > 0 && per_sm > occ) per_sm = occ;
        grid = (int64_t)ctx->num_sms * per_sm;
        if (grid > a.M) grid = a.M;
        if (grid < 1) grid = 1;
    }
    char *ws = static_cast<char *>(lagp_ws(ctx, WS_ALC_PANEL,
                                           (size_t)grid * a.Npmax * ((size_t)a.nmax + 1) * 8 + 256));
    int *counter = static_cast<int *>(lagp_ws(ctx, WS_ALC_COUNTER, 256));
    if (!ws || !counter) return LAGP_ENOMEM;
    double *panel = reinterpret_cast<double *>(ws);
    double *kappa = panel + (size_t)grid * a.Npmax * a.nmax;
    LAGP_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), st));
    if (cs > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(F64_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        LAGP_CUDA(ctx, cudaLaunchKernelEx(&cfg, alc_f64_kernel<true>, a, counter, panel, kappa));
    } else {
        alc_f64_kernel<false><<<(unsigned)grid, F64_THREADS, smem, st>>>(a, counter, panel, kappa);
    }
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
