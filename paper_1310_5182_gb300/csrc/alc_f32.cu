// a2..a6, FP32-bulk form: greedy ALC local design search (Fig. 1 step 2 of
// the paper) with the candidate screen in FP32 and every decision in FP64.
//
// Why not K_j^{-1} in FP32: the local matrices of these workloads are
// ill-conditioned (cond(K_j) ~ 1e5..1e7 for nuggets 1e-4..1e-6), so the FP32
// quadratic form k_c^T K_j^{-1} k_c carries absolute errors ~1e-2 while the
// criterion values are ~1e-7: the FP32 ranking of Eq. (dxy) is noise.  The
// same two quantities of Eq. (dxy) are therefore carried in the Cholesky
// (Schur-complement) basis, where every stored entry is bounded by 1:
//   u_c  = L_j^{-1} k_j(x_c)          whitened candidate vector (column j of U)
//   v_c  = 1 + g - |u_c|^2            = m_j^{-1}(x_c) of Eq. (piedef)
//   r_c  = K(x_c,x) - (L_j^{-1}k_j(x))^T u_c  = K(x_c,x) - k_j(x)^T K_j^{-1} k_j(x_c)
//   Delta_c = r_c^2 / v_c             = Eq. (dxy) after simplification.
// Adding x* (Schur pivot, lambda = sqrt(v_{x*})) appends one entry per
// candidate:  u_{c,j} = (K(x_c,x*) - u_{x*}^T u_c) / lambda,
//   v_c -= u_{c,j}^2,   r_c -= (r_{x*}/lambda) u_{c,j}.
// The per-step contraction U^T u_{x*} is O(j) per candidate (the paper's
// direct form is O(j^2)); its FP32 rounding error is ~j 2^-24 absolute.
//
// Each step: FP32 scores -> contenders (FP32 score within rescore_rel of the
// FP32 maximum, at most rescore_max, best first, ties to the lower row) ->
// FP64 re-score of the contenders with Eq. (dxy) using FP64 K_j^{-1} ->
// argmax (ties to the lower row) -> FP64 partitioned-inverse update of
// K_j^{-1} (Sec. 2.2) -> FP32 recurrence with pivot x*, whose lambda and
// r_{x*} come from the pivot's own FP32 state (self-consistent factor).
//
// Layout: one persistent CTA per location at a time (atomic work counter);
// candidate c lives in thread c / CPT, register slot c % CPT (v, r, score);
// the whitened panel U is a per-CTA global buffer U[i][c] (contiguous in c,
// vector loads), L2-resident; K_j^{-1}, k_j(x) and the design coordinates
// (FP64) and the candidate coordinates (FP32) sit in shared memory.
#include <cuda_runtime.h>
#include <float.h>

#include "device_util.cuh"
#include "lagp_internal.h"

namespace {

constexpr int F32_THREADS = 256;
constexpr int F32_WARPS = F32_THREADS / 32;
constexpr int LIST_CAP = 256;  // contender list capacity
// Adaptive contender margin: FP32 scores within `margin` (relative) of the
// FP32 maximum are re-scored in FP64, margin = min(rescore_rel,
// max(MARGIN_MIN, MARGIN_KAPPA * err)), where err is the largest relative
// FP32-vs-FP64 score error seen among the contenders re-scored so far,
// decaying by ERR_DECAY per step (starting at ERR_INIT).
constexpr float MARGIN_MIN = 0.02f;
constexpr float MARGIN_KAPPA = 8.0f;
constexpr float ERR_DECAY = 0.75f;
constexpr float ERR_INIT = 0.05f;

template <int JQ>
__device__ __forceinline__ void contract64(const double *__restrict__ kc_s, const double *Kinv, int ld,
                                           const double *kx, int j, int lane, double *b_out,
                                           double &quad, double &kxb) {
    double kc[JQ], b[JQ];
#pragma unroll
    for (int r = 0; r < JQ; r++) {
        kc[r] = (lane + 32 * r < j) ? kc_s[lane + 32 * r] : 0.0;
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
            b_out[lane + 32 * r] = b[r];
        }
    quad = warp_sum(q);
    kxb = warp_sum(x);
}

template <int CPT>
__device__ __forceinline__ void load_vec(const float *p, float (&v)[CPT]) {
    if constexpr (CPT % 4 == 0) {
#pragma unroll
        for (int r = 0; r < CPT; r += 4) {
            float4 t = *reinterpret_cast<const float4 *>(p + r);
            v[r] = t.x;
            v[r + 1] = t.y;
            v[r + 2] = t.z;
            v[r + 3] = t.w;
        }
    } else if constexpr (CPT == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int r = 0; r < CPT; r++) v[r] = p[r];
    }
}

template <int CPT>
__device__ __forceinline__ void store_vec(float *p, const float (&v)[CPT]) {
    if constexpr (CPT % 4 == 0) {
#pragma unroll
        for (int r = 0; r < CPT; r += 4)
            *reinterpret_cast<float4 *>(p + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
    } else if constexpr (CPT == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int r = 0; r < CPT; r++) p[r] = v[r];
    }
}

struct F32Params {
    AlcArgs a;
    int *counter;
    float *U_ws;      // per CTA: nmax x Npad
    int Npad;         // F32_THREADS * CPT
    int tmax;         // rescore_max
    float rel;        // rescore_rel
};

template <int CPT>
__global__ void __launch_bounds__(F32_THREADS)
alc_f32_kernel(F32Params P) {
    const AlcArgs &a = P.a;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, Npmax = a.Npmax, Npad = P.Npad, tmax = P.tmax;
    const int ld = (nmax + 31) & ~31;
    double *Kinv = reinterpret_cast<double *>(smem_raw);       // (nmax+1) x ld
    double *kx = Kinv + (size_t)(nmax + 1) * ld;               // ld
    double *xd = kx + ld;                                      // nmax x p
    double *xq = xd + (size_t)nmax * p;                        // p
    double *con_b = xq + p;                                    // tmax x ld
    double *con_k = con_b + (size_t)tmax * ld;                 // tmax x ld
    double *con_x = con_k + (size_t)tmax * ld;                 // tmax x p
    float *coords = reinterpret_cast<float *>(con_x + (size_t)tmax * p);  // p x Npad
    float *ustar = coords + (size_t)p * Npad;                  // ld
    float *xs32 = ustar + ld;                                  // p
    float *list_s = xs32 + p;                                  // LIST_CAP scores
    int *list_c = reinterpret_cast<int *>(list_s + LIST_CAP);  // LIST_CAP slots
    int *list_r = list_c + LIST_CAP;                           // LIST_CAP design rows

    __shared__ int s_loc, s_bad, s_ncon, s_win;
    __shared__ int w_cnt[F32_WARPS];
    __shared__ float w_best[F32_WARPS];
    __shared__ int w_brow[F32_WARPS];
    __shared__ int con_slot[32], con_row[32];
    __shared__ double con_delta[32], con_minv[32], con_kxb[32], con_kap[32];
    __shared__ float s_vstar, s_covstar, s_fmax, s_err;
    __shared__ float con_s32[32];

    float *U = P.U_ws + (size_t)blockIdx.x * nmax * Npad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = tid * CPT;  // first candidate slot of this thread

    for (;;) {
        if (tid == 0) s_loc = atomicAdd(P.counter, 1);
        __syncthreads();
        const int64_t loc = s_loc;
        __syncthreads();
        if (loc >= a.M) break;

        const int k = a.Np ? a.Np[loc] : Npmax;
        const int nm = a.n ? a.n[loc] : nmax;
        const double d = a.d[loc], g = a.g;
        const int32_t *cands = a.idx + loc * Npmax;
        int32_t *sel = a.sel + loc * nmax;
        double *alc = a.alc ? a.alc + loc * nmax : nullptr;

        if (tid == 0) s_bad = (k < 1 || k > Npmax || nm < a.n0 || nm > nmax || nm > k || !(d > 0.0) ||
                               !isfinite(d)) ? LAGP_EINVAL : LAGP_OK;
        __syncthreads();
        if (s_bad == LAGP_OK)
            for (int c = tid; c < k; c += F32_THREADS) {
                int32_t r = cands[c];
                if (r < 0 || r >= a.N) s_bad = LAGP_EINVAL;
            }
        __syncthreads();
        for (int t = tid; t < nmax; t += F32_THREADS) {
            sel[t] = -1;
            if (alc) alc[t] = CUDART_NAN;
        }
        if (s_bad != LAGP_OK) {
            if (tid == 0) a.status[loc] = s_bad;
            continue;
        }

        // ---- per-location set-up: coordinates, kappa, initial FP32 state
        for (int i = tid; i < p; i += F32_THREADS) xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
        for (int e = tid; e < p * Npad; e += F32_THREADS) {
            int i = e / Npad, c = e - i * Npad;
            coords[e] = c < k ? load_coord32(a.X, cands[c], p, i, a.dtype) : 0.f;
        }
        __syncthreads();
        const float inv_d = (float)(1.0 / d);
        const float gf = fmaxf((float)g, FLT_MIN);
        float v[CPT], cov[CPT], score[CPT];
        int rows[CPT];  // design rows of this thread's candidates (tie-break key)
        unsigned chosen = 0;
#pragma unroll
        for (int r = 0; r < CPT; r++) {
            const int c = c0 + r;
            rows[r] = c < k ? cands[c] : INT32_MAX;
            float s = 0.f;
            for (int i = 0; i < p; i++) {
                float df = coords[i * Npad + c] - (float)xq[i];
                s = fmaf(df, df, s);
            }
            v[r] = (float)(1.0 + g);
            cov[r] = __expf(-s * inv_d);  // K(x_c, x), no nugget
            score[r] = c < k ? cov[r] * cov[r] / v[r] : -1.f;
            if (c >= k) chosen |= 1u << r;  // padding slots never compete
        }

        int status = LAGP_OK;
        if (tid == 0) s_err = ERR_INIT;
        for (int j = 0; j < nm; j++) {
            // ---------------- contenders for design index j
            if (j < a.n0) {
                if (tid == 0) {
                    s_ncon = 1;
                    con_slot[0] = j;  // Fig. 1 step 2(a): nearest neighbours in order
                    con_row[0] = cands[j];
                }
            } else {
                // FP32 block maximum
                float bm = -1.f;
                int brow = INT32_MAX;
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (!(chosen >> r & 1u)) {
                        if (score[r] > bm || (score[r] == bm && rows[r] < brow)) {
                            bm = score[r];
                            brow = rows[r];
                        }
                    }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float ov = __shfl_xor_sync(LAGP_FULL_MASK, bm, o);
                    int orow = __shfl_xor_sync(LAGP_FULL_MASK, brow, o);
                    if (ov > bm || (ov == bm && orow < brow)) {
                        bm = ov;
                        brow = orow;
                    }
                }
                if (lane == 0) {
                    w_best[warp] = bm;
                    w_brow[warp] = brow;
                }
                __syncthreads();
                if (tid == 0) {
                    float m0 = w_best[0];
                    for (int w = 1; w < F32_WARPS; w++) m0 = fmaxf(m0, w_best[w]);
                    s_fmax = m0;
                }
                __syncthreads();
                // contenders: FP32 score >= (1 - margin) * max, gathered in slot order
                const float margin = fminf(P.rel, fmaxf(MARGIN_MIN, MARGIN_KAPPA * s_err));
                const float thr = s_fmax - margin * fabsf(s_fmax);
                unsigned flags = 0;
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (!(chosen >> r & 1u) && score[r] >= thr) flags |= 1u << r;
                const int mine = __popc(flags);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(LAGP_FULL_MASK, incl, o);
                    if (lane >= o) incl += t;
                }
                if (lane == 31) w_cnt[warp] = incl;
                __syncthreads();
                int off = 0, total = 0;
                for (int w = 0; w < F32_WARPS; w++) {
                    if (w < warp) off += w_cnt[w];
                    total += w_cnt[w];
                }
                int pos = off + incl - mine;
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (flags >> r & 1u) {
                        if (pos < LIST_CAP) {
                            list_s[pos] = score[r];
                            list_c[pos] = c0 + r;
                            list_r[pos] = rows[r];
                        }
                        pos++;
                    }
                __syncthreads();
                // warp 0: the best tmax of the list (score desc, row asc)
                if (warp == 0) {
                    const int cnt = min(total, LIST_CAP);
                    int ncon = 0;
                    for (int t = 0; t < tmax && t < cnt; t++) {
                        float bs = -FLT_MAX;
                        int brw = INT32_MAX, bpos = -1;
                        for (int e = lane; e < cnt; e += 32) {
                            if (list_c[e] < 0) continue;
                            const int row = list_r[e];
                            if (list_s[e] > bs || (list_s[e] == bs && row < brw)) {
                                bs = list_s[e];
                                brw = row;
                                bpos = e;
                            }
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            float ov = __shfl_xor_sync(LAGP_FULL_MASK, bs, o);
                            int orw = __shfl_xor_sync(LAGP_FULL_MASK, brw, o);
                            int opos = __shfl_xor_sync(LAGP_FULL_MASK, bpos, o);
                            if (ov > bs || (ov == bs && orw < brw)) {
                                bs = ov;
                                brw = orw;
                                bpos = opos;
                            }
                        }
                        if (bpos < 0) break;
                        if (lane == 0) {
                            con_slot[ncon] = list_c[bpos];
                            con_row[ncon] = brw;
                            con_s32[ncon] = bs;
                            list_c[bpos] = -1;
                        }
                        __syncwarp();
                        ncon++;
                    }
                    if (lane == 0) s_ncon = ncon;
                }
            }
            __syncthreads();
            const int ncon = s_ncon;
            if (ncon < 1) {
                status = LAGP_ENOTPD;
                break;
            }
            // ---------------- FP64 re-score of the contenders (Eq. dxy), one warp each
            for (int w = warp; w < ncon; w += F32_WARPS) {
                const int row = con_row[w];
                double *xc = con_x + (size_t)w * p;
                double *kc = con_k + (size_t)w * ld;
                for (int i = lane; i < p; i += 32) xc[i] = load_coord64(a.X, row, p, i, a.dtype);
                __syncwarp();
                for (int t = lane; t < j; t += 32) {
                    double s = 0.0;
                    for (int i = 0; i < p; i++) {
                        double df = xc[i] - xd[(size_t)t * p + i];
                        s = fma(df, df, s);
                    }
                    kc[t] = exp(-s / d);
                }
                double sk = 0.0;
                for (int i = 0; i < p; i++) {
                    double df = xc[i] - xq[i];
                    sk = fma(df, df, sk);
                }
                const double kap = exp(-sk / d);
                __syncwarp();
                double quad = 0.0, kxb = 0.0;
                double *bo = con_b + (size_t)w * ld;
                if (j > 0) {
                    switch ((j + 31) >> 5) {
                        case 1: contract64<1>(kc, Kinv, ld, kx, j, lane, bo, quad, kxb); break;
                        case 2: contract64<2>(kc, Kinv, ld, kx, j, lane, bo, quad, kxb); break;
                        case 3: contract64<3>(kc, Kinv, ld, kx, j, lane, bo, quad, kxb); break;
                        default: contract64<4>(kc, Kinv, ld, kx, j, lane, bo, quad, kxb); break;
                    }
                }
                if (lane == 0) {
                    const double minv = (1.0 + g) - quad;
                    const double m = 1.0 / minv;
                    const double kxg = -m * kxb;
                    con_minv[w] = minv;
                    con_kxb[w] = kxb;
                    con_kap[w] = kap;
                    con_delta[w] = minv > 0.0 ? kxg * kxg * minv + 2.0 * kxg * kap + kap * kap * m
                                              : -CUDART_INF;
                }
            }
            __syncthreads();
            if (tid == 0) {
                int wb = 0;
                float e = 0.f;
                for (int w = 0; w < ncon; w++) {
                    if (w > 0 && better(con_delta[w], con_row[w], con_delta[wb], con_row[wb])) wb = w;
                    if (j >= a.n0 && con_delta[w] > 0.0)
                        e = fmaxf(e, (float)fabs((double)con_s32[w] / con_delta[w] - 1.0));
                }
                if (j >= a.n0) s_err = fmaxf(ERR_DECAY * s_err, e);
                s_win = wb;
                if (!(con_minv[wb] > 0.0)) s_bad = LAGP_ENOTPD;
            }
            __syncthreads();
            if (s_bad != LAGP_OK) {
                status = s_bad;
                break;
            }
            // ---------------- FP64 partitioned-inverse update (Sec. 2.2)
            const int wb = s_win, cstar = con_slot[wb];
            {
                const double mu = 1.0 / con_minv[wb];
                const double *b = con_b + (size_t)wb * ld;
                // lower triangle with its mirror: j(j+1)/2 FMAs
                for (int e = tid; e < j * (j + 1) / 2; e += F32_THREADS) {
                    int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
                    while ((r + 1) * (r + 2) / 2 <= e) r++;
                    while (r * (r + 1) / 2 > e) r--;
                    const int c = e - r * (r + 1) / 2;
                    const double val = fma(mu * b[r], b[c], Kinv[(size_t)r * ld + c]);
                    Kinv[(size_t)r * ld + c] = val;
                    Kinv[(size_t)c * ld + r] = val;
                }
                for (int t = tid; t < j; t += F32_THREADS) {
                    double gt = -mu * b[t];
                    Kinv[(size_t)t * ld + j] = gt;
                    Kinv[(size_t)j * ld + t] = gt;
                }
                if (tid == 0) {
                    Kinv[(size_t)j * ld + j] = mu;
                    kx[j] = con_kap[wb];
                    sel[j] = con_row[wb];
                    if (alc && j >= a.n0) alc[j] = con_delta[wb];
                }
                for (int i = tid; i < p; i += F32_THREADS) {
                    xd[(size_t)j * p + i] = con_x[(size_t)wb * p + i];
                    xs32[i] = coords[i * Npad + cstar];
                }
                for (int i = tid; i < j; i += F32_THREADS) ustar[i] = U[(size_t)i * Npad + cstar];
            }
            // The FP32 recurrence continues from the pivot's own FP32 state:
            // lambda^2 = v_{x*} and r_{x*}, so that U stays the Cholesky factor
            // of one (slightly perturbed) matrix; mixing in the FP64 values
            // breaks that consistency and the recurrence drifts.
#pragma unroll
            for (int r = 0; r < CPT; r++)
                if (c0 + r == cstar) {
                    s_vstar = v[r];
                    s_covstar = cov[r];
                    chosen |= 1u << r;
                }
            __syncthreads();
            if (j + 1 >= nm) break;
            // ---------------- FP32 Schur recurrence with pivot x* (new column j of U)
            {
                const float inv_lam = rsqrtf(fmaxf(s_vstar, gf));
                const float wnew = s_covstar * inv_lam;
                float acc[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) acc[r] = 0.f;
                const float *Ub = U + c0;
                int i = 0;
                for (; i + 4 <= j; i += 4) {
                    float u0[CPT], u1[CPT], u2[CPT], u3[CPT];
                    load_vec<CPT>(Ub + (size_t)(i + 0) * Npad, u0);
                    load_vec<CPT>(Ub + (size_t)(i + 1) * Npad, u1);
                    load_vec<CPT>(Ub + (size_t)(i + 2) * Npad, u2);
                    load_vec<CPT>(Ub + (size_t)(i + 3) * Npad, u3);
                    const float s0 = ustar[i], s1 = ustar[i + 1], s2 = ustar[i + 2], s3 = ustar[i + 3];
#pragma unroll
                    for (int r = 0; r < CPT; r++) {
                        acc[r] = fmaf(u0[r], s0, acc[r]);
                        acc[r] = fmaf(u1[r], s1, acc[r]);
                        acc[r] = fmaf(u2[r], s2, acc[r]);
                        acc[r] = fmaf(u3[r], s3, acc[r]);
                    }
                }
                for (; i < j; i++) {
                    float u0[CPT];
                    load_vec<CPT>(Ub + (size_t)i * Npad, u0);
                    const float s0 = ustar[i];
#pragma unroll
                    for (int r = 0; r < CPT; r++) acc[r] = fmaf(u0[r], s0, acc[r]);
                }
                float un[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) {
                    const int c = c0 + r;
                    float s = 0.f;
                    for (int ii = 0; ii < p; ii++) {
                        float df = coords[ii * Npad + c] - xs32[ii];
                        s = fmaf(df, df, s);
                    }
                    const float kcs = __expf(-s * inv_d);  // K(x_c, x*), no nugget
                    un[r] = (kcs - acc[r]) * inv_lam;
                    v[r] = fmaf(-un[r], un[r], v[r]);
                    cov[r] = fmaf(-wnew, un[r], cov[r]);
                    score[r] = (chosen >> r & 1u) ? -1.f : cov[r] * cov[r] / fmaxf(v[r], gf);
                }
                store_vec<CPT>(U + (size_t)j * Npad + c0, un);
            }
            __syncthreads();  // U column j visible before the next pivot reads it
        }
        if (status != LAGP_OK) {
            for (int t = tid; t < nmax; t += F32_THREADS) {
                sel[t] = -1;
                if (alc) alc[t] = CUDART_NAN;
            }
        }
        if (tid == 0) a.status[loc] = status;
        __syncthreads();
    }
}

template <int CPT>
lagp_status launch_cpt(lagp_ctx *ctx, const AlcArgs &a) {
    cudaStream_t st = ctx->stream;
    const int Npad = F32_THREADS * CPT;
    const int tmax = ctx->tuning.rescore_max > 0 ? ctx->tuning.rescore_max : 8;
    const size_t ld = (size_t)((a.nmax + 31) & ~31);
    size_t smem = ((size_t)a.nmax + 1) * ld * 8 + ld * 8 + (size_t)a.nmax * a.p * 8 + (size_t)a.p * 8 +
                  (size_t)tmax * ld * 8 * 2 + (size_t)tmax * a.p * 8 + (size_t)a.p * Npad * 4 + ld * 4 +
                  (size_t)a.p * 4 + (size_t)LIST_CAP * 12 + 64;
    if (smem > ctx->smem_optin)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: shared memory exceeded (n_max, N', p too large)");
    cudaFuncSetAttribute(alc_f32_kernel<CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alc_f32_kernel<CPT>, F32_THREADS, smem);
    int per_sm = ctx->tuning.ctas_per_sm > 0 ? ctx->tuning.ctas_per_sm : 2;
    if (occ > 0 && per_sm > occ) per_sm = occ;
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    if (grid > a.M) grid = a.M;
    if (grid < 1) grid = 1;
    float *U = static_cast<float *>(lagp_ws(ctx, WS_ALC_PANEL, (size_t)grid * a.nmax * Npad * 4 + 256));
    int *counter = static_cast<int *>(lagp_ws(ctx, WS_ALC_COUNTER, 256));
    if (!U || !counter) return LAGP_ENOMEM;
    LAGP_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), st));
    F32Params P{a, counter, U, Npad, tmax, (float)ctx->tuning.rescore_rel};
    alc_f32_kernel<CPT><<<(unsigned)grid, F32_THREADS, smem, st>>>(P);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

}  // namespace

lagp_status launch_alc_f32(lagp_ctx *ctx, const AlcArgs &a) {
    if (a.nmax > 128)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: n_max above 128 is not supported");
    const int need = (a.Npmax + F32_THREADS - 1) / F32_THREADS;
    if (need <= 1) return launch_cpt<1>(ctx, a);
    if (need <= 2) return launch_cpt<2>(ctx, a);
    if (need <= 4) return launch_cpt<4>(ctx, a);
    if (need <= 8) return launch_cpt<8>(ctx, a);
    return launch_cpt<16>(ctx, a);
}
