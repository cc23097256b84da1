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
// Layout: one persistent CTA per location at a time (atomic work counter),
// three CTAs per SM so that one location's serial FP64 phase overlaps other
// locations' FP32 passes; candidate c lives in thread c / CPT, register slot
// c % CPT (v, r, score); the whitened panel U[i][c] and the FP32 candidate
// coordinates C[i][c] are per-CTA global buffers (contiguous in c, vector
// loads, L2-resident); K_j^{-1}, k_j(x), the design coordinates and the
// contenders' FP64 vectors sit in shared memory.  Contenders are found with
// per-warp lists merged by one warp; each contender's FP32 column of U is
// fetched during its FP64 re-score, so the winner's column (the next pivot)
// is already in shared memory when the FP32 pass starts.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "device_util.cuh"
#include "lagp_internal.h"

namespace {

constexpr int F32_THREADS = 256;
constexpr int F32_WARPS = F32_THREADS / 32;
// Adaptive contender margin: FP32 scores within `margin` (relative) of the
// FP32 maximum are re-scored in FP64, margin = min(rescore_rel,
// max(MARGIN_MIN, MARGIN_KAPPA * err)), where err is the largest relative
// FP32-vs-FP64 score error seen among the contenders re-scored so far,
// decaying by ERR_DECAY per step (starting at ERR_INIT).
constexpr float MARGIN_MIN = 0.02f;
constexpr float MARGIN_KAPPA = 8.0f;
constexpr float ERR_DECAY = 0.75f;
constexpr float ERR_INIT = 0.05f;

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
    float *U_ws;      // per CTA: nmax x Npad (whitened panel U[i][c])
    float *C_ws;      // per CTA: p x Npad (FP32 candidate coordinates C[i][c])
    double *K_ws;     // per CTA: Npad (FP64 K(x_c, x), computed once per location)
    int Npad;         // F32_THREADS * CPT
    int tmax;         // rescore_max
    float rel;        // rescore_rel (cap of the contender margin)
};

// Rows [k0, k1) of the contraction b = K^{-1} kc: lane t writes
// sum_{kk in [k0,k1)} K^{-1}[kk][t] kc[kk] for its columns t = lane + 32 r
// (rows of the symmetric K^{-1} have leading dimension ld, a multiple of 32).
template <int JQ>
__device__ __forceinline__ void partial_contract(const double *kc, const double *Kinv, int ld, int k0,
                                                 int k1, int j, int lane, double *out) {
    double b0[JQ], b1[JQ];
#pragma unroll
    for (int r = 0; r < JQ; r++) b0[r] = b1[r] = 0.0;
    int kk = k0;
    for (; kk + 2 <= k1; kk += 2) {
        const double v0 = kc[kk], v1 = kc[kk + 1];
        const double *row0 = Kinv + (size_t)kk * ld + lane, *row1 = row0 + ld;
#pragma unroll
        for (int r = 0; r < JQ; r++) {
            b0[r] = fma(row0[32 * r], v0, b0[r]);
            b1[r] = fma(row1[32 * r], v1, b1[r]);
        }
    }
    if (kk < k1) {
        const double v0 = kc[kk];
        const double *row0 = Kinv + (size_t)kk * ld + lane;
#pragma unroll
        for (int r = 0; r < JQ; r++) b0[r] = fma(row0[32 * r], v0, b0[r]);
    }
#pragma unroll
    for (int r = 0; r < JQ; r++)
        if (lane + 32 * r < j) out[lane + 32 * r] = b0[r] + b1[r];
}

// Integer key with the order of the doubles (for comparisons off the FP64 pipe)
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// (score, row, slot) argmax across a warp: larger score, ties to the lower row
__device__ __forceinline__ void warp_best3(float &s, int &row, int &slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float os = __shfl_xor_sync(LAGP_FULL_MASK, s, o);
        int orow = __shfl_xor_sync(LAGP_FULL_MASK, row, o);
        int oslot = __shfl_xor_sync(LAGP_FULL_MASK, slot, o);
        if (os > s || (os == s && orow < row)) {
            s = os;
            row = orow;
            slot = oslot;
        }
    }
}

// four resident CTAs per SM (64 registers a thread) for up to 4 candidate
// slots a thread, fewer for the wider variants whose state needs more
template <int CPT>
__global__ void __launch_bounds__(F32_THREADS, CPT >= 16 ? 2 : (CPT >= 8 ? 3 : 4))
alc_f32_kernel(F32Params P) {
    const AlcArgs &a = P.a;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, Npmax = a.Npmax, Npad = P.Npad, tmax = P.tmax;
    const int ld = (nmax + 31) & ~31;
    double *Kinv = reinterpret_cast<double *>(smem_raw);       // (nmax+1) x ld
    double *kx = Kinv + (size_t)(nmax + 1) * ld;               // ld: k_j(x)
    double *yd = kx + ld;                                      // ld: responses of the design
    double *alpha = yd + ld;                                   // ld: K_j^{-1} Y_j
    double *xd = alpha + ld;                                   // nmax x p: design coordinates
    double *xq = xd + (size_t)nmax * p;                        // p: reference location
    double *con_b = xq + p;                                    // tmax x ld: K^{-1} k_j(x_c)
    double *con_k = con_b + (size_t)tmax * ld;                 // tmax x ld: k_j(x_c), FP64
    double *con_x = con_k + (size_t)tmax * ld;                 // tmax x p: coordinates, FP64
    float *con_u = reinterpret_cast<float *>(con_x + (size_t)tmax * p);  // tmax x ld: U column
    float *con_c = con_u + (size_t)tmax * ld;                  // tmax x p: coordinates, FP32
    // max(8, tmax) x ld partial contractions (one row per R2 job)
    double *cpart = reinterpret_cast<double *>(con_c + (((size_t)tmax * p + 1) & ~(size_t)1));
    float *list_s = reinterpret_cast<float *>(cpart + (size_t)max(F32_WARPS, tmax) * ld);  // Npad scores
    int *list_c = reinterpret_cast<int *>(list_s + Npad);      // Npad: their slots
    int *list_r = list_c + Npad;                               // Npad: their design rows

    __shared__ int s_loc, s_bad, s_ncon, s_win;
    __shared__ int w_cnt[F32_WARPS];
    __shared__ float w_max[F32_WARPS];
    __shared__ int con_slot[32], con_row[32];
    __shared__ float con_s32[32], con_err[32];
    __shared__ double con_delta[32], con_minv[32], con_mu[32], con_kxb[32], con_kap[32], con_ry[32],
        con_y[32], con_dot[3][32];
    __shared__ long long con_key[32];
    __shared__ double s_psi, s_qx;
    __shared__ float s_vstar, s_covstar, s_err;
    const bool fused = a.mean != nullptr;

    float *U = P.U_ws + (size_t)blockIdx.x * nmax * Npad;
    float *Cg = P.C_ws + (size_t)blockIdx.x * p * Npad;
    double *kap64 = P.K_ws + (size_t)blockIdx.x * Npad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = tid * CPT;  // first candidate slot of this thread
    const int rot = blockIdx.x & (F32_WARPS - 1);

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
            if (tid == 0) {
                a.status[loc] = s_bad;
                if (fused) a.mean[loc] = a.s2[loc] = a.df[loc] = CUDART_NAN;
            }
            continue;
        }

        // ---- per-location set-up: coordinates, kappa, initial FP32 state
        for (int i = tid; i < p; i += F32_THREADS) xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
        for (int e = tid; e < p * Npad; e += F32_THREADS) {
            int i = e / Npad, c = e - i * Npad;
            Cg[e] = c < k ? load_coord32(a.X, cands[c], p, i, a.dtype) : 0.f;
        }
        const double inv_d64 = 1.0 / d;
        __syncthreads();
        // K(x_c, x) in FP64 for every candidate, once per location (the FP64
        // re-score then reads it instead of recomputing an exponential)
        for (int c = tid; c < k; c += F32_THREADS) {
            const int32_t r = cands[c];
            double s0 = 0.0, s1 = 0.0;
            int i = 0;
            for (; i + 2 <= p; i += 2) {
                const double d0 = load_coord64(a.X, r, p, i, a.dtype) - xq[i];
                const double d1 = load_coord64(a.X, r, p, i + 1, a.dtype) - xq[i + 1];
                s0 = fma(d0, d0, s0);
                s1 = fma(d1, d1, s1);
            }
            if (i < p) {
                const double d0 = load_coord64(a.X, r, p, i, a.dtype) - xq[i];
                s0 = fma(d0, d0, s0);
            }
            kap64[c] = exp(-(s0 + s1) * inv_d64);
        }
        const float inv_d = (float)(1.0 / d);
        const float gf = fmaxf((float)g, FLT_MIN);
        float v[CPT], cov[CPT], score[CPT];
        int rows[CPT];  // design rows of this thread's candidates (tie-break key)
        unsigned chosen = 0;
        {
            float s[CPT];
#pragma unroll
            for (int r = 0; r < CPT; r++) s[r] = 0.f;
            for (int i = 0; i < p; i++) {
                float cv[CPT];
                load_vec<CPT>(Cg + (size_t)i * Npad + c0, cv);
                const float qi = (float)xq[i];
#pragma unroll
                for (int r = 0; r < CPT; r++) {
                    float df = cv[r] - qi;
                    s[r] = fmaf(df, df, s[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < CPT; r++) {
                const int c = c0 + r;
                rows[r] = c < k ? cands[c] : INT32_MAX;
                v[r] = (float)(1.0 + g);
                cov[r] = __expf(-s[r] * inv_d);  // K(x_c, x), no nugget
                score[r] = c < k ? cov[r] * cov[r] / v[r] : -1.f;
                if (c >= k) chosen |= 1u << r;  // padding slots never compete
            }
        }

        {
            float wm = -FLT_MAX;
#pragma unroll
            for (int r = 0; r < CPT; r++)
                if (!(chosen >> r & 1u)) wm = fmaxf(wm, score[r]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(LAGP_FULL_MASK, wm, o));
            if (lane == 0) w_max[warp] = wm;
        }
        int status = LAGP_OK;
        if (tid == 0) {
            s_err = ERR_INIT;
            s_psi = 0.0;
            s_qx = 0.0;
        }
        __syncthreads();
        for (int j = 0; j < nm; j++) {
            // ---------------- contenders for design index j
            if (j < a.n0) {
                if (tid == 0) {
                    s_ncon = 1;
                    con_slot[0] = j;  // Fig. 1 step 2(a): nearest neighbours in order
                    con_row[0] = cands[j];
                    con_s32[0] = 0.f;
                }
            } else {
                __syncthreads();  // the per-warp maxima of the last FP32 pass
                const float margin = fminf(P.rel, fmaxf(MARGIN_MIN, MARGIN_KAPPA * s_err));
                float gmax = w_max[0];
#pragma unroll
                for (int w = 1; w < F32_WARPS; w++) gmax = fmaxf(gmax, w_max[w]);
                const float thr = gmax - margin * fabsf(gmax);
                unsigned flags = 0;
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (!(chosen >> r & 1u) && score[r] >= thr) flags |= 1u << r;
                const int mine = __popc(flags);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(LAGP_FULL_MASK, incl, o);
                    if (lane >= o) incl += t;
                }
                if (lane == 31) w_cnt[warp] = incl;
                __syncthreads();
                int off = 0, total = 0;
#pragma unroll
                for (int w = 0; w < F32_WARPS; w++) {
                    off += w < warp ? w_cnt[w] : 0;
                    total += w_cnt[w];
                }
                int pos = off + incl - mine;  // slot order: deterministic
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (flags >> r & 1u) {
                        list_s[pos] = score[r];
                        list_c[pos] = c0 + r;
                        list_r[pos] = rows[r];
                        pos++;
                    }
                __syncthreads();
                if (warp == 0) {
                    if (total <= tmax) {  // every flagged candidate is re-scored
                        for (int e = lane; e < total; e += 32) {
                            con_slot[e] = list_c[e];
                            con_row[e] = list_r[e];
                            con_s32[e] = list_s[e];
                        }
                        if (lane == 0) s_ncon = total;
                    } else {  // the best tmax by FP32 score, ties to the lower row
                        int ncon = 0;
                        for (int t = 0; t < tmax; t++) {
                            float bs = -FLT_MAX;
                            int brow = INT32_MAX, bpos = -1;
                            for (int e = lane; e < total; e += 32)
                                if (list_c[e] >= 0 &&
                                    (list_s[e] > bs || (list_s[e] == bs && list_r[e] < brow))) {
                                    bs = list_s[e];
                                    brow = list_r[e];
                                    bpos = e;
                                }
                            warp_best3(bs, brow, bpos);
                            if (bpos < 0) break;
                            if (lane == 0) {
                                con_slot[ncon] = list_c[bpos];
                                con_row[ncon] = brow;
                                con_s32[ncon] = bs;
                                list_c[bpos] = -1;
                            }
                            __syncwarp();
                            ncon++;
                        }
                        if (lane == 0) s_ncon = ncon;
                    }
                }
            }
            __syncthreads();
            const int ncon = s_ncon;
            if (ncon < 1) {
                status = LAGP_ENOTPD;
                break;
            }
            // ---------------- FP64 re-score of the contenders (Eq. dxy).  On this
            // GPU an FP64 warp instruction holds its sub-partition's FP64 unit
            // for ~64 cycles whatever the number of active lanes, so the work is
            // cut into phases spread over all warps (with a per-CTA rotation of
            // roles, so that co-resident CTAs use different sub-partitions).
            const int we = (warp + rot) & (F32_WARPS - 1);  // rotated warp role
            // R0: contender data: FP64 and FP32 coordinates, response, and the
            // FP32 column of U that serves as the next Schur pivot if it wins
            for (int e = tid; e < ncon * p; e += F32_THREADS) {
                const int w = e / p, i = e - w * p;
                con_x[(size_t)w * p + i] = load_coord64(a.X, con_row[w], p, i, a.dtype);
                con_c[(size_t)w * p + i] = Cg[(size_t)i * Npad + con_slot[w]];
            }
            for (int e = tid; e < ncon * j; e += F32_THREADS) {
                const int w = e / j, t = e - w * j;
                con_u[(size_t)w * ld + t] = U[(size_t)t * Npad + con_slot[w]];
            }
            if (fused && tid < ncon) {
                const int row = con_row[tid];
                con_y[tid] = a.dtype == LAGP_F64 ? static_cast<const double *>(a.Y)[row]
                                                 : (double)static_cast<const float *>(a.Y)[row];
            }
            __syncthreads();
            // R1: k_j(x_c) in FP64, (contender, design row) pairs packed over lanes
            {
                const int te = (tid + 32 * rot) & (F32_THREADS - 1);
                for (int e = te; e < ncon * j; e += F32_THREADS) {
                    const int w = e / j, t = e - w * j;
                    const double *xc = con_x + (size_t)w * p;
                    const double *xt = xd + (size_t)t * p;
                    double s0 = 0.0, s1 = 0.0;
                    int i = 0;
                    for (; i + 2 <= p; i += 2) {
                        const double d0 = xc[i] - xt[i], d1 = xc[i + 1] - xt[i + 1];
                        s0 = fma(d0, d0, s0);
                        s1 = fma(d1, d1, s1);
                    }
                    if (i < p) {
                        const double d0 = xc[i] - xt[i];
                        s0 = fma(d0, d0, s0);
                    }
                    con_k[(size_t)w * ld + t] = exp(-(s0 + s1) * inv_d64);
                }
            }
            __syncthreads();
            // R2: partial contractions K^{-1} k_j(x_c), each contender's rows
            // split over wpc warps
            // warps per contender: the largest power of two with ncon * wpc <= 8,
            // so that the R2 jobs fit the max(8, tmax) rows of cpart
            const int wpc = ncon >= 5 ? 1 : (ncon >= 3 ? 2 : (ncon >= 2 ? 4 : 8));
            if (j > 0) {
                const int rows = max(F32_WARPS, tmax);  // rows of cpart
                for (int job = we; job < ncon * wpc && job < rows; job += F32_WARPS) {
                    const int w = job / wpc, part = job - w * wpc;
                    const int k0 = part * j / wpc, k1 = (part + 1) * j / wpc;
                    switch ((j + 31) >> 5) {
                        case 1: partial_contract<1>(con_k + (size_t)w * ld, Kinv, ld, k0, k1, j, lane, cpart + (size_t)job * ld); break;
                        case 2: partial_contract<2>(con_k + (size_t)w * ld, Kinv, ld, k0, k1, j, lane, cpart + (size_t)job * ld); break;
                        case 3: partial_contract<3>(con_k + (size_t)w * ld, Kinv, ld, k0, k1, j, lane, cpart + (size_t)job * ld); break;
                        default: partial_contract<4>(con_k + (size_t)w * ld, Kinv, ld, k0, k1, j, lane, cpart + (size_t)job * ld); break;
                    }
                }
            }
            __syncthreads();
            // R3: b = sum of the partials; the dot products k^T b, k(x)^T b and
            // Y^T b, one warp each
            {
                const int ns = fused ? 3 : 2;
                for (int job = we; job < ncon * ns; job += F32_WARPS) {
                    const int w = job / ns, sdot = job - w * ns;
                    const double *v = sdot == 0 ? con_k + (size_t)w * ld : (sdot == 1 ? kx : yd);
                    double acc = 0.0;
                    for (int t = lane; t < j; t += 32) {
                        double bt = 0.0;
                        for (int q = 0; q < wpc; q++) bt += cpart[(size_t)(w * wpc + q) * ld + t];
                        if (sdot == 0) con_b[(size_t)w * ld + t] = bt;
                        acc = fma(v[t], bt, acc);
                    }
                    acc = warp_sum(acc);
                    if (lane == 0) con_dot[sdot][w] = acc;
                }
            }
            __syncthreads();
            // R4: per-contender scalars of Eqs. (piedef), (dxy), in parallel
            if (tid < ncon) {
                const int w = tid;
                const double quad = j > 0 ? con_dot[0][w] : 0.0, kxb = j > 0 ? con_dot[1][w] : 0.0;
                const double kap = kap64[con_slot[w]];
                const double minv = (1.0 + g) - quad;  // m_j^{-1}(x_c)
                const double m = 1.0 / minv;
                const double kxg = -m * kxb;           // k_j(x)^T g_j(x_c)
                const double dl = kxg * kxg * minv + 2.0 * kxg * kap + kap * kap * m;
                con_minv[w] = minv;
                con_mu[w] = m;
                con_kxb[w] = kxb;
                con_kap[w] = kap;
                const bool valid = minv > 0.0 && dl == dl;  // positive m^{-1}, not NaN
                con_delta[w] = valid ? dl : -CUDART_INF;
                con_key[w] = valid ? order_key(dl) : INT64_MIN;
                if (fused) con_ry[w] = con_y[w] - (j > 0 ? con_dot[2][w] : 0.0);  // y - Y^T K^{-1} k
                con_err[w] = (j >= a.n0 && minv > 0.0 && dl > 0.0)
                                 ? fabsf(con_s32[w] / (float)dl - 1.f) : 0.f;
            }
            __syncthreads();
            if (tid == 0) {
                int wb = 0;
                float e = 0.f;
                for (int w = 0; w < ncon; w++) {
                    if (w > 0 && (con_key[w] > con_key[wb] ||
                                  (con_key[w] == con_key[wb] && con_row[w] < con_row[wb])))
                        wb = w;
                    e = fmaxf(e, con_err[w]);
                }
                if (j >= a.n0) s_err = fmaxf(ERR_DECAY * s_err, e);
                s_win = wb;
                if (con_key[wb] == INT64_MIN) s_bad = LAGP_ENOTPD;
            }
            __syncthreads();
            if (s_bad != LAGP_OK) {
                status = s_bad;
                break;
            }
            // ---------------- FP64 partitioned-inverse update (Sec. 2.2)
            const int wb = s_win, cstar = con_slot[wb];
            {
                const double mu = con_mu[wb];
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
                const double ry = fused ? con_ry[wb] : 0.0;
                for (int t = tid; t < j; t += F32_THREADS) {
                    double gt = -mu * b[t];
                    Kinv[(size_t)t * ld + j] = gt;
                    Kinv[(size_t)j * ld + t] = gt;
                    if (fused) alpha[t] = fma(-mu * ry, b[t], alpha[t]);
                }
                if (tid == 0) {
                    if (fused) {
                        // Eqs. (predgp), (preds2) carried by the same partitioned
                        // inverse: alpha = K^{-1} Y, psi = Y^T K^{-1} Y,
                        // qx = k(x)^T K^{-1} k(x)
                        alpha[j] = mu * ry;
                        yd[j] = con_y[wb];
                        s_psi = fma(mu * ry, ry, s_psi);
                        const double cx = con_kap[wb] - con_kxb[wb];
                        s_qx = fma(mu * cx, cx, s_qx);
                    }
                    Kinv[(size_t)j * ld + j] = mu;
                    kx[j] = con_kap[wb];
                    sel[j] = con_row[wb];
                    if (alc && j >= a.n0) alc[j] = con_delta[wb];
                }
                for (int i = tid; i < p; i += F32_THREADS) xd[(size_t)j * p + i] = con_x[(size_t)wb * p + i];
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
                const float *ustar = con_u + (size_t)wb * ld;
                const float *xs32 = con_c + (size_t)wb * p;
                float acc[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) acc[r] = 0.f;
                const float *Ub = U + c0;
                // loads in flight per thread: UNR rows of CPT floats
                constexpr int UNR = CPT >= 16 ? 2 : 4;
                int i = 0;
                for (; i + UNR <= j; i += UNR) {
                    float u[UNR][CPT];
#pragma unroll
                    for (int q = 0; q < UNR; q++) load_vec<CPT>(Ub + (size_t)(i + q) * Npad, u[q]);
#pragma unroll
                    for (int q = 0; q < UNR; q++) {
                        const float sq = ustar[i + q];
#pragma unroll
                        for (int r = 0; r < CPT; r++) acc[r] = fmaf(u[q][r], sq, acc[r]);
                    }
                }
                for (; i < j; i++) {
                    float u0[CPT];
                    load_vec<CPT>(Ub + (size_t)i * Npad, u0);
                    const float s0 = ustar[i];
#pragma unroll
                    for (int r = 0; r < CPT; r++) acc[r] = fmaf(u0[r], s0, acc[r]);
                }
                float s[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) s[r] = 0.f;
                for (int ii = 0; ii < p; ii++) {
                    float cv[CPT];
                    load_vec<CPT>(Cg + (size_t)ii * Npad + c0, cv);
                    const float xi = xs32[ii];
#pragma unroll
                    for (int r = 0; r < CPT; r++) {
                        float df = cv[r] - xi;
                        s[r] = fmaf(df, df, s[r]);
                    }
                }
                float un[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) {
                    const float kcs = __expf(-s[r] * inv_d);  // K(x_c, x*), no nugget
                    un[r] = (kcs - acc[r]) * inv_lam;
                    v[r] = fmaf(-un[r], un[r], v[r]);
                    cov[r] = fmaf(-wnew, un[r], cov[r]);
                    score[r] = (chosen >> r & 1u) ? -1.f : cov[r] * cov[r] / fmaxf(v[r], gf);
                }
                store_vec<CPT>(U + (size_t)j * Npad + c0, un);
                float wm = -FLT_MAX;
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (!(chosen >> r & 1u)) wm = fmaxf(wm, score[r]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(LAGP_FULL_MASK, wm, o));
                if (lane == 0) w_max[warp] = wm;
            }
            // the next step's selection starts with a barrier, which orders
            // column j of U and the per-warp maxima before their readers
        }
        if (status != LAGP_OK) {
            for (int t = tid; t < nmax; t += F32_THREADS) {
                sel[t] = -1;
                if (alc) alc[t] = CUDART_NAN;
            }
        }
        __syncthreads();
        if (fused && warp == 0) {
            double m = 0.0;
            for (int t = lane; t < nm; t += 32) m = fma(kx[t], alpha[t], m);
            m = warp_sum(m);
            if (lane == 0) {
                const bool ok = status == LAGP_OK;
                a.mean[loc] = ok ? m : CUDART_NAN;
                a.s2[loc] = ok ? s_psi * ((1.0 + g) - s_qx) / nm : CUDART_NAN;
                a.df[loc] = ok ? (double)nm : CUDART_NAN;
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
    const size_t smem = ((size_t)a.nmax + 1) * ld * 8 + ld * 8 * 3 + (size_t)a.nmax * a.p * 8 +
                        (size_t)a.p * 8 + (size_t)tmax * ld * 8 * 2 + (size_t)tmax * a.p * 8 +
                        (size_t)tmax * ld * 4 + ((size_t)tmax * a.p + 1) * 4 + 8 +
                        (size_t)std::max(F32_WARPS, tmax) * ld * 8 + (size_t)Npad * 12 + 64;
    if (smem > ctx->smem_optin)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: shared memory exceeded (n_max, p too large)");
    cudaFuncSetAttribute(alc_f32_kernel<CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alc_f32_kernel<CPT>, F32_THREADS, smem);
    int per_sm = alc_ctas_per_sm(ctx, alc_shape_key("alc_f32", CPT, a.nmax, a.p, a.mean != nullptr), 4);
    if (occ > 0 && per_sm > occ) per_sm = occ;
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    if (grid > a.M) grid = a.M;
    if (grid < 1) grid = 1;
    const size_t U_floats = (size_t)grid * a.nmax * Npad, C_floats = (size_t)grid * a.p * Npad;
    const size_t K_doubles = (size_t)grid * Npad;
    float *U = static_cast<float *>(
        lagp_ws(ctx, WS_ALC_PANEL, (U_floats + C_floats) * 4 + K_doubles * 8 + 256));
    int *counter = static_cast<int *>(lagp_ws(ctx, WS_ALC_COUNTER, 256));
    if (!U || !counter) return LAGP_ENOMEM;
    LAGP_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), st));
    double *Kw = reinterpret_cast<double *>(U + U_floats + C_floats);  // 8-byte aligned: floats counts are even
    F32Params P{a, counter, U, U + U_floats, Kw, Npad, tmax, (float)ctx->tuning.rescore_rel};
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
