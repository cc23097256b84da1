// a2..a6 in the Schur-complement (incremental) form with the candidate state
// in FP64 -- the FP64 Schur form of the greedy ALC local design search
// (Fig. 1 step 2 of the paper) -- or in FP32 (the FP32-bulk form with FP64
// decisions and FP64 inverse update), and every decision in FP64.  (The FP32
// state with the decisions in double-float is alc_bulk32.cu.)
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
// direct form is O(j^2)); in FP32 its rounding error is ~j 2^-24 absolute,
// in FP64 ~j 2^-53.
//
// Each step: FP32 roundings of the FP64 scores r^2 / v -> contenders (scores
// within a margin of the maximum, at most rescore_max; the FP32 rounding
// alone separates them from the exact scores, so the margin floor is 1e-5
// and one contender is the rule) -> FP64 re-score of the contenders with the
// three-term Eq. (dxy) against FP64 K_j^{-1} -> argmax (ties to the lower
// row) -> FP64 partitioned-inverse update of K_j^{-1} (Sec. 2.2) -> the bulk
// recurrence with pivot x*, whose lambda and r_{x*} come from the pivot's own
// bulk state (self-consistent factor).
//
// Layout: one persistent CTA per location at a time (atomic work counter),
// several CTAs per SM so that one location's serial FP64 phases overlap
// other locations' bulk passes; candidate c lives in thread c / CPT, register
// slot c % CPT (v, r, score); the whitened panel U[i][c] and the candidate
// coordinates C[i][c] are per-CTA global buffers (contiguous in c, vector
// loads, L2-resident); K_j^{-1} (with a = K^{-1} k(x) and alpha = K^{-1} Y
// beside it), k_j(x), the design coordinates and the contenders' FP64
// vectors sit in shared memory.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "alc_common.cuh"
#include "device_util.cuh"
#include "exp64.cuh"
#include "lagp_internal.h"

namespace {

constexpr int F32_THREADS = 256;
constexpr int F32_WARPS = F32_THREADS / 32;
// Contender margin: FP32 scores within `margin` (relative) of the FP32
// maximum are re-scored in FP64, margin = min(rescore_rel,
// max(MARGIN_MIN_F64STATE, MARGIN_KAPPA * err)), where err is the largest
// relative FP32-vs-FP64 score error seen among the contenders re-scored so
// far, decaying by ERR_DECAY per step (starting at ERR_INIT).
// with FP64 state the FP32 scores only round (the state is exact to FP64
// rounding), so the margin's floor is a few FP32 ulps
constexpr float MARGIN_MIN_F64STATE = 1e-5f;
// with FP32 state the FP32 scores carry the recurrence's own error
constexpr float MARGIN_MIN_F32STATE = 0.02f;
constexpr float MARGIN_KAPPA = 8.0f;
constexpr float ERR_DECAY = 0.75f;
constexpr float ERR_INIT = 0.05f;

using alc::load_vec;
using alc::store_vec;
using alc::order_key;
using alc::warp_best3;

// K = exp(a) for the bulk state (table method)
__device__ __forceinline__ double bulk_exp(double a, const double *etab) { return exp64_tang(a, etab); }
__device__ __forceinline__ float bulk_exp(float a, const double *) { return __expf(a); }

// FP32 screening score r^2 / v of the FP64 bulk state
__device__ __forceinline__ float bulk_score(float cov, float v, float gf) { return cov * cov / fmaxf(v, gf); }
__device__ __forceinline__ float bulk_score(double cov, double v, float gf) {
    const float c = (float)cov;
    return c * c / fmaxf((float)v, gf);
}

struct F32Params {
    AlcArgs a;
    int *counter;
    unsigned long long *work;  // 4 counters: locations, sum ncon, sum ncon*j, sum ncon*j^2
    void *U_ws;       // per CTA: nmax x Npad of T (whitened panel U[i][c])
    void *C_ws;       // per CTA: p x Npad of T (candidate coordinates C[i][c])
    int Npad;         // F32_THREADS * CPT
    int num_sms;      // the co-resident CTAs of an SM are blockIdx.x, + num_sms, + 2 num_sms, ...
    int tmax;         // rescore_max
    float rel;        // rescore_rel (cap of the contender margin)
    int etab_smem;    // 1: the exp table copied to shared memory; 0: read through L1 (when
                      // the copy would cost the SM a resident CTA)
};

// Contenders kept in the first (static) part of the appended list; at least
// the largest rescore_max.
constexpr int LCAP = 32;

// Rows [k0, k1) of the contraction with the symmetric K^{-1} and the two
// vectors stored beside it: lane t writes sum_{kk in [k0,k1)} S[kk][t] kc[kk]
// for its columns t = lane + 32 r < jo, where S[kk][t] is K^{-1} for t < j,
// a = K^{-1} k_j(x) for t = j and alpha = K^{-1} Y_j for t = j + 1.
template <int JQ>
__device__ __forceinline__ void partial_contract(const double *kc, const double *Kinv, int ld, int k0,
                                                 int k1, int jo, int lane, double *out) {
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
        if (lane + 32 * r < jo) out[lane + 32 * r] = b0[r] + b1[r];
}

// resident CTAs per SM: two for up to 4 candidate slots a thread, one for
// the wider variants.  T is the type of the bulk state (U, v, r and the
// candidate coordinates): double.
template <typename T, int CPT>
constexpr int bulk_min_blocks() {
    return sizeof(T) == 8 ? (CPT >= 8 ? 1 : 2) : (CPT >= 16 ? 2 : (CPT >= 8 ? 3 : 4));
}

template <int CPT, typename T>
__global__ void __launch_bounds__(F32_THREADS, bulk_min_blocks<T, CPT>())
alc_bulk_kernel(F32Params P) {
    const AlcArgs &a = P.a;
    // retry of the FP32-bulk form's failed locations: nothing to do
    if (a.retry_count && *static_cast<const volatile int *>(a.retry_count) == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, Npmax = a.Npmax, Npad = P.Npad, tmax = P.tmax;
    const bool fused = a.mean != nullptr;
    const int extra = fused ? 2 : 1;        // columns of a (and alpha) beside K^{-1}
    const int ld = (nmax + 3) & ~1;         // >= nmax + 2, even
    double *Kinv = reinterpret_cast<double *>(smem_raw);        // (nmax+1) x ld
    double *kx = Kinv + (size_t)(nmax + 1) * ld;                // nmax (even): k_j(x)
    double *xd = kx + ((nmax + 1) & ~1);                        // nmax x p: design coordinates
    double *xq = xd + (size_t)nmax * p;                         // p (even): reference location
    double *etab_s = xq + ((p + 1) & ~1);                       // EXP64_TABLE_SIZE (or 0): exp table
    double *con_k = etab_s + (P.etab_smem ? EXP64_TABLE_SIZE : 0);  // tmax x ld: k_j(x_c), FP64
    double *con_b = con_k + (size_t)tmax * ld;                  // tmax x ld: K^{-1} k_j(x_c)
    double *cpart = con_b + (size_t)tmax * ld;                  // max(8,tmax) x ld partials;
                                                                // row 0 then holds mu b of the winner
    // the appended list beyond its first LCAP entries shares the space of
    // con_k.. (it is dead before the re-score starts)
    float *ov_s = reinterpret_cast<float *>(con_k);
    int *ov_slot = reinterpret_cast<int *>(ov_s + Npad);
    const size_t union_doubles =
        max((size_t)Npad, ((size_t)2 * tmax + max(F32_WARPS, tmax)) * ld);
    T *w_u = reinterpret_cast<T *>(con_k + union_doubles);  // ld: U column of the winner
    T *w_c = w_u + ld;                                        // p: its coordinates
    double *mb = cpart;

    __shared__ int s_loc, s_bad, s_total, s_wl;
    __shared__ float w_max[F32_WARPS];
    __shared__ int lst_slot[LCAP], lst_row[LCAP], top_slot[LCAP], top_row[LCAP];
    __shared__ float lst_s[LCAP], top_s[LCAP];
    __shared__ double con_kap[LCAP], con_y[LCAP], con_quad[LCAP], con_kxb[LCAP], con_yb[LCAP];
    __shared__ double con_mu[LCAP], con_dl[LCAP], con_ry[LCAP];
    __shared__ long long con_key[LCAP];
    __shared__ float con_err[LCAP];
    __shared__ double s_mu, s_ex, s_ry, s_kap, s_kxb, s_dl, s_psi, s_qx;
    __shared__ T s_invlam, s_wnew;
    __shared__ float s_err;
    __shared__ unsigned long long s_work[4];

    T *U = static_cast<T *>(P.U_ws) + (size_t)blockIdx.x * nmax * Npad;
    T *Cg = static_cast<T *>(P.C_ws) + (size_t)blockIdx.x * p * Npad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = tid * CPT;  // first candidate slot of this thread
    // warp roles rotate with the CTA's residency slot on its SM (the CTAs
    // sharing an SM are blockIdx.x = i, i + num_sms, ...), so that the
    // co-resident CTAs' serial FP64 phases run on different sub-partitions
    // (warp w runs on sub-partition w mod 4)
    const int rot = (blockIdx.x / P.num_sms) & 3;
    const int lead = 32 * rot;  // the thread with the CTA's scalar duties
    const double *etab = P.etab_smem ? etab_s : exp64_table_g;  // table of exp64_tang
    if (P.etab_smem)
        for (int i = tid; i < EXP64_TABLE_SIZE; i += F32_THREADS) etab_s[i] = exp64_table_g[i];
    if (tid < 4) s_work[tid] = 0ull;

    for (;;) {
        if (tid == 0) s_loc = atomicAdd(P.counter, 1);
        __syncthreads();
        const int64_t loc = s_loc;
        __syncthreads();
        if (loc >= a.M) break;
        if (a.retry_count && a.status[loc] != LAGP_ENOTPD) continue;  // (retry: failed locations only)

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

        // ---- per-location set-up: coordinates and the initial FP32 state
        for (int i = tid; i < p; i += F32_THREADS) xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
        for (int e = tid; e < p * Npad; e += F32_THREADS) {
            int i = e / Npad, c = e - i * Npad;
            if constexpr (sizeof(T) == 8) Cg[e] = c < k ? load_coord64(a.X, cands[c], p, i, a.dtype) : 0.0;
            else Cg[e] = c < k ? load_coord32(a.X, cands[c], p, i, a.dtype) : 0.f;
        }
        const double inv_d64 = 1.0 / d, onepg = 1.0 + g;
        if (tid == 0) {
            s_err = ERR_INIT;
            s_psi = 0.0;
            s_qx = 0.0;
            s_total = 0;
            s_work[0] += 1ull;
        }
        __syncthreads();
        const T inv_d = (T)(1.0 / d);
        const float gf = fmaxf((float)g, FLT_MIN);  // floor of v in the FP32 scores
        const T gT = sizeof(T) == 8 ? (T)fmax(g, DBL_MIN) : (T)fmaxf((float)g, FLT_MIN);
        T v[CPT], cov[CPT];
        float score[CPT];
        int rows[CPT];  // design rows of this thread's candidates (tie-break key)
        unsigned chosen = 0;
        {
            T s[CPT];
#pragma unroll
            for (int r = 0; r < CPT; r++) s[r] = T(0);
            for (int i = 0; i < p; i++) {
                T cv[CPT];
                load_vec<CPT>(Cg + (size_t)i * Npad + c0, cv);
                const T qi = (T)xq[i];
#pragma unroll
                for (int r = 0; r < CPT; r++) {
                    T df = cv[r] - qi;
                    s[r] = fma(df, df, s[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < CPT; r++) {
                const int c = c0 + r;
                rows[r] = c < k ? cands[c] : INT32_MAX;
                v[r] = (T)onepg;
                cov[r] = bulk_exp(-s[r] * inv_d, etab);  // K(x_c, x), no nugget
                score[r] = c < k ? bulk_score(cov[r], v[r], gf) : -1.f;
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
        for (int j = 0; j < nm; j++) {
            const int jo = j + extra;  // outputs of the contraction: K^{-1} k, a^T k (, alpha^T k)
            // ---------------- contenders for design index j.  The barrier
            // orders the last FP32 pass (per-warp maxima, column j-1 of U) and
            // the last update before everything below.
            __syncthreads();
            if (j < a.n0) {
                if (tid == lead) {
                    lst_slot[0] = j;  // Fig. 1 step 2(a): nearest neighbours in order
                    lst_row[0] = cands[j];
                    lst_s[0] = 0.f;
                    s_total = 1;
                }
            } else {
                const float margin =
                    fminf(P.rel, fmaxf(sizeof(T) == 8 ? MARGIN_MIN_F64STATE : MARGIN_MIN_F32STATE,
                                       MARGIN_KAPPA * s_err));
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
                const int wtot = __shfl_sync(LAGP_FULL_MASK, incl, 31);
                int base = 0;
                if (lane == 31 && wtot > 0) base = atomicAdd(&s_total, wtot);
                base = __shfl_sync(LAGP_FULL_MASK, base, 31);
                // list order depends on the warps' arrival; the contender set,
                // and every result, does not
                int pos = base + incl - mine;
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (flags >> r & 1u) {
                        if (pos < LCAP) {
                            lst_s[pos] = score[r];
                            lst_slot[pos] = c0 + r;
                            lst_row[pos] = rows[r];
                        } else {
                            ov_s[pos] = score[r];
                            ov_slot[pos] = c0 + r;
                        }
                        pos++;
                    }
            }
            __syncthreads();
            const int total = s_total;
            if (total > tmax) {  // keep the best tmax by FP32 score, ties to the lower row
                if (warp == 0) {
                    for (int t = 0; t < tmax; t++) {
                        float bs = -FLT_MAX;
                        int brow = INT32_MAX, bpos = -1;
                        for (int e = lane; e < total; e += 32) {
                            const int sl = e < LCAP ? lst_slot[e] : ov_slot[e];
                            if (sl < 0) continue;
                            const float sc = e < LCAP ? lst_s[e] : ov_s[e];
                            const int rw = e < LCAP ? lst_row[e] : cands[sl];
                            if (sc > bs || (sc == bs && rw < brow)) {
                                bs = sc;
                                brow = rw;
                                bpos = e;
                            }
                        }
                        warp_best3(bs, brow, bpos);
                        if (bpos < 0) break;
                        if (lane == 0) {
                            const bool lo = bpos < LCAP;
                            top_slot[t] = lo ? lst_slot[bpos] : ov_slot[bpos];
                            top_row[t] = brow;
                            top_s[t] = bs;
                            if (lo) lst_slot[bpos] = -1;
                            else ov_slot[bpos] = -1;
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();
            }
            const int ncon = min(total, tmax);
            const int *cslot = total > tmax ? top_slot : lst_slot;
            const int *crow = total > tmax ? top_row : lst_row;
            const float *cs32 = total > tmax ? top_s : lst_s;
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
            // R1: k_j(x_c) and K(x_c, x) in FP64, (contender, design row) pairs
            // packed over lanes; coordinates straight from the design
            {
                const int jp = j + 1;
                const int te = (tid + 32 * rot) & (F32_THREADS - 1);
                for (int e = te; e < ncon * jp; e += F32_THREADS) {
                    const int w = e / jp, t = e - w * jp;
                    const int32_t row = crow[w];
                    const double *xt = t < j ? xd + (size_t)t * p : xq;
                    double s0 = 0.0, s1 = 0.0;
                    int i = 0;
                    for (; i + 2 <= p; i += 2) {
                        const double d0 = load_coord64(a.X, row, p, i, a.dtype) - xt[i];
                        const double d1 = load_coord64(a.X, row, p, i + 1, a.dtype) - xt[i + 1];
                        s0 = fma(d0, d0, s0);
                        s1 = fma(d1, d1, s1);
                    }
                    if (i < p) {
                        const double d0 = load_coord64(a.X, row, p, i, a.dtype) - xt[i];
                        s0 = fma(d0, d0, s0);
                    }
                    const double kv = exp64_tang(-(s0 + s1) * inv_d64, etab);
                    if (t < j) {
                        con_k[(size_t)w * ld + t] = kv;
                    } else {
                        con_kap[w] = kv;
                        if (fused)
                            con_y[w] = a.dtype == LAGP_F64 ? static_cast<const double *>(a.Y)[row]
                                                           : (double)static_cast<const float *>(a.Y)[row];
                    }
                }
            }
            __syncthreads();
            // R2: partial contractions [K^{-1} | a | alpha]^T k_j(x_c), each
            // contender's rows split over wpc warps (two for one or two
            // contenders, else one).  Every split costs FP64 instructions (the
            // partials' sums) on the unit that bounds the kernel, so the split
            // stays small: two halves shorten the chain without costing more.
            const int wpc = ncon >= 3 ? 1 : 2;
            if (j > 0) {
                const int nrows = max(F32_WARPS, tmax);  // rows of cpart
                for (int job = we; job < ncon * wpc && job < nrows; job += F32_WARPS) {
                    const int w = job / wpc, part = job - w * wpc;
                    const int k0 = part * j / wpc, k1 = (part + 1) * j / wpc;
                    const double *kc = con_k + (size_t)w * ld;
                    double *out = cpart + (size_t)job * ld;
                    switch ((jo + 31) >> 5) {
                        case 1: partial_contract<1>(kc, Kinv, ld, k0, k1, jo, lane, out); break;
                        case 2: partial_contract<2>(kc, Kinv, ld, k0, k1, jo, lane, out); break;
                        case 3: partial_contract<3>(kc, Kinv, ld, k0, k1, jo, lane, out); break;
                        case 4: partial_contract<4>(kc, Kinv, ld, k0, k1, jo, lane, out); break;
                        default: partial_contract<5>(kc, Kinv, ld, k0, k1, jo, lane, out); break;
                    }
                }
            }
            __syncthreads();
            // R3: sum of the partials (first half + second half): b = K^{-1} k,
            // a^T k, alpha^T k; then k^T b, one warp per contender
            for (int w = we; w < ncon; w += F32_WARPS) {
                if (j == 0) {
                    if (lane == 0) con_quad[w] = con_kxb[w] = con_yb[w] = 0.0;
                    continue;
                }
                const double *P0 = cpart + (size_t)w * wpc * ld;
                double acc = 0.0;
                for (int t = lane; t < jo; t += 32) {
                    const double bt = wpc == 1 ? P0[t] : P0[t] + P0[ld + t];
                    if (t < j) {
                        con_b[(size_t)w * ld + t] = bt;
                        acc = fma(con_k[(size_t)w * ld + t], bt, acc);
                    } else if (t == j) {
                        con_kxb[w] = bt;
                    } else {
                        con_yb[w] = bt;
                    }
                }
                acc = warp_sum(acc);
                if (lane == 0) con_quad[w] = acc;
            }
            __syncthreads();
            // R4, in the lanes of the lead warp (one contender a lane: the FP64
            // unit takes a warp instruction whatever the number of active lanes,
            // so the contenders' scalars share instructions): the scalars of
            // Eqs. (piedef), (dxy), the winner (largest FP64 value, ties to the
            // lower row) by integer keys, and mu b of the winner
            if (warp == rot) {
                if (lane < ncon) {
                    const int w = lane;
                    const double quad = con_quad[w], kxb = con_kxb[w], kap = con_kap[w];
                    const double minv = onepg - quad;  // m_j^{-1}(x_c)
                    const double m = 1.0 / minv;
                    const double kxg = -m * kxb;       // k_j(x)^T g_j(x_c)
                    const double dl = kxg * kxg * minv + 2.0 * kxg * kap + kap * kap * m;
                    const bool valid = minv > 0.0 && dl == dl;  // positive m^{-1}, not NaN
                    con_key[w] = valid ? order_key(dl) : INT64_MIN;
                    con_mu[w] = m;
                    con_dl[w] = dl;
                    if (fused) con_ry[w] = con_y[w] - con_yb[w];  // y - Y^T K^{-1} k
                    con_err[w] = (j >= a.n0 && minv > 0.0 && dl > 0.0) ? fabsf(cs32[w] / (float)dl - 1.f) : 0.f;
                }
                __syncwarp();
                long long key = INT64_MIN;
                int row = INT32_MAX;
                float err = 0.f;
                if (lane < ncon) {
                    key = con_key[lane];
                    row = crow[lane];
                    err = con_err[lane];
                }
                int wl = lane;
                long long bk = key;
                int brow = row;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long ok = __shfl_xor_sync(LAGP_FULL_MASK, bk, o);
                    const int orow = __shfl_xor_sync(LAGP_FULL_MASK, brow, o);
                    const int owl = __shfl_xor_sync(LAGP_FULL_MASK, wl, o);
                    if (ok > bk || (ok == bk && orow < brow)) {
                        bk = ok;
                        brow = orow;
                        wl = owl;
                    }
                    err = fmaxf(err, __shfl_xor_sync(LAGP_FULL_MASK, err, o));
                }
                const double mu = con_mu[wl];
                const double *b = con_b + (size_t)wl * ld;
                for (int t = lane; t < j; t += 32) mb[t] = mu * b[t];
                if (lane == 0) {
                    const double kap = con_kap[wl], kxb = con_kxb[wl];
                    s_wl = wl;
                    s_mu = mu;
                    s_kap = kap;
                    s_kxb = kxb;
                    s_ex = mu * (kap - kxb);  // new entry of a = K^{-1} k(x)
                    s_ry = fused ? con_ry[wl] : 0.0;
                    s_dl = con_dl[wl];
                    if (j >= a.n0) s_err = fmaxf(ERR_DECAY * s_err, err);
                    if (bk == INT64_MIN) s_bad = LAGP_ENOTPD;
                    s_work[1] += (unsigned long long)ncon;
                    s_work[2] += (unsigned long long)ncon * j;
                    s_work[3] += (unsigned long long)ncon * j * j;
                }
            }
            __syncthreads();
            if (s_bad != LAGP_OK) {
                status = s_bad;
                break;
            }
            // ---------------- FP64 partitioned-inverse update (Sec. 2.2) of K^{-1}
            // and of the vectors a = K^{-1} k(x), alpha = K^{-1} Y beside it
            const int wl = s_wl, cstar = cslot[wl], rstar = crow[wl];
            {
                // the winner's U column, FP32 and FP64 coordinates (next pivot)
                for (int t = tid; t < j; t += F32_THREADS) w_u[t] = U[(size_t)t * Npad + cstar];
                for (int i = tid; i < p; i += F32_THREADS) {
                    w_c[i] = Cg[(size_t)i * Npad + cstar];
                    xd[(size_t)j * p + i] = load_coord64(a.X, rstar, p, i, a.dtype);
                }
                const double *b = con_b + (size_t)wl * ld;
                // lower triangle with its mirror: K^{-1} += (mu b) b^T
                for (int e = tid; e < j * (j + 1) / 2; e += F32_THREADS) {
                    int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
                    while ((r + 1) * (r + 2) / 2 <= e) r++;
                    while (r * (r + 1) / 2 > e) r--;
                    const int c = e - r * (r + 1) / 2;
                    const double val = fma(mb[r], b[c], Kinv[(size_t)r * ld + c]);
                    Kinv[(size_t)r * ld + c] = val;
                    Kinv[(size_t)c * ld + r] = val;
                }
                const double ex = s_ex, ry = s_ry;
                for (int t = tid; t < j; t += F32_THREADS) {
                    double *Kt = Kinv + (size_t)t * ld;
                    const double a_old = Kt[j];
                    const double al_old = fused ? Kt[j + 1] : 0.0;
                    const double gt = -mb[t];
                    Kt[j] = gt;
                    Kinv[(size_t)j * ld + t] = gt;
                    Kt[j + 1] = fma(-ex, b[t], a_old);          // a - e_x b
                    if (fused) Kt[j + 2] = fma(-ry, mb[t], al_old);  // alpha - mu r_y b
                }
                if (tid == lead) {
                    const double mu = s_mu;
                    double *Kj = Kinv + (size_t)j * ld;
                    Kj[j] = mu;
                    Kj[j + 1] = ex;
                    if (fused) {
                        // Eqs. (predgp), (preds2) carried by the same partitioned
                        // inverse: alpha = K^{-1} Y, psi = Y^T K^{-1} Y,
                        // qx = k(x)^T K^{-1} k(x)
                        Kj[j + 2] = mu * ry;
                        s_psi = fma(mu * ry, ry, s_psi);
                        const double cx = s_kap - s_kxb;
                        s_qx = fma(mu * cx, cx, s_qx);
                    }
                    kx[j] = s_kap;
                    sel[j] = rstar;
                    if (alc && j >= a.n0) alc[j] = s_dl;
                    s_total = 0;
                }
            }
            // The bulk recurrence continues from the pivot's own bulk state:
            // lambda^2 = v_{x*} and r_{x*}, so that U stays the Cholesky factor
            // of one (slightly perturbed) matrix; mixing in the FP64 values
            // breaks that consistency and the recurrence drifts.
#pragma unroll
            for (int r = 0; r < CPT; r++)
                if (c0 + r == cstar) {
                    const T vs = v[r] > gT ? v[r] : gT;
                    T il;
                    if constexpr (sizeof(T) == 8) il = 1.0 / sqrt(vs);
                    else il = rsqrtf(vs);
                    s_invlam = il;
                    s_wnew = cov[r] * il;
                    chosen |= 1u << r;
                }
            __syncthreads();
            if (j + 1 >= nm) break;
            // ---------------- FP32 Schur recurrence with pivot x* (new column j of U)
            {
                const T inv_lam = s_invlam;
                const T wnew = s_wnew;
                T acc[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) acc[r] = T(0);
                const T *Ub = U + c0;
                // loads in flight per thread: UNR rows of CPT values
                constexpr int UNR = (sizeof(T) == 8 || CPT >= 16) ? 2 : 6;
                int i = 0;
                for (; i + UNR <= j; i += UNR) {
                    T u[UNR][CPT];
#pragma unroll
                    for (int q = 0; q < UNR; q++) load_vec<CPT>(Ub + (size_t)(i + q) * Npad, u[q]);
#pragma unroll
                    for (int q = 0; q < UNR; q++) {
                        const T sq = w_u[i + q];
#pragma unroll
                        for (int r = 0; r < CPT; r++) acc[r] = fma(u[q][r], sq, acc[r]);
                    }
                }
                for (; i < j; i++) {
                    T u0[CPT];
                    load_vec<CPT>(Ub + (size_t)i * Npad, u0);
                    const T s0 = w_u[i];
#pragma unroll
                    for (int r = 0; r < CPT; r++) acc[r] = fma(u0[r], s0, acc[r]);
                }
                T s[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) s[r] = T(0);
                for (int ii = 0; ii < p; ii++) {
                    T cv[CPT];
                    load_vec<CPT>(Cg + (size_t)ii * Npad + c0, cv);
                    const T xi = w_c[ii];
#pragma unroll
                    for (int r = 0; r < CPT; r++) {
                        T df = cv[r] - xi;
                        s[r] = fma(df, df, s[r]);
                    }
                }
                T un[CPT];
#pragma unroll
                for (int r = 0; r < CPT; r++) {
                    const T kcs = bulk_exp(-s[r] * inv_d, etab);  // K(x_c, x*), no nugget
                    un[r] = (kcs - acc[r]) * inv_lam;
                    v[r] = fma(-un[r], un[r], v[r]);
                    cov[r] = fma(-wnew, un[r], cov[r]);
                    score[r] = (chosen >> r & 1u) ? -1.f : bulk_score(cov[r], v[r], gf);
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
        }
        if (status != LAGP_OK) {
            for (int t = tid; t < nmax; t += F32_THREADS) {
                sel[t] = -1;
                if (alc) alc[t] = CUDART_NAN;
            }
        }
        __syncthreads();
        if (fused && warp == 0) {
            // mean = k(x)^T alpha; alpha sits in column nm + 1 after the last update
            double m = 0.0;
            for (int t = lane; t < nm; t += 32) m = fma(kx[t], Kinv[(size_t)t * ld + nm + 1], m);
            m = warp_sum(m);
            if (lane == 0) {
                const bool ok = status == LAGP_OK;
                a.mean[loc] = ok ? m : CUDART_NAN;
                a.s2[loc] = ok ? s_psi * (onepg - s_qx) / nm : CUDART_NAN;
                a.df[loc] = ok ? (double)nm : CUDART_NAN;
            }
        }
        if (tid == 0) {
            a.status[loc] = status;
            if (status == LAGP_ENOTPD && a.fail_count) atomicAdd(a.fail_count, 1);  // (the FP64 Schur retry)
        }
        __syncthreads();
    }
    if (tid < 4 && P.work) atomicAdd(P.work + tid, s_work[tid]);
}

template <int CPT, typename T>
lagp_status launch_cpt(lagp_ctx *ctx, const AlcArgs &a) {
    cudaStream_t st = ctx->stream;
    const int Npad = F32_THREADS * CPT;
    const int tmax = ctx->tuning.rescore_max > 0 ? ctx->tuning.rescore_max : 8;
    // dynamic shared memory, in the kernel's order (see alc_bulk_kernel)
    const size_t nmax = (size_t)a.nmax, p = (size_t)a.p;
    const size_t ld = (nmax + 3) & ~(size_t)1;
    const size_t union_doubles = std::max((size_t)Npad, (2 * (size_t)tmax + std::max(F32_WARPS, tmax)) * ld);
    const size_t smem_notab = 8 * ((nmax + 1) * ld + ((nmax + 1) & ~(size_t)1) + nmax * p +
                                   ((p + 1) & ~(size_t)1) + union_doubles) +
                              sizeof(T) * (ld + p);
    const size_t smem_tab = smem_notab + 8 * (size_t)EXP64_TABLE_SIZE;
    if (smem_notab > ctx->smem_optin)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: shared memory exceeded (n_max, p too large)");
    // the exp table goes to shared memory unless that costs a resident CTA
    // (large n_max: the table's 8 KB decide between one and two CTAs an SM)
    int occ = 0, occ_notab = 0;
    cudaFuncSetAttribute(alc_bulk_kernel<CPT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)std::min(smem_tab, (size_t)ctx->smem_optin));
    if (smem_tab <= ctx->smem_optin)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alc_bulk_kernel<CPT, T>, F32_THREADS, smem_tab);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_notab, alc_bulk_kernel<CPT, T>, F32_THREADS, smem_notab);
    const int etab_smem = occ > 0 && occ >= occ_notab ? 1 : 0;
    const size_t smem = etab_smem ? smem_tab : smem_notab;
    if (!etab_smem) occ = occ_notab;
    const bool f64state = sizeof(T) == 8;
    int per_sm = alc_ctas_per_sm(ctx, alc_shape_key(f64state ? "alc_f64schur" : "alc_f32x64", CPT, a.nmax, a.p,
                                                    a.mean != nullptr),
                                 f64state ? 2 : 4);
    if (occ > 0 && per_sm > occ) per_sm = occ;
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    if (grid > a.M) grid = a.M;
    if (grid < 1) grid = 1;
    const size_t U_elems = (size_t)grid * a.nmax * Npad, C_elems = (size_t)grid * a.p * Npad;
    T *U = static_cast<T *>(lagp_ws(ctx, WS_ALC_PANEL, (U_elems + C_elems) * sizeof(T) + 256));
    int *counter = nullptr;
    unsigned long long *work = nullptr;
    LAGP_TRY(alc_counters(ctx, &counter, &work));
    if (!U) return LAGP_ENOMEM;
    LAGP_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), st));
    F32Params P{a, counter, work, U, U + U_elems, Npad, ctx->num_sms, tmax, (float)ctx->tuning.rescore_rel,
                etab_smem};
    alc_bulk_kernel<CPT, T><<<(unsigned)grid, F32_THREADS, smem, st>>>(P);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

template <typename T>
lagp_status launch_bulk(lagp_ctx *ctx, const AlcArgs &a) {
    if (a.nmax > 128)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: n_max above 128 is not supported");
    const int need = (a.Npmax + F32_THREADS - 1) / F32_THREADS;
    if (need <= 1) return launch_cpt<1, T>(ctx, a);
    if (need <= 2) return launch_cpt<2, T>(ctx, a);
    if (need <= 4) return launch_cpt<4, T>(ctx, a);
    if (need <= 8) return launch_cpt<8, T>(ctx, a);
    return launch_cpt<16, T>(ctx, a);
}

}  // namespace

lagp_status launch_alc_f64schur(lagp_ctx *ctx, const AlcArgs &a) { return launch_bulk<double>(ctx, a); }
lagp_status launch_alc_f32x64(lagp_ctx *ctx, const AlcArgs &a) { return launch_bulk<float>(ctx, a); }
