// a2..a7 in the Schur-complement (incremental) form with the candidate state
// in FP32 -- the FP32-bulk form of the greedy ALC local design search
// (Fig. 1 step 2 of the paper) -- with every decision, and the growing
// inverse, in double-float arithmetic on the FP32 pipes.
//
// The criterion.  Eq. (dxy) with g_j, m_j of Eq. (piedef) simplifies
// exactly to Delta_c = (K(x_c,x) - k_j(x)^T K_j^{-1} k_j(x_c))^2 m_j, with
// m_j^{-1} = 1 + g - k_j(x_c)^T K_j^{-1} k_j(x_c).  With K_j = L_j L_j^T and
//   u_c = L_j^{-1} k_j(x_c),   w = L_j^{-1} k_j(x),   z = L_j^{-1} Y_j,
// the two quadratic forms are |u_c|^2 and w^T u_c, so
//   v_c = m_j^{-1} = 1 + g - |u_c|^2,  r_c = K(x_c,x) - w^T u_c,
//   Delta_c = r_c^2 / v_c.
// K_j^{-1} = L_j^{-T} L_j^{-1} grows by the partitioned inverse of the
// bordered factor: with x* chosen, u* = L_j^{-1} k_j(x*), lambda^2 = v_{x*}
// and b = L_j^{-T} u* = K_j^{-1} k_j(x*) (the b of Eq. piedef's g_j = -m_j b),
//   L_{j+1}^{-1} = [[L_j^{-1}, 0], [-b^T / lambda, 1 / lambda]],
// and w, z gain the entries r_{x*} / lambda and (y* - z^T u*) / lambda.  The
// predictive equations (Eqs. predgp, preds2) follow on the chosen design:
// mean = w^T z, psi = |z|^2, s2 = psi (1 + g - |w|^2) / n.
//
// Why this basis, and why double-float: on this GPU an FP64 warp
// instruction (or a double <-> float conversion) holds its sub-partition's
// FP64 unit for ~64 cycles whatever the number of active lanes, so the
// re-score runs in double-float (~48 significant bits, 3..20 FP32
// instructions an operation).  In the K^{-1} basis the quadratic form
// k^T K^{-1} k carries an absolute error of about cond(K_j) times the unit
// roundoff (cond ~1e5..1e7 here): at 2^-48 that broke the 1e-6 parity bars
// (an ALC value 7.9e-6 off, a prediction 1.1e-6 off, measured); in the
// Cholesky basis the error is about sqrt(cond(K_j)) times the unit roundoff,
// smaller than FP64 in the K^{-1} basis.
//
// The FP32 bulk state, per candidate: the same u_c, v_c, r_c in FP32, u_c in
// the per-CTA whitened panel U[i][c] (L2-resident), v_c and r_c in shared
// memory, updated by the pivot's FP32 column: u_{c,j} = (K(x_c,x*) -
// U_c^T u_{x*}) / lambda, v_c -= u_{c,j}^2, r_c -= (r_{x*}/lambda) u_{c,j}:
// an O(j) dot product per candidate per step (the paper's form is O(j^2)).
// The FP32 recurrence continues from the pivot's own FP32 state (a
// self-consistent factor: mixing in the double-float values makes it
// drift).  The FP32 scores r^2 / v only select the contenders -- those
// within an adaptive margin of the FP32 maximum, all of them -- and no
// decision is taken on them.
//
// Two warp groups per CTA (one location at a time, persistent CTAs with an
// atomic work counter):
//   FP32 group (warps 0-3): owns the candidates (slot c in thread c / CPT);
//     lists the contenders, and runs the Schur pass of each step;
//   double-float group (warps 4-7): re-scores the contenders
//     (R1 k_j(x_c), K(x_c,x): squared distances and Tang's exponential;
//      R2 u_c = L^{-1} k_j(x_c); R3 |u_c|^2, w^T u_c, z^T u_c -> Delta;
//      the argmax, ties to the lower design row), then grows L^{-1}, w, z
//     and the prediction's sums for the winner.
// In a step with a single contender (the common case) the winner is known
// as soon as the list is, so the FP32 group's Schur pass and the
// double-float group's work on the winner run at the same time; with two or
// more contenders the Schur pass waits for the argmax.  The groups meet at
// two CTA barriers a step (three with several contenders); inside the
// double-float group a named barrier orders its phases.
//
// Shared memory holds L^{-1} (transposed, an odd leading dimension so that
// both its row and its column reads are free of bank conflicts, zero below
// the diagonal), w, z, the design coordinates, the contenders' vectors and
// the FP32 v, r of every candidate.
//
// Code size.  A step runs from the instruction cache, and the kernel's
// machine code (110 KB at CPT = 8 with the compiler's own unrolling) did not
// fit: the set-up of a location and the double-float group's per-step phases
// evicted one another.  The loops of the per-location set-up and outputs, of
// the triangular products, of R3, of the argmax of several contenders and of
// the winner's bookkeeping therefore carry `#pragma unroll 1`, and so does
// the Schur pass's loop over the coordinates at CPT <= 8 (77 KB); the rest
// of the Schur pass, the listing, R1 and R2 keep their unrolling, which the
// wide candidate sets (CPT = 16) and the steps with many contenders need.
// Measured on the borehole batch: 11.4 -> 9.4 ms a search, the same designs
// bit for bit.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "alc_common.cuh"
#include "df64.cuh"
#include "device_util.cuh"
#include "exp64.cuh"
#include "lagp_internal.h"

namespace {

using alc::load_vec;
using alc::store_vec;

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int FTHREADS = 128;              // FP32 group: warps 0..3
constexpr int FWARPS = FTHREADS / 32;
constexpr int DTHREADS = THREADS - FTHREADS;  // double-float group: warps 4..7
constexpr int DWARPS = DTHREADS / 32;
// Adaptive contender margin: FP32 scores within `margin` (relative) of the
// FP32 maximum are re-scored, margin = min(rescore_rel, max(MARGIN_MIN,
// MARGIN_KAPPA * err)), err = the largest FP32-vs-double-float score error
// seen among the contenders re-scored so far, relative to the step's best
// score (what decides whether the best can be missed), decaying by ERR_DECAY
// per step (from ERR_INIT, which puts the first margin at its floor: after
// n0 steps of the recurrence the FP32 state is still close to exact, and the
// first re-scores measure its error).
constexpr float MARGIN_MIN = 0.02f;
constexpr float MARGIN_KAPPA = 8.0f;
constexpr float ERR_DECAY = 0.75f;
constexpr float ERR_INIT = MARGIN_MIN / MARGIN_KAPPA;
// contenders kept in the static list; more go to the per-CTA global list
constexpr int LCAP = 32;
// largest batch of contenders re-scored together (batches of 16 took the
// 2-d toy's search 1.59 -> 1.41 ms and the 1M-point workload's 203 -> 192 ms)
constexpr int TMAX_CAP = 16;
// rows of the partial contractions: a warp's, or a batch contender's
__host__ __device__ __forceinline__ int b32_cprows(int tmax) { return tmax > WARPS ? tmax : WARPS; }

struct B32Params {
    AlcArgs a;
    int *counter;
    unsigned long long *work;  // locations, sum ncon, sum ncon*j, sum ncon*j^2
    float *U_ws;               // per CTA: nmax x Npad whitened panel U[i][c]
    float *C_ws;               // per CTA: p x Npad candidate coordinates (FP32, rounded)
    float *Clo_ws;             // per CTA: p x Npad low parts of FP64 coordinates
    float2 *Yc_ws;             // per CTA: Npad double-float responses of the candidates (fused)
    float *ovs_ws;             // per CTA: 3 x Npad: score, FP32 v, FP32 r of contenders beyond LCAP
    int *ovi_ws;               // per CTA: Npad contender slots beyond LCAP
    int num_sms;
    int tmax;                  // batch size, 1..TMAX_CAP
    float rel;                 // cap of the contender margin
};

// leading dimensions of the shared-memory arrays (in elements)
__host__ __device__ __forceinline__ int b32_ldl(int nmax) { return nmax | 1; }         // L^{-T}: odd
__host__ __device__ __forceinline__ int b32_ldc(int nmax) { return (nmax + 2) & ~1; }  // >= nmax + 1
__host__ __device__ __forceinline__ int b32_ldx(int nmax) { return (nmax + 1) & ~1; }  // >= nmax

// the double-float group's barrier (named barrier 1, its 128 threads) and the
// FP32 group's (named barrier 2)
__device__ __forceinline__ void dsync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void fsync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

__device__ __forceinline__ float f32_score(float cov, float v, float gf) {
    return __fdividef(cov * cov, fmaxf(v, gf));
}

// double-float value of element i of an FP64 or FP32 array
__device__ __forceinline__ dfl load_df(const void *A, int64_t i, lagp_dtype dt) {
    if (dt == LAGP_F64) return df_from_double(static_cast<const double *>(A)[i]);
    return dfl{static_cast<const float *>(A)[i], 0.f};
}

__device__ __forceinline__ dfl ld2(const float2 *p) {
    const float2 v = *p;
    return dfl{v.x, v.y};
}
__device__ __forceinline__ void st2(float2 *p, dfl v) { *p = make_float2(v.hi, v.lo); }

// 1 / sqrt(v) of a positive normalised double-word: the FP32 estimate r0
// (relative error ~2^-23) and one Newton step r0 + r0 (1 - v r0^2) / 2, with
// 1 - v r0^2 formed in double-float: relative error a few u^2
__device__ __forceinline__ dfl df_rsqrt(dfl v) {
    const float r0 = rsqrtf(v.hi);
    const dfl e = df_sub(dfl{1.f, 0.f}, df_mul(v, two_prod(r0, r0)));
    return fast_two_sum(r0, 0.5f * r0 * e.hi);
}

// R2: rows s in [s0, s1) of u = L^{-1} k: lane t accumulates
// sum_s LT[s][t] k[s] for t = lane + 32 q < j, written to out.  LT is zero
// below its diagonal, so no term needs a test; one block of 32 outputs at a
// time keeps the code small (it runs from the instruction cache every step).
__device__ __noinline__ void df_tri_lower(const float2 *kc, const float2 *LT, int ldl, int s0, int s1, int j,
                                          int lane, float2 *out) {
    #pragma unroll 1
    for (int t = lane; t < ((j + 31) & ~31); t += 32) {
        if (t < j) {
            dfl acc = df_zero();
            const float2 *row = LT + s0 * ldl + t;
            #pragma unroll 1
            for (int s = s0; s < s1; s++, row += ldl) df_fma_acc(acc, ld2(row), ld2(kc + s));
            st2(out + t, acc);
        }
    }
}

// The winner's b = L^{-T} u* over t in [t0, t1): lane s accumulates
// sum_t LT[s][t] u*[t] for s = lane + 32 q < t1 (zeros below the diagonal
// stand in for the test t >= s); partials of s < t1 written to out
__device__ __noinline__ void df_tri_upper(const float2 *us, const float2 *LT, int ldl, int t0, int t1, int lane,
                                          float2 *out) {
    #pragma unroll 1
    for (int sb = lane; sb < ((t1 + 31) & ~31); sb += 32) {
        if (sb < t1) {
            dfl acc = df_zero();
            const float2 *col = LT + sb * ldl;
            #pragma unroll 1
            for (int t = t0; t < t1; t++) df_fma_acc(acc, ld2(col + t), ld2(us + t));
            st2(out + sb, acc);
        }
    }
}

// The winner's scalars (one warp, uniform; lane 0 stores): 1 / lambda, the
// new entries of w and z (w_j = r / lambda, z_j = (y - z^T u) / lambda), the
// corner of L^{-1}, the prediction's sums psi = |z|^2, |w|^2 and w^T z, the
// design row (the ALC value and the margin's error estimate follow in the
// next phase, off this chain)
__device__ __noinline__ void winner_scalars(dfl vs, dfl rs, dfl rys, int j, bool fused, int32_t *sel, int row,
                                            int lane, float2 *wv, float2 *zv, float2 *LT, int ldl, float2 &s_il,
                                            float2 &s_qx, float2 &s_psi, float2 &s_mean, int &s_total) {
    const dfl il = df_rsqrt(vs);  // 1 / lambda
    const dfl wn = df_mul(rs, il);
    const dfl zn = fused ? df_mul(rys, il) : df_zero();
    const dfl qx = df_add_sloppy(ld2(&s_qx), df_sqr(wn));
    const dfl psi = df_add_sloppy(ld2(&s_psi), df_sqr(zn));
    const dfl mean = df_add(ld2(&s_mean), df_mul(wn, zn));
    __syncwarp();
    if (lane == 0) {
        st2(wv + j, wn);
        st2(zv + j, zn);
        st2(&s_il, il);
        st2(LT + j * ldl + j, il);
        st2(&s_qx, qx);
        st2(&s_psi, psi);
        st2(&s_mean, mean);
        sel[j] = row;
        s_total = 0;
    }
}

// resident CTAs per SM the register allocation is sized for (64 registers a
// thread at four)
template <int CPT>
constexpr int b32_min_blocks() {
    return CPT >= 32 ? 2 : (CPT >= 16 ? 3 : 4);
}

template <int CPT>
__global__ void __launch_bounds__(THREADS, b32_min_blocks<CPT>())
alc_bulk32_kernel(B32Params P) {
    constexpr int NPAD = FTHREADS * CPT;
    // candidates of an FP32 thread per pass of the Schur recurrence
    constexpr int CH = CPT < 8 ? CPT : 8;
    const AlcArgs &a = P.a;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, Npmax = a.Npmax, tmax = P.tmax;
    const bool fused = a.mean != nullptr;
    const int ldl = b32_ldl(nmax), ldc = b32_ldc(nmax), ldx = b32_ldx(nmax);
    // ---- dynamic shared memory (the host's b32_smem_bytes mirrors this order)
    float2 *LT = reinterpret_cast<float2 *>(smem_raw);   // nmax x ldl: LT[s][t] = (L^{-1})[t][s], 0 for t < s
    float2 *etab = LT + nmax * ldl;                        // 1024: 2^(k/1024)
    float2 *xdd = etab + EXP64_TABLE_SIZE;                 // p x ldx design coordinates
    float2 *xqd = xdd + p * ldx;                           // p (even): the reference location
    float2 *wv = xqd + ((p + 1) & ~1);                     // ldx: w = L^{-1} k_j(x)
    float2 *zv = wv + ldx;                                 // ldx: z = L^{-1} Y_j
    float2 *con_k = zv + ldx;                              // tmax x ldc: k_j(x_c); [j] = K(x_c, x)
    float2 *con_u = con_k + tmax * ldc;                    // tmax x ldc: u_c = L^{-1} k_j(x_c)
    float2 *cpart = con_u + tmax * ldc;                    // b32_cprows(tmax) x ldc partial contractions
    float2 *con_x = cpart + b32_cprows(tmax) * ldc;        // tmax x p: the batch's coordinates
    float2 *win_u = con_x + tmax * p;                      // ldc: the running best's u (several batches)
    float2 *win_x = win_u + ldc;                           // p (even): its coordinates
    // NPAD: FP32 v of every candidate (16-byte aligned for vector loads)
    float *v_s = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(win_x + ((p + 1) & ~1)) + 15) & ~(uintptr_t)15);
    float *r_s = v_s + NPAD;                               // NPAD: FP32 r of every candidate

    __shared__ int s_loc, s_bad, s_total, s_wl, s_save, s_win_saved;
    __shared__ float w_max[FWARPS];
    __shared__ int w_cnt[FWARPS];
    // contender list (the first LCAP; the rest in the per-CTA global list),
    // each with the FP32 pivot data of its candidate
    __shared__ int lst_slot[LCAP];
    __shared__ float lst_s[LCAP], lst_v[LCAP], lst_r[LCAP];
    // the batch being re-scored
    __shared__ int bat_slot[TMAX_CAP], bat_row[TMAX_CAP];
    __shared__ float bat_s[TMAX_CAP], bat_v[TMAX_CAP], bat_r[TMAX_CAP];
    __shared__ float2 con_y[TMAX_CAP], con_v[TMAX_CAP], con_r[TMAX_CAP], con_ry[TMAX_CAP];
    __shared__ float2 win_s[3];  // the running best's v, r, y - z^T u (several batches)
    __shared__ int best_slot, best_row;
    __shared__ float best_v, best_r;
    __shared__ float2 best_dl;
    __shared__ float2 s_il, s_mean, s_psi, s_qx;
    __shared__ float s_err, s_steperr;
    __shared__ unsigned long long s_work[4];

    float *U = P.U_ws + (size_t)blockIdx.x * nmax * NPAD;
    float *Cg = P.C_ws + (size_t)blockIdx.x * p * NPAD;
    float *Clo = P.Clo_ws + (size_t)blockIdx.x * p * NPAD;
    float2 *Yc = P.Yc_ws + (size_t)blockIdx.x * NPAD;
    int *ov_slot = P.ovi_ws + (size_t)blockIdx.x * NPAD;
    float *ov_s = P.ovs_ws + (size_t)blockIdx.x * 3 * NPAD, *ov_v = ov_s + NPAD, *ov_r = ov_v + NPAD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool fgroup = tid < FTHREADS;
    const int dt = tid - FTHREADS, dw = warp - FWARPS;  // index within the double-float group
    const int c0 = tid * CPT;                           // FP32 group: first candidate slot
    const bool x64 = a.dtype == LAGP_F64;
    #pragma unroll 1
    for (int k = tid; k < EXP64_TABLE_SIZE; k += THREADS) st2(etab + k, df_from_double(exp64_table_g[k]));
    if (tid < 4) s_work[tid] = 0ull;

    #pragma unroll 1
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
            #pragma unroll 1
            for (int c = tid; c < k; c += THREADS) {
                int32_t r = cands[c];
                if (r < 0 || r >= a.N) s_bad = LAGP_EINVAL;
            }
        __syncthreads();
        #pragma unroll 1
        for (int t = tid; t < nmax; t += THREADS) {
            sel[t] = -1;
            if (alc) alc[t] = CUDART_NAN;
        }
        if (s_bad != LAGP_OK) {
            if (tid == 0) {
                a.status[loc] = s_bad;
                if (fused) a.mean[loc] = a.s2[loc] = a.df[loc] = CUDART_NAN;
            }
            __syncthreads();
            continue;
        }

        // ---- per-location set-up: L^{-1} cleared (its zeros below the
        // diagonal spare the triangular products any per-element test), the
        // coordinates (FP32 and, for FP64 inputs, their low parts), the
        // responses, the initial FP32 state
        #pragma unroll 1
        for (int e = tid; e < nmax * ldl; e += THREADS) LT[e] = make_float2(0.f, 0.f);
        #pragma unroll 1
        for (int i = tid; i < p; i += THREADS) st2(xqd + i, load_df(a.Xref, loc * p + i, a.dtype));
        #pragma unroll 1
        for (int e = tid; e < p * NPAD; e += THREADS) {
            const int i = e / NPAD, c = e - i * NPAD;
            dfl xv = df_zero();
            if (c < k) xv = load_df(a.X, (int64_t)cands[c] * p + i, a.dtype);
            Cg[e] = xv.hi;
            if (x64) Clo[e] = xv.lo;
        }
        if (fused)
            #pragma unroll 1
            for (int c = tid; c < k; c += THREADS) st2(Yc + c, load_df(a.Y, cands[c], a.dtype));
        const dfl onepg = df_from_double(1.0 + g);
        const dfl inv_d = df_from_double(1.0 / d);
        if (tid == 0) {
            s_err = ERR_INIT;
            s_mean = s_psi = s_qx = make_float2(0.f, 0.f);
            s_total = 0;
            s_work[0] += 1ull;
        }
        __syncthreads();
        const float inv_df = inv_d.hi;
        const float gf = fmaxf(df_from_double(g).hi, FLT_MIN);  // floor of v in the FP32 scores
        unsigned chosen = 0;  // FP32 group: chosen (or padding) slots of this thread
        if (fgroup) {
            float wm = -FLT_MAX;
#pragma unroll
            for (int h = 0; h < CPT; h += CH) {
                float s[CH];
#pragma unroll
                for (int r = 0; r < CH; r++) s[r] = 0.f;
                #pragma unroll 1
                for (int i = 0; i < p; i++) {
                    float cv[CH];
                    load_vec<CH>(Cg + i * NPAD + c0 + h, cv);
                    const float qi = xqd[i].x;
#pragma unroll
                    for (int r = 0; r < CH; r++) {
                        const float df = cv[r] - qi;
                        s[r] = fmaf(df, df, s[r]);
                    }
                }
                float vv[CH], rr[CH];
#pragma unroll
                for (int r = 0; r < CH; r++) {
                    vv[r] = onepg.hi;
                    rr[r] = __expf(-s[r] * inv_df);  // K(x_c, x), no nugget
                    if (c0 + h + r >= k) chosen |= 1u << (h + r);  // padding slots never compete
                    else wm = fmaxf(wm, f32_score(rr[r], vv[r], gf));
                }
                store_vec<CH>(v_s + c0 + h, vv);
                store_vec<CH>(r_s + c0 + h, rr);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(LAGP_FULL_MASK, wm, o));
            if (lane == 0) w_max[warp] = wm;
        }
        int status = LAGP_OK;
        for (int j = 0; j < nm; j++) {
            // ---------------- contenders for design index j (FP32 group).  The
            // barrier orders the last step's Schur pass (v, r, per-warp maxima,
            // column j-1 of U) and its double-float work before all below.
            __syncthreads();
            if (s_bad != LAGP_OK) {
                status = s_bad;
                break;
            }
            if (fgroup) {
                unsigned flags = 0;
                if (j < a.n0) {
                    // Fig. 1 step 2(a): the nearest neighbours in order
                    if (j >= c0 && j < c0 + CPT) flags = 1u << (j - c0);
                } else {
                    const float margin = fminf(P.rel, fmaxf(MARGIN_MIN, MARGIN_KAPPA * s_err));
                    float gmax = w_max[0];
#pragma unroll
                    for (int w = 1; w < FWARPS; w++) gmax = fmaxf(gmax, w_max[w]);
                    const float thr = gmax - margin * fabsf(gmax);
#pragma unroll
                    for (int h = 0; h < CPT; h += CH) {
                        float vv[CH], rr[CH];
                        load_vec<CH>(v_s + c0 + h, vv);
                        load_vec<CH>(r_s + c0 + h, rr);
#pragma unroll
                        for (int r = 0; r < CH; r++)
                            if (!(chosen >> (h + r) & 1u) && f32_score(rr[r], vv[r], gf) >= thr)
                                flags |= 1u << (h + r);
                    }
                }
                const int mine = __popc(flags);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(LAGP_FULL_MASK, incl, o);
                    if (lane >= o) incl += t;
                }
                // the list in slot order (the batches below are its chunks, so
                // that every result is independent of the warps' timing)
                if (lane == 31) w_cnt[warp] = incl;
                fsync();
                int base = 0, all = 0;
#pragma unroll
                for (int w = 0; w < FWARPS; w++) {
                    base += w < warp ? w_cnt[w] : 0;
                    all += w_cnt[w];
                }
                if (tid == 0) s_total = all;
                int pos = base + incl - mine;
                for (unsigned f = flags; f; f &= f - 1, pos++) {
                    const int c = c0 + __ffs(f) - 1;
                    const float vc = v_s[c], rc = r_s[c], sc = f32_score(rc, vc, gf);
                    if (pos < LCAP) {
                        lst_s[pos] = sc;
                        lst_slot[pos] = c;
                        lst_v[pos] = vc;
                        lst_r[pos] = rc;
                    } else {
                        ov_slot[pos] = c;
                        ov_s[pos] = sc;
                        ov_v[pos] = vc;
                        ov_r[pos] = rc;
                    }
                }
            } else if (dt == 0) {
                s_steperr = 0.f;
                best_slot = -1;
                s_win_saved = 0;
                best_row = INT32_MAX;
                best_dl = make_float2(-FLT_MAX, 0.f);
            }
            __syncthreads();
            const int total = s_total;
            if (total < 1) {
                status = LAGP_ENOTPD;
                break;
            }
            const bool lone = total == 1;  // the common case: no comparison to make
            const bool last = j + 1 >= nm;
            // ---------------- the FP32 group: with a single contender the
            // Schur pass starts now; with several it waits for the argmax
            if (fgroup) {
                if (!lone) __syncthreads();  // (matched by the double-float group after its argmax)
                int cstar;
                float pv, pr;
                if (lone) {
                    cstar = lst_slot[0];
                    pv = lst_v[0];
                    pr = lst_r[0];
                } else {
                    cstar = best_slot;
                    pv = best_v;
                    pr = best_r;
                }
#pragma unroll
                for (int r = 0; r < CPT; r++)
                    if (c0 + r == cstar) chosen |= 1u << r;
                if (!last) {
                    // ---------------- FP32 Schur recurrence with pivot x* (new
                    // column j of U), from the pivot's own FP32 state
                    const float inv_lam = rsqrtf(fmaxf(pv, gf));
                    const float wnew = pr * inv_lam;
                    const float *Up = U + cstar;  // the pivot's column
                    float wm = -FLT_MAX;
#pragma unroll
                    for (int h = 0; h < CPT; h += CH) {
                        const float *Ub = U + c0 + h;
                        float acc[CH];
#pragma unroll
                        for (int r = 0; r < CH; r++) acc[r] = 0.f;
                        constexpr int UNR = CH >= 8 ? 4 : 8;
                        int i = 0;
                        for (; i + UNR <= j; i += UNR) {
                            float u[UNR][CH], sq[UNR];
#pragma unroll
                            for (int q = 0; q < UNR; q++) {
                                load_vec<CH>(Ub + (i + q) * NPAD, u[q]);
                                sq[q] = Up[(i + q) * NPAD];
                            }
#pragma unroll
                            for (int q = 0; q < UNR; q++)
#pragma unroll
                                for (int r = 0; r < CH; r++) acc[r] = fmaf(u[q][r], sq[q], acc[r]);
                        }
                        for (; i < j; i++) {
                            float u0[CH];
                            load_vec<CH>(Ub + i * NPAD, u0);
                            const float s0 = Up[i * NPAD];
#pragma unroll
                            for (int r = 0; r < CH; r++) acc[r] = fmaf(u0[r], s0, acc[r]);
                        }
                        float s[CH];
#pragma unroll
                        for (int r = 0; r < CH; r++) s[r] = 0.f;
#pragma unroll(CPT <= 8 ? 1 : 4)
                        for (int ii = 0; ii < p; ii++) {
                            float cv[CH];
                            load_vec<CH>(Cg + ii * NPAD + c0 + h, cv);
                            const float xi = Cg[ii * NPAD + cstar];
#pragma unroll
                            for (int r = 0; r < CH; r++) {
                                const float df = cv[r] - xi;
                                s[r] = fmaf(df, df, s[r]);
                            }
                        }
                        float vv[CH], rr[CH], un[CH];
                        load_vec<CH>(v_s + c0 + h, vv);
                        load_vec<CH>(r_s + c0 + h, rr);
#pragma unroll
                        for (int r = 0; r < CH; r++) {
                            const float kcs = __expf(-s[r] * inv_df);  // K(x_c, x*), no nugget
                            un[r] = (kcs - acc[r]) * inv_lam;
                            vv[r] = fmaf(-un[r], un[r], vv[r]);
                            rr[r] = fmaf(-wnew, un[r], rr[r]);
                            if (!(chosen >> (h + r) & 1u)) wm = fmaxf(wm, f32_score(rr[r], vv[r], gf));
                        }
                        store_vec<CH>(U + j * NPAD + c0 + h, un);
                        store_vec<CH>(v_s + c0 + h, vv);
                        store_vec<CH>(r_s + c0 + h, rr);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(LAGP_FULL_MASK, wm, o));
                    if (lane == 0) w_max[warp] = wm;
                }
                continue;  // to the next step's barrier
            }
            // ---------------- the double-float group.  First the previous
            // winner's new row of L^{-1}, -b^T / lambda, from the warps' partials
            // (deferred to here, where it overlaps the staging; the next R2
            // reads it after two barriers)
            if (j > 1 && dt < j - 1) {
                dfl b = ld2(cpart + dt);
#pragma unroll
                for (int q = 1; q < DWARPS; q++) b = df_add_sloppy(b, ld2(cpart + q * ldc + dt));
                st2(LT + dt * ldl + j - 1, df_neg(df_mul(df_normalize(b), ld2(&s_il))));
            }
            // Re-score in batches of at most tmax contenders, the consecutive
            // chunks of the list (one batch holding every contender when there
            // are at most tmax of them, the rule); when the running best
            // improves in a batch that others follow, its vectors are kept
            // (win_*) for the winner's phase
            for (int b0 = 0; b0 < total; b0 += tmax) {
                const int ncon = min(tmax, total - b0), remaining = total - b0 - ncon;
                // ---- the batch: its list entries, coordinates and responses
                if (dt < ncon) {
                    const int e = b0 + dt, slot = e < LCAP ? lst_slot[e] : ov_slot[e];
                    bat_slot[dt] = slot;
                    bat_row[dt] = cands[slot];
                    bat_s[dt] = e < LCAP ? lst_s[e] : ov_s[e];
                    bat_v[dt] = e < LCAP ? lst_v[e] : ov_v[e];
                    bat_r[dt] = e < LCAP ? lst_r[e] : ov_r[e];
                    if (fused) con_y[dt] = Yc[slot];
                }
                #pragma unroll 1
                for (int e2 = dt; e2 < ncon * p; e2 += DTHREADS) {
                    const int w = e2 / p, i = e2 - w * p, e = b0 + w;
                    const int slot = e < LCAP ? lst_slot[e] : ov_slot[e];
                    con_x[e2] = make_float2(Cg[i * NPAD + slot], x64 ? Clo[i * NPAD + slot] : 0.f);
                }
                dsync();
                // ---- R1: k_j(x_c) (t < j) and K(x_c, x) (t = j) in double-float;
                // each squared distance split over G lanes (G in 1, 2, 4).  G,
                // and R2's layout below, follow the step's contender count, not
                // the batch's, so that a contender's arithmetic (and every
                // result) is the same for any batch size
                {
                    const int jp = j + 1, pairs = ncon * jp, tpairs = min(total, TMAX_CAP) * jp;
                    const int G = tpairs * 4 <= DTHREADS ? 4 : (tpairs * 2 <= DTHREADS ? 2 : 1);
                    const int gi = dt & (G - 1), per = DTHREADS / G;
                    for (int base = 0; base < pairs; base += per) {
                        const int pr = base + dt / G;
                        const bool ok = pr < pairs;
                        const int w = ok ? pr / jp : 0, t = ok ? pr - w * jp : 0;
                        const float2 *cx = con_x + w * p;
                        dfl s = df_zero();
                        for (int i = gi; i < p; i += G) {
                            const float2 xt = t < j ? xdd[i * ldx + t] : xqd[i];
                            const float2 xc = cx[i];
                            dfl df = two_sum(xc.x, -xt.x);
                            df.lo = __fadd_rn(df.lo, __fsub_rn(xc.y, xt.y));
                            // (df.hi + df.lo)^2 with the exact leading product
                            const dfl sq = two_prod(df.hi, df.hi);
                            const float sql = __fmaf_rn(df.hi + df.hi, df.lo, sq.lo);
                            const dfl ss = two_sum(s.hi, sq.hi);
                            s.hi = ss.hi;
                            s.lo = __fadd_rn(s.lo, __fadd_rn(ss.lo, sql));
                        }
                        s = df_normalize(s);
                        for (int o = 1; o < G; o <<= 1)
                            s = df_add_sloppy(s, dfl{__shfl_xor_sync(LAGP_FULL_MASK, s.hi, o),
                                                     __shfl_xor_sync(LAGP_FULL_MASK, s.lo, o)});
                        const dfl kv = df_exp(df_neg(df_mul(s, inv_d)), etab);
                        if (ok && gi == 0) st2(con_k + w * ldc + t, kv);
                    }
                }
                dsync();
                // ---- R2: u_c = L^{-1} k_j(x_c): with one or two contenders
                // each contender's rows split over wpc warps; with more, one
                // thread per (contender, t) over the whole group (two
                // accumulation chains), so that the chains are j/2 long
                const int wpc = total == 1 ? 4 : (total == 2 ? 2 : 1);
                if (j > 0) {
                    if (total >= 3) {
                        for (int e = dt; e < ncon * j; e += DTHREADS) {
                            const int w = e / j, t = e - w * j;
                            const float2 *kc = con_k + w * ldc;
                            dfl a0 = df_zero(), a1 = df_zero();
                            int s = 0;
                            for (; s < t; s += 2) {
                                df_fma_acc(a0, ld2(LT + s * ldl + t), ld2(kc + s));
                                df_fma_acc(a1, ld2(LT + (s + 1) * ldl + t), ld2(kc + s + 1));
                            }
                            if (s == t) df_fma_acc(a0, ld2(LT + s * ldl + t), ld2(kc + s));
                            st2(cpart + w * ldc + t, df_add(df_normalize(a0), df_normalize(a1)));
                        }
                    } else {
                        for (int item = dw; item < ncon * wpc; item += DWARPS) {
                            const int w = item / wpc, part = item - w * wpc;
                            df_tri_lower(con_k + w * ldc, LT, ldl, part * j / wpc, (part + 1) * j / wpc, j, lane,
                                         cpart + item * ldc);
                        }
                    }
                }
                dsync();
                // ---- R3: u_c from the partials; |u_c|^2, w^T u_c, z^T u_c by
                // one warp per contender -> v_c, r_c and (fused) y_c - z^T u_c.
                // The step's only contender is decided here, and its warp goes
                // on to the winner's scalars.
                #pragma unroll 1
                for (int w = dw; w < ncon; w += DWARPS) {
                    dfl uu = df_zero(), uw = df_zero(), uz = df_zero();
                    float2 *uc = con_u + w * ldc;
                    #pragma unroll 1
                    for (int t = lane; t < j; t += 32) {
                        const float2 *P0 = cpart + w * wpc * ldc + t;
                        dfl ut = ld2(P0);
                        #pragma unroll 1
                        for (int q = 1; q < wpc; q++) ut = df_add_sloppy(ut, ld2(P0 + q * ldc));
                        ut = df_normalize(ut);
                        st2(uc + t, ut);
                        df_fma_acc(uu, ut, ut);
                        df_fma_acc(uw, ut, ld2(wv + t));
                        if (fused) df_fma_acc(uz, ut, ld2(zv + t));
                    }
                    uu = df_normalize(uu);
                    uw = df_normalize(uw);
                    uz = df_normalize(uz);
#pragma unroll 1
                    for (int o = 16; o > 0; o >>= 1) {
                        const dfl ou{__shfl_xor_sync(LAGP_FULL_MASK, uu.hi, o), __shfl_xor_sync(LAGP_FULL_MASK, uu.lo, o)};
                        const dfl ow{__shfl_xor_sync(LAGP_FULL_MASK, uw.hi, o), __shfl_xor_sync(LAGP_FULL_MASK, uw.lo, o)};
                        const dfl oz{__shfl_xor_sync(LAGP_FULL_MASK, uz.hi, o), __shfl_xor_sync(LAGP_FULL_MASK, uz.lo, o)};
                        uu = df_add_sloppy(uu, ou);
                        uw = df_add_sloppy(uw, ow);
                        uz = df_add_sloppy(uz, oz);
                    }
                    const dfl vc = df_sub(onepg, uu);                       // m_j^{-1}(x_c)
                    const dfl rc = df_sub(ld2(con_k + w * ldc + j), uw);     // K(x_c,x) - w^T u_c
                    const dfl ryc = fused ? df_sub(ld2(con_y + w), uz) : df_zero();
                    if (lane == 0) {
                        st2(con_v + w, vc);
                        st2(con_r + w, rc);
                        st2(con_ry + w, ryc);
                    }
                    if (lone) {
                        // the only contender is the winner when v > 0 (its
                        // Delta is computed in the winner phase, off this chain)
                        if (vc.hi > 0.f && rc.hi == rc.hi) {
                            if (lane == 0) {
                                best_row = bat_row[0];
                                best_slot = bat_slot[0];
                                best_v = bat_v[0];
                                best_r = bat_r[0];
                                best_dl = make_float2(0.f, 0.f);  // (computed below)
                                s_wl = 0;
                                s_work[1] += 1ull;
                                s_work[2] += (unsigned long long)j;
                                s_work[3] += (unsigned long long)j * j;
                            }
                            winner_scalars(vc, rc, ryc, j, fused, sel, bat_row[0], lane, wv, zv, LT, ldl, s_il, s_qx,
                                           s_psi, s_mean, s_total);
                        }
                    }
                }
                dsync();
                if (lone) break;
                // ---- R4: Delta = r^2 / v in the lanes of one warp; the batch's
                // best against the running best
                if (dw == 0) {
                    dfl dl = dfl{-FLT_MAX, 0.f};
                    int row = INT32_MAX, slot = -1;
                    float err = 0.f, bv = 0.f, bc = 0.f;
                    if (lane < ncon) {
                        const dfl vc = ld2(con_v + lane);
                        if (vc.hi > 0.f) {
                            dl = df_div(df_sqr(ld2(con_r + lane)), vc);
                            if (!(dl.hi == dl.hi)) {
                                dl = dfl{-FLT_MAX, 0.f};
                            } else {
                                row = bat_row[lane];
                                slot = bat_slot[lane];
                                bv = bat_v[lane];
                                bc = bat_r[lane];
                            }
                            // (the error against the step's best score below:
                            // a low contender's error cannot displace the best)
                            if (j >= a.n0 && dl.hi > 0.f) err = fabsf(bat_s[lane] - dl.hi);
                        }
                    }
                    int wl = lane;
#pragma unroll 1
                    for (int o = 16; o > 0; o >>= 1) {
                        const float oh = __shfl_xor_sync(LAGP_FULL_MASK, dl.hi, o);
                        const float ol = __shfl_xor_sync(LAGP_FULL_MASK, dl.lo, o);
                        const int orow = __shfl_xor_sync(LAGP_FULL_MASK, row, o);
                        const int oslot = __shfl_xor_sync(LAGP_FULL_MASK, slot, o);
                        const int owl = __shfl_xor_sync(LAGP_FULL_MASK, wl, o);
                        const float obv = __shfl_xor_sync(LAGP_FULL_MASK, bv, o);
                        const float obc = __shfl_xor_sync(LAGP_FULL_MASK, bc, o);
                        const dfl od{oh, ol};
                        if (df_gt(od, dl) || (!df_gt(dl, od) && orow < row)) {
                            dl = od;
                            row = orow;
                            slot = oslot;
                            wl = owl;
                            bv = obv;
                            bc = obc;
                        }
                        err = fmaxf(err, __shfl_xor_sync(LAGP_FULL_MASK, err, o));
                    }
                    if (lane == 0) {
                        const dfl bd = ld2(&best_dl);
                        s_steperr = fmaxf(s_steperr, err);  // (absolute: divided by the step's best below)
                        const bool improved = slot >= 0 && (df_gt(dl, bd) || (!df_gt(bd, dl) && row < best_row));
                        if (improved) {
                            st2(&best_dl, dl);
                            best_row = row;
                            best_slot = slot;
                            best_v = bv;
                            best_r = bc;
                            s_wl = wl;
                            s_win_saved = remaining > 0;  // (copied below: later batches overwrite)
                        }
                        s_save = improved && remaining > 0;
                        s_work[1] += (unsigned long long)ncon;
                        s_work[2] += (unsigned long long)ncon * j;
                        s_work[3] += (unsigned long long)ncon * j * j;
                    }
                }
                dsync();
                // (s_save is written again only after the next batch has passed
                // four more barriers, so every thread reads this value)
                if (s_save) {
                    // the new running best's vectors, before the next batch
                    // overwrites the batch arrays
                    const int wl = s_wl;
                    #pragma unroll 1
                    for (int t = dt; t < j; t += DTHREADS) win_u[t] = con_u[wl * ldc + t];
                    #pragma unroll 1
                    for (int i = dt; i < p; i += DTHREADS) win_x[i] = con_x[wl * p + i];
                    if (dt == 0) {
                        win_s[0] = con_v[wl];
                        win_s[1] = con_r[wl];
                        win_s[2] = con_ry[wl];
                    }
                    dsync();
                }
            }
            // several contenders: release the FP32 group with the winner
            if (!lone) __syncthreads();
            if (best_slot < 0) {
                // no valid contender (for a lone contender: v <= 0 in
                // double-float, while the FP32 group went ahead with it)
                if (dt == 0) s_bad = LAGP_ENOTPD;
                continue;
            }
            // ---------------- the winner: its scalars (several contenders),
            // the partials of b = L^{-T} u* for the next row of L^{-1}, its
            // coordinates in the design
            const int wl = s_wl;
            const bool saved = s_win_saved;  // the winner's vectors were kept from an earlier batch
            const float2 *wu = saved ? win_u : con_u + wl * ldc, *wx = saved ? win_x : con_x + wl * p;
            if (!lone && dw == 0)
                winner_scalars(ld2(saved ? win_s : con_v + wl), ld2(saved ? win_s + 1 : con_r + wl),
                               ld2(saved ? win_s + 2 : con_ry + wl), j, fused, sel, best_row, lane, wv, zv, LT, ldl,
                               s_il, s_qx, s_psi, s_mean, s_total);
            if (dt == 32) {
                // the ALC value (a lone contender's Delta is computed here) and
                // the contender margin's error estimate
                dfl dl = ld2(&best_dl);
                // the batches' largest error over the step's best score (the
                // same whatever the batches)
                float err = dl.hi > 0.f ? __fdividef(s_steperr, dl.hi) : 0.f;
                if (lone) {
                    dl = df_div(df_sqr(ld2(con_r)), ld2(con_v));
                    if (j >= a.n0 && dl.hi > 0.f) err = fabsf(__fdividef(bat_s[0], dl.hi) - 1.f);
                }
                if (alc && j >= a.n0) alc[j] = df_to_double(dl);
                if (j >= a.n0) s_err = fmaxf(ERR_DECAY * s_err, err);
            }
            if (!last && j > 0) {
                // warp dw takes t in [t0, t1): equal lengths, so that the
                // longest chain is j / DWARPS; its partial covers s < t1
                const int t0 = dw * j / DWARPS, t1 = (dw + 1) * j / DWARPS;
                float2 *part = cpart + dw * ldc;
                df_tri_upper(wu, LT, ldl, t0, t1, lane, part);
                #pragma unroll 1
                for (int s = t1 + lane; s < j; s += 32) part[s] = make_float2(0.f, 0.f);
            }
            #pragma unroll 1
            for (int i = dt; i < p; i += DTHREADS) xdd[i * ldx + j] = wx[i];
        }
        // (a double-float failure in the last step is seen here)
        __syncthreads();
        if (s_bad != LAGP_OK) status = s_bad;
        if (status != LAGP_OK) {
            #pragma unroll 1
            for (int t = tid; t < nmax; t += THREADS) {
                sel[t] = -1;
                if (alc) alc[t] = CUDART_NAN;
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (fused) {
                // Eqs. (predgp), (preds2): mean = w^T z, s2 = psi (1 + g - |w|^2) / n
                const bool ok = status == LAGP_OK;
                const dfl s2 = df_div(df_mul(ld2(&s_psi), df_sub(onepg, ld2(&s_qx))), dfl{(float)nm, 0.f});
                a.mean[loc] = ok ? df_to_double(ld2(&s_mean)) : CUDART_NAN;
                a.s2[loc] = ok ? df_to_double(s2) : CUDART_NAN;
                a.df[loc] = ok ? (double)nm : CUDART_NAN;
            }
            a.status[loc] = status;
            if (status == LAGP_ENOTPD && a.fail_count) atomicAdd(a.fail_count, 1);  // (the FP64 Schur retry)
            s_bad = LAGP_OK;
        }
        __syncthreads();
    }
    if (tid < 4 && P.work) atomicAdd(P.work + tid, s_work[tid]);
}

// dynamic shared memory of alc_bulk32_kernel, in the kernel's order
size_t b32_smem_bytes(int nmax, int p, int tmax, int npad) {
    const size_t ldl = b32_ldl(nmax), ldc = b32_ldc(nmax), ldx = b32_ldx(nmax);
    return 8 * ((size_t)nmax * ldl + EXP64_TABLE_SIZE + (size_t)p * ldx + (((size_t)p + 1) & ~(size_t)1) +
                2 * ldx + 2 * (size_t)tmax * ldc + (size_t)b32_cprows(tmax) * ldc + (size_t)tmax * p + ldc +
                (((size_t)p + 1) & ~(size_t)1)) +
           4 * 2 * (size_t)npad + 16;
}

template <int CPT>
lagp_status launch_b32(lagp_ctx *ctx, const AlcArgs &a) {
    constexpr int NPAD = FTHREADS * CPT;
    cudaStream_t st = ctx->stream;
    const std::string key = alc_shape_key("alc_f32", CPT, a.nmax, a.p, a.mean != nullptr);
    int tmax = std::max(1, std::min(alc_rescore_batch(ctx, key), TMAX_CAP));
    // the largest batch whose vectors fit in shared memory (the batch size
    // changes no result)
    while (tmax > 1 && b32_smem_bytes(a.nmax, a.p, tmax, NPAD) > ctx->smem_optin) tmax--;
    auto kern = alc_bulk32_kernel<CPT>;
    const size_t smem = b32_smem_bytes(a.nmax, a.p, tmax, NPAD);
    if (smem > ctx->smem_optin)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: shared memory exceeded (n_max, p too large)");
    LAGP_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    LAGP_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem));
    int per_sm = alc_ctas_per_sm(ctx, key, b32_min_blocks<CPT>());
    if (occ > 0 && per_sm > occ) per_sm = occ;
    int64_t grid = (int64_t)ctx->num_sms * std::max(1, per_sm);
    if (grid > a.M) grid = a.M;
    if (grid < 1) grid = 1;
    const size_t nU = (size_t)grid * a.nmax * NPAD, nC = (size_t)grid * a.p * NPAD, nO = (size_t)grid * NPAD;
    char *ws = static_cast<char *>(lagp_ws(ctx, WS_ALC_PANEL, 4 * (nU + 2 * nC + 6 * nO) + 512));
    int *counter = nullptr;
    unsigned long long *work = nullptr;
    LAGP_TRY(alc_counters(ctx, &counter, &work));
    if (!ws) return LAGP_ENOMEM;
    float *U = reinterpret_cast<float *>(ws);
    float *C = U + nU, *Clo = C + nC, *ovs = Clo + nC;
    int *ovi = reinterpret_cast<int *>(ovs + 3 * nO);
    float2 *Yc = reinterpret_cast<float2 *>(ovi + nO);  // 8-byte aligned: nO is a multiple of 128
    LAGP_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), st));
    B32Params P{a, counter, work, U, C, Clo, Yc, ovs, ovi, ctx->num_sms, tmax, (float)ctx->tuning.rescore_rel};
    kern<<<(unsigned)grid, THREADS, smem, st>>>(P);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

}  // namespace

lagp_status launch_alc_f32(lagp_ctx *ctx, const AlcArgs &a) {
    if (a.nmax > 128) return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_select: n_max above 128 is not supported");
    const int need = (a.Npmax + FTHREADS - 1) / FTHREADS;
    if (need <= 2) return launch_b32<2>(ctx, a);
    if (need <= 4) return launch_b32<4>(ctx, a);
    if (need <= 8) return launch_b32<8>(ctx, a);
    if (need <= 16) return launch_b32<16>(ctx, a);
    return launch_b32<32>(ctx, a);
}
