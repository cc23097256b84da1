// a1: exact N'-nearest-neighbour candidate sets (Sec. 3.1 of the paper: the
// ALC search runs over the N' nearest neighbours of x; Fig. 1 step 2(a)).
//
// Design (GB300): distances are screened in FP32 (74 TFLOP/s) and only the
// few candidates near the N'-th distance are re-ranked in FP64 (1.2 TFLOP/s).
//   knn_bounds  per-coordinate minimum and maximum of the design and the
//               reference locations (the centre c and half-width B).
//   knn_prep    centred FP32 copy of the design, y = fl32(x - c), with the
//               FP32 squared norm |y|^2 as an extra column.
//   knn_screen  persistent; 16 queries per CTA, two per warp, sharing every
//               design tile in shared memory.  The main launch evaluates
//               |y_x|^2 + |y_q|^2 - 2 y_x . y_q (one add and p FMAs a pair);
//               the exact retry the direct sum of squared differences.
//               (A, B) 2-level histogram (FP32 distance bits [30:21], then
//               [20:11] inside the boundary bin) over a strided sample of the
//               design, giving a threshold tau0 expected to bound about 1.3 N'
//               rows (with stride 1, exactly the N'-th smallest distance);
//               (C) one pass over the whole design collecting every row below
//               tau0 widened by a rigorous FP32-vs-FP64 error margin (see
//               expansion_margin, screen_margin) and counting the rows below
//               tau0.  A query whose count is short of N', or whose buffer
//               overflowed, is redone by a second launch with stride 1 (the
//               exact method), where a block with at most four such queries
//               gives each a team of warps that share its sweep.
//   knn_sort    one CTA per query: exact FP64 distances of the collected rows
//               (separately rounded subtract/multiply/add in coordinate order,
//               on the original coordinates), bitonic sort on (d2, row), first
//               N' rows written out.
// The collected set provably contains the exact FP64 top-N', so the result
// equals an FP64 sort of all N rows bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "knn_common.cuh"
#include "lagp_internal.h"

namespace {

constexpr int QPW = 2;                // queries per warp
constexpr int SCREEN_THREADS = 256;
constexpr int QB = QPW * SCREEN_THREADS / 32;  // 16 queries per CTA
constexpr int HB = 1024;              // histogram bins per level (10 bits)
constexpr int L1_SHIFT = 21;          // level 1: FP32 distance bits [30:21]
constexpr int L2_SHIFT = 11;          // level 2: bits [20:11] inside the boundary bin
constexpr uint32_t L2_LOW = (1u << L2_SHIFT) - 1;
constexpr int TILE_FLOATS = 4096;     // floats of one design tile (tile length x row stride)

// Floats per centred row: p coordinates and the squared norm, padded to an
// odd count so that lanes reading consecutive rows of a shared-memory tile
// hit distinct banks.
__host__ __device__ inline int row_stride(int p) { return (p + 1) | 1; }

// Design rows per tile: a multiple of 32 with tile length x row stride <=
// TILE_FLOATS, at most 512.
__host__ __device__ inline int tile_len(int ps) {
    int t = (TILE_FLOATS / ps) & ~31;
    return t > 512 ? 512 : (t < 32 ? 32 : t);
}


// 16-byte asynchronous global-to-shared copy (bypassing L1), and its fences
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
constexpr int CAND_CAP = 8192;        // candidate capacity cap (sort in shared memory)
constexpr int SORT_SMALL = 1024;      // survivors the first sort launch holds
// kNN meta area: the tensor-core screen's failure word (offset 0), two block
// counters (64), the coordinate bounds (256 and 768, 64 keys each), the
// launch constants (KnnConst, 1280), then per-query candidate counts and
// retry flags
constexpr size_t META_HEAD = 2048;
constexpr size_t META_CONST = 1280;

// Constants of one kNN launch, written once by knn_prep: the centre c and
// half-width B of the coordinates, e2 = 2uB sqrt(p) and the power bounds
// g_half >= (1 + u)^((p+4)/2), (1 - u)^(-(p+4)/2) and g_full >= (1 + u)^(p+4).
struct KnnConst {
    double c[64];
    double B, e2, g_half, g_full;
};
constexpr int SORT_THREADS = 256;

// Per-coordinate bounds of the design and the reference locations:
// kmax[i] = key of max_i, kmin[i] = ~key of min_i (both maximised).  Eight
// coordinates per sweep: each thread keeps their bounds in registers over its
// rows, then warp and block reductions, one atomic per block and coordinate.
__global__ void knn_bounds(const void *__restrict__ X, int64_t N, const void *__restrict__ Xr,
                           int64_t M, int p, lagp_dtype dt, unsigned long long *kmax,
                           unsigned long long *kmin) {
    __shared__ unsigned long long smax[64], smin[64];
    for (int i = threadIdx.x; i < p; i += blockDim.x) smax[i] = smin[i] = 0ull;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int i0 = 0; i0 < p; i0 += 8) {
        double lo[8], hi[8];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            lo[c] = CUDART_INF;
            hi[c] = -CUDART_INF;
        }
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N + M; r += stride) {
            const bool des = r < N;
            const void *A = des ? X : Xr;
            const int64_t rr = des ? r : r - N;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                if (i0 + c >= p) break;
                const double v = load_coord64(A, rr, p, i0 + c, dt);
                if (isfinite(v)) {  // a non-finite row only spoils its own distances
                    lo[c] = fmin(lo[c], v);
                    hi[c] = fmax(hi[c], v);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 8; c++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo[c] = fmin(lo[c], __shfl_xor_sync(LAGP_FULL_MASK, lo[c], o));
                hi[c] = fmax(hi[c], __shfl_xor_sync(LAGP_FULL_MASK, hi[c], o));
            }
            if ((threadIdx.x & 31) == 0 && i0 + c < p && hi[c] >= lo[c]) {
                atomicMax(&smax[i0 + c], dkey(hi[c]));
                atomicMax(&smin[i0 + c], ~dkey(lo[c]));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        if (smax[i]) atomicMax(&kmax[i], smax[i]);
        if (smin[i]) atomicMax(&kmin[i], smin[i]);
    }
}

// Centred FP32 copy of design row r, (y_0 .. y_{p-1}, |y|^2, 0 padding),
// with y_i = fl32(x_i - c_i) and |y|^2 an FP32 fused multiply-add chain in
// coordinate order; rows past N are zero.
__device__ __forceinline__ void centred_row(const void *X, int64_t N, int64_t r, int p, int ps,
                                            lagp_dtype dt, const double *c, float *out) {
    float n2 = 0.f;
    for (int i = 0; i < p; i++) {
        const float y = r < N ? (float)(load_coord64(X, r, p, i, dt) - c[i]) : 0.f;
        out[i] = y;
        n2 = fmaf(y, y, n2);
    }
    for (int i = p; i < ps; i++) out[i] = i == p ? n2 : 0.f;
}

// Rigorous upper bounds of the powers of (1 + u) and 1 / (1 - u) that the
// margins need (n u < 1): (1 + u)^m <= (1 - u)^-m <= 1 / (1 - m u) for
// m <= n, without a call to pow (whose latency on the FP64 unit would
// serialise the threads that wait for the margin).
__device__ __forceinline__ double pow_bound(double u, double n) { return 1.0 / (1.0 - ceil(n) * u); }

// Y: all rows (Npad of them), Ys: rows 0, s, 2s, ... (nsamp_pad of them;
// null when s = 1, where the sample is the whole design), Yv: the
// coordinates of Y with a row stride of p rounded up to 4; kc: the launch's
// constants (block 0).
__global__ void knn_prep(const void *__restrict__ X, int64_t N, int p, lagp_dtype dt,
                         const unsigned long long *kmax, const unsigned long long *kmin,
                         float *__restrict__ Y, int64_t Npad, float *__restrict__ Ys,
                         int64_t nsamp_pad, int64_t sstride, KnnConst *kc, float *__restrict__ Yv) {
    __shared__ double c[64];
    __shared__ double sB;
    if (threadIdx.x == 0) {
        centre_and_bound(kmax, kmin, p, c, sB);
        if (blockIdx.x == 0) {
            const double u = 0x1p-24 * (1.0 + 0x1p-27);
            for (int i = 0; i < p; i++) kc->c[i] = c[i];
            kc->B = sB;
            kc->e2 = 2.0 * u * sB * sqrt((double)p);
            kc->g_half = pow_bound(u, 0.5 * (p + 4));
            kc->g_full = pow_bound(u, (double)(p + 4));
        }
    }
    __syncthreads();
    const int ps = row_stride(p);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < Npad; r += stride) {
        centred_row(X, N, r, p, ps, dt, c, Y + r * ps);
        // the same coordinates with a row stride of p rounded up to 4 (vector gathers in the sort)
        const int pv = (p + 3) & ~3;
        for (int i = 0; i < pv; i++) Yv[r * pv + i] = i < p ? Y[r * ps + i] : 0.f;
    }
    if (Ys)
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nsamp_pad; r += stride)
            centred_row(X, N, r * sstride, p, ps, dt, c, Ys + r * ps);
}

// Widened thresholds for the collection pass.  With u = 2^-24 (widened by
// 2^-27 for the FP64 centring), centred coordinates rounded to FP32 with
// absolute error <= u B, the FP32 screen value s of a row relates to its
// exact distance r as follows.
//
// screen_margin (direct form: FP32 differences, squares and sums, each
// rounded once):
//     (1-u)^((p+4)/2) (r - 2uB sqrt(p)) <= sqrt(s) <= (1+u)^((p+4)/2) (r + 2uB sqrt(p)).
// Every row with s <= tau then has r <= r_hi = sqrt(tau) (1-u)^(-(p+4)/2) + 2uB sqrt(p),
// so the N'-th exact distance is <= r_hi, and every row of the exact top-N' has
// sqrt(s) <= (r_hi + 2uB sqrt(p)) (1+u)^((p+4)/2).
//
// expansion_margin (s = max(0, |y_x|^2 + |y_q|^2 - 2 y_x . y_q), every norm
// and the dot product FMA chains of at most 2p + 4 roundings in all):
//     |s - |y_q - y_x|^2| <= E = gamma_{2p+4} 4 p B^2,   gamma_k = k u / (1 - k u),
// and |y_q - y_x| lies within 2uB sqrt(p) of r.  A row with s <= tau then has
// r <= r_hi = sqrt(tau + E) + 2uB sqrt(p), and every row of the exact top-N'
// has s <= (r_hi + 2uB sqrt(p))^2 + E.
//
// The final factors cover the rounding of the FP64 reference distances (the
// order is that of the FP64 sums, within a relative 1e-15 of r^2) and of
// this computation.
// g >= (1 - u)^-(p+4)/2 and (1 + u)^(p+4)/2, e2 = 2uB sqrt(p)
__device__ __forceinline__ double screen_margin_c(float tau, double g, double e2) {
    const double r_hi = sqrt((double)tau) * g * (1.0 + 1e-13) + e2;
    const double r_col = (r_hi + e2) * g;
    return r_col * r_col * (1.0 + 1e-12);
}

__device__ double screen_margin(float tau, int p, double B) {
    const double u = 0x1p-24 * (1.0 + 0x1p-27);
    return screen_margin_c(tau, pow_bound(u, 0.5 * (p + 4)), 2.0 * u * B * sqrt((double)p));
}

__device__ double expansion_margin(float tau, int p, double B) {
    const double u = 0x1p-24 * (1.0 + 0x1p-27);
    const double Bt = B * (1.0 + u);
    const double e2 = 2.0 * u * B * sqrt((double)p);
    const double k = 2.0 * p + 4.0;
    const double E = (k * u / (1.0 - k * u)) * 4.0 * p * Bt * Bt;
    const double r_hi = sqrt((double)tau + E) * (1.0 + 1e-13) + e2;
    const double r_col = r_hi + e2;
    return (r_col * r_col + E) * (1.0 + 1e-12);
}

// Smallest bin b of the warp's histogram h with cum(h[0..b]) >= target,
// and the count strictly before it.  Requires sum(h) >= target >= 1.
__device__ void find_bin(const uint32_t *h, uint32_t target, int lane, uint32_t &bin,
                         uint32_t &before) {
    constexpr int PER = HB / 32;
    uint32_t s = 0;
    for (int b = 0; b < PER; b++) s += h[lane * PER + b];
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(LAGP_FULL_MASK, incl, o);
        if (lane >= o) incl += v;
    }
    unsigned ball = __ballot_sync(LAGP_FULL_MASK, incl >= target);
    int L = ball ? __ffs(ball) - 1 : 31;
    uint32_t base = __shfl_sync(LAGP_FULL_MASK, incl - s, L);
    // resolve inside lane L's PER bins, 32 at a time
    bin = (uint32_t)(L * PER + PER - 1);
    before = base;
    for (int half = 0; half < PER; half += 32) {
        uint32_t v = h[L * PER + half + lane];
        uint32_t c = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(LAGP_FULL_MASK, c, o);
            if (lane >= o) c += t;
        }
        unsigned bb = __ballot_sync(LAGP_FULL_MASK, base + c >= target);
        if (bb) {
            int l2 = __ffs(bb) - 1;
            bin = (uint32_t)(L * PER + half + l2);
            before = base + __shfl_sync(LAGP_FULL_MASK, c - v, l2);
            return;
        }
        base += __shfl_sync(LAGP_FULL_MASK, c, 31);
    }
}

// One design tile against a warp's QPW queries, rows r0, r0 + rstep, ... of
// the tile.  PASS 0: level-1 histogram; PASS 1: level-2 histogram inside the
// boundary bin; PASS 2: collection.
// Tile row pt holds (y_0 .. y_{p-1}, |y|^2) of a centred design row, with
// row stride PS.  EXP: s = max(0, |y_x|^2 + |y_q|^2 - 2 y_x . y_q) with
// qr = -2 y_q and qn = |y_q|^2 (negative values, from rounding, clamped to 0);
// otherwise s = sum (y_x - y_q)^2 with qr = y_q.
template <int P, int PASS, bool EXP>
__device__ __forceinline__ void screen_tile(const float *t, int ps_rt, int cnt, int r0, int rstep, int p,
                                            const float (&qr)[QPW][P > 0 ? P : 1],
                                            const float (&qn)[QPW], const float *qsw,
                                            const bool (&ok)[QPW], uint32_t *histw,
                                            const uint32_t (&b1)[QPW], const float (&tau0)[QPW],
                                            const float (&tau2f)[QPW], int32_t *cntw, int32_t *cnt0w,
                                            int32_t *__restrict__ cand, const int64_t (&q)[QPW],
                                            int32_t Cmax, int64_t base) {
    const int np = P > 0 ? P : p;
    const int PS = P > 0 ? ((P + 1) | 1) : ps_rt;
    for (int pt = r0; pt < cnt; pt += rstep) {
        const float *row = t + pt * PS;
        float sd[QPW];
        if constexpr (EXP) {
            const float xn = row[np];
#pragma unroll
            for (int h = 0; h < QPW; h++) sd[h] = xn + qn[h];
        } else {
#pragma unroll
            for (int h = 0; h < QPW; h++) sd[h] = 0.f;
        }
        if constexpr (P > 0) {
#pragma unroll
            for (int i = 0; i < P; i++) {
                const float x = row[i];
#pragma unroll
                for (int h = 0; h < QPW; h++) {
                    if constexpr (EXP) {
                        sd[h] = fmaf(x, qr[h][i], sd[h]);
                    } else {
                        const float df = x - qr[h][i];
                        sd[h] = fmaf(df, df, sd[h]);
                    }
                }
            }
        } else {
            for (int i = 0; i < p; i++) {
                const float x = row[i];
#pragma unroll
                for (int h = 0; h < QPW; h++) {
                    const float qv = qsw[h * PS + i];
                    if constexpr (EXP) {
                        sd[h] = fmaf(x, -2.f * qv, sd[h]);
                    } else {
                        const float df = x - qv;
                        sd[h] = fmaf(df, df, sd[h]);
                    }
                }
            }
        }
#pragma unroll
        for (int h = 0; h < QPW; h++) {
            if constexpr (EXP) sd[h] = sd[h] < 0.f ? 0.f : sd[h];  // keeps NaN
            if constexpr (PASS == 0) {
                if (ok[h]) atomicAdd(&histw[h * HB + ((__float_as_uint(sd[h]) >> L1_SHIFT) & (HB - 1))], 1u);
            } else if constexpr (PASS == 1) {
                const uint32_t bits = __float_as_uint(sd[h]);
                if (ok[h] && ((bits >> L1_SHIFT) & (HB - 1)) == b1[h])
                    atomicAdd(&histw[h * HB + ((bits >> L2_SHIFT) & (HB - 1))], 1u);
            } else {
                if (ok[h] && sd[h] <= tau2f[h]) {
                    if (sd[h] <= tau0[h]) atomicAdd(&cnt0w[h], 1);
                    const int pos = atomicAdd(&cntw[h], 1);
                    if (pos < Cmax) cand[q[h] * Cmax + pos] = (int32_t)(base + pt);
                }
            }
        }
    }
}

// Screen of one block of QB queries (two per warp) against the design.
//   Passes A, B: 2-level histogram of the FP32 distances to the sampled rows
//   r = 0, s, 2s, ...; the rtarget-th smallest sampled distance gives tau0
//   (upper edge of its level-2 bin).  With s = 1 (small designs, and the exact
//   retry) rtarget = N' and tau0 bounds the N'-th smallest FP32 distance.
//   Pass C: every row whose FP32 distance is <= the widened threshold is
//   collected, and the rows <= tau0 are counted; when that count reaches N'
//   the collected set provably holds the exact FP64 top N' (see the margin
//   functions).  Otherwise (a sample that underestimated the threshold) or
//   when the buffer overflows, the query is flagged for the exact retry.
template <int P, bool EXP>
__global__ void __launch_bounds__(SCREEN_THREADS, 2)
knn_screen(const float *__restrict__ Y32, const float *__restrict__ Ys, int64_t N, int p,
           const void *__restrict__ Xref,
           lagp_dtype dt, int64_t M, const int32_t *__restrict__ Np, int32_t Npmax,
           const unsigned long long *__restrict__ kmax, const unsigned long long *__restrict__ kmin,
           int32_t *__restrict__ cand, int32_t Cmax, int32_t *__restrict__ cand_count,
           int32_t *__restrict__ status, int64_t stride, int32_t *__restrict__ retry, int retry_pass,
           int *__restrict__ counter, float *__restrict__ tau_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pp = row_stride(p);              // floats per centred row (coordinates, norm, pad)
    const int TT = tile_len(pp);               // rows per tile
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_raw);   // QB x HB
    float *tiles = reinterpret_cast<float *>(hist + QB * HB);  // 2 x TT x pp, 16-byte aligned
    float *qs = tiles + 2 * (size_t)TT * pp;                     // (QB + 1) x pp: centred queries
    __shared__ int32_t s_count[QB], s_count0[QB], s_flag[QB], s_rt[QB];
    __shared__ int64_t s_blk;
    __shared__ double s_c[64], s_B;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) centre_and_bound(kmax, kmin, p, s_c, s_B);
    // a spare zero slot past the QB queries (read, never used, by the second
    // query slot of a warp that screens the last query of a block together
    // with other warps)
    for (int i = threadIdx.x; i < pp; i += SCREEN_THREADS) qs[QB * pp + i] = 0.f;
    __syncthreads();
    const double B = s_B;
    const int64_t nsamp = (N + stride - 1) / stride;

    for (;;) {
        if (threadIdx.x == 0) s_blk = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t blk = s_blk;
        __syncthreads();
        if (blk * QB >= M) break;

        int64_t q[QPW];
        int k[QPW], rtarget[QPW];
        bool ok[QPW], active[QPW];
        bool mine_any = false;
#pragma unroll
        for (int h = 0; h < QPW; h++) {
            const int ql = w * QPW + h;
            q[h] = blk * QB + ql;
            active[h] = q[h] < M;
            k[h] = active[h] ? (Np ? Np[q[h]] : Npmax) : 0;
            ok[h] = active[h] && k[h] >= 1 && k[h] <= Npmax;
            if (retry_pass) ok[h] = ok[h] && retry[q[h]] != 0;  // exact retry: flagged queries only
            mine_any |= ok[h];
            rtarget[h] = stride == 1 ? k[h]
                                     : (int)min((int64_t)((13 * (int64_t)k[h] + 10 * stride - 1) / (10 * stride)) + 16, nsamp);
            if (lane == 0) {
                float n2 = 0.f;
                for (int i = 0; i < p; i++) {
                    const float y = active[h] ? (float)(load_coord64(Xref, q[h], p, i, dt) - s_c[i]) : 0.f;
                    qs[ql * pp + i] = y;
                    n2 = fmaf(y, y, n2);
                }
                qs[ql * pp + p] = n2;
                for (int i = p + 1; i < pp; i++) qs[ql * pp + i] = 0.f;
            }
            for (int b = lane; b < HB; b += 32) hist[ql * HB + b] = 0;
            if (lane == 0) {
                s_count[ql] = s_count0[ql] = 0;
                s_flag[ql] = ok[h] ? 1 : 0;
                s_rt[ql] = rtarget[h];
            }
        }
        // a block without a query to screen skips the passes (not the results)
        const bool any_ok = __syncthreads_or(mine_any);
        // The queries a warp screens: its own QPW (slots sbase, sbase + 1) or,
        // in the exact retry of a block with at most four flagged queries,
        // one flagged query shared by a team of W = 8 / nf warps (nf rounded
        // up to a power of two; a team of four idle when nf = 3).  A team
        // splits every tile's rows (warp `sub` of the team takes the 32-row
        // groups sub, sub + W, ...) and adds into the query's one histogram
        // and counters, so that one query's sweep over all N rows runs on
        // the whole CTA instead of one warp.  The results are the same
        // either way: the counts do not depend on which warp adds them, and
        // the sort orders the collected rows.
        int nf = 0;
        if (retry_pass)
            for (int c = 0; c < QB; c++) nf += s_flag[c];
        const bool coop = nf >= 1 && nf <= 4;
        int sbase = w * QPW, r0 = lane, rstep = 32;
        bool leader = true;  // the warp that clears the team's histogram
        bool sok[QPW];
        int srt[QPW];
        int64_t sq[QPW];
#pragma unroll
        for (int h = 0; h < QPW; h++) {
            sok[h] = ok[h];
            srt[h] = rtarget[h];
            sq[h] = q[h];
        }
        if (coop) {
            const int W = nf == 1 ? 8 : (nf == 2 ? 4 : 2);
            const int team = w / W, sub = w - team * W;
            int slot = -1;  // the team-th flagged slot
            for (int c = 0, f = 0; c < QB; c++)
                if (s_flag[c]) {
                    if (f == team) slot = c;
                    f++;
                }
            sbase = slot >= 0 ? slot : 0;
#pragma unroll
            for (int h = 0; h < QPW; h++) {
                sok[h] = h == 0 && slot >= 0;
                srt[h] = s_rt[sbase];
                sq[h] = blk * QB + sbase;
            }
            r0 = lane + 32 * sub;
            rstep = 32 * W;
            leader = sub == 0;
        }
        float qr[QPW][P > 0 ? P : 1] = {};
        float qn[QPW] = {};
#pragma unroll
        for (int h = 0; h < QPW; h++) {
            qn[h] = qs[(sbase + h) * pp + p];
            if constexpr (P > 0) {
#pragma unroll
                for (int i = 0; i < P; i++) {
                    const float y = qs[(sbase + h) * pp + i];
                    qr[h][i] = EXP ? -2.f * y : y;
                }
            }
        }

        uint32_t b1[QPW] = {}, before[QPW] = {};
        // thresholds as floats: for a float distance s, s <= t (t real) holds
        // exactly when s <= t rounded down to a float, so the hot loop compares
        // in FP32 (an FP64 compare per point would occupy the slow FP64 unit)
        float tau0[QPW] = {}, tau2f[QPW] = {};
        // with tau_out, passes A and B only: the sampled threshold tau0 of
        // every query (NaN for one that is not screened) for the collection
        // pass on the tensor cores
        const int npass = !any_ok ? 0 : (tau_out ? 2 : 3);
        for (int pass = 0; pass < npass; pass++) {
            // passes A, B: the sampled rows (contiguous in Ys); C: all rows
            const float *src = pass < 2 ? Ys : Y32;
            const int64_t nrows = pass < 2 ? nsamp : N;
            const int64_t ntiles = (nrows + TT - 1) / TT;
            // tile `tile` into buffer `buf`: its rows rounded up to a multiple of
            // 4 (zero rows past the end of the padded copies), 16 bytes a copy
            auto issue = [&](int64_t tile, int buf) {
                const int64_t base = tile * TT;
                const int cnt4 = (int)round_up(min((int64_t)TT, nrows - base), 4);
                const int nchunk = cnt4 * pp / 4;
                const float *g = src + base * pp;
                float *t = tiles + (size_t)buf * TT * pp;
                for (int e = threadIdx.x; e < nchunk; e += SCREEN_THREADS) cp_async16(t + 4 * e, g + 4 * e);
                cp_async_commit();
            };
            issue(0, 0);
            cp_async_wait_all();
            __syncthreads();
            for (int64_t tile = 0; tile < ntiles; tile++) {
                const int buf = (int)(tile & 1);
                if (tile + 1 < ntiles) issue(tile + 1, buf ^ 1);  // in flight during the screen
                const int64_t base = tile * TT;
                const int cnt = (int)min((int64_t)TT, nrows - base);
                const float *t = tiles + (size_t)buf * TT * pp;
                const float *qsw = qs + sbase * pp;
                uint32_t *histw = hist + sbase * HB;
                if (pass == 0)
                    screen_tile<P, 0, EXP>(t, pp, cnt, r0, rstep, p, qr, qn, qsw, sok, histw, b1, tau0, tau2f,
                                           s_count + sbase, s_count0 + sbase, cand, sq, Cmax, base);
                else if (pass == 1)
                    screen_tile<P, 1, EXP>(t, pp, cnt, r0, rstep, p, qr, qn, qsw, sok, histw, b1, tau0, tau2f,
                                           s_count + sbase, s_count0 + sbase, cand, sq, Cmax, base);
                else
                    screen_tile<P, 2, EXP>(t, pp, cnt, r0, rstep, p, qr, qn, qsw, sok, histw, b1, tau0, tau2f,
                                           s_count + sbase, s_count0 + sbase, cand, sq, Cmax, base);
                // the next tile has landed and every warp is done with this one
                cp_async_wait_all();
                __syncthreads();
            }
#pragma unroll
            for (int h = 0; h < QPW; h++) {
                if (!sok[h]) continue;
                const uint32_t *hh = hist + (sbase + h) * HB;
                if (pass == 0) {
                    find_bin(hh, (uint32_t)srt[h], lane, b1[h], before[h]);
                } else if (pass == 1) {
                    uint32_t b2, before2;
                    find_bin(hh, (uint32_t)srt[h] - before[h], lane, b2, before2);
                    tau0[h] = __uint_as_float((b1[h] << L1_SHIFT) | (b2 << L2_SHIFT) | L2_LOW);
                    tau2f[h] = __double2float_rd(EXP ? expansion_margin(tau0[h], p, B)
                                                     : screen_margin(tau0[h], p, B));
                }
            }
            if (pass == 0) {
                // every warp of a team has read the level-1 histogram before
                // its leader clears it for level 2
                __syncthreads();
                if (leader)
#pragma unroll
                    for (int h = 0; h < QPW; h++)
                        if (sok[h])
                            for (int b = lane; b < HB; b += 32) hist[(sbase + h) * HB + b] = 0;
            }
            __syncthreads();
        }
        if (tau_out) {
#pragma unroll
            for (int h = 0; h < QPW; h++)
                if (active[h] && lane == 0) tau_out[q[h]] = ok[h] ? tau0[h] : CUDART_NAN_F;
            continue;
        }
#pragma unroll
        for (int h = 0; h < QPW; h++) {
            if (!active[h] || lane != 0) continue;
            const int ql = w * QPW + h;
            const int c = s_count[ql], c0 = s_count0[ql];
            const bool kvalid = k[h] >= 1 && k[h] <= Npmax;
            if (!retry_pass) {
                const bool done = ok[h] && c0 >= k[h] && c <= Cmax;
                retry[q[h]] = (ok[h] && !done) ? 1 : 0;
                cand_count[q[h]] = done ? c : 0;
                if (status) status[q[h]] = kvalid ? LAGP_OK : LAGP_EINVAL;
            } else if (ok[h]) {
                // exact retry: fewer rows than N' under the threshold only happens
                // with non-finite distances (NaN or overflowing coordinates)
                cand_count[q[h]] = (c0 >= k[h] && c <= Cmax) ? c : 0;
                if (status) status[q[h]] = c0 < k[h] ? LAGP_EINVAL : (c > Cmax ? LAGP_ENOMEM : LAGP_OK);
            }
        }
        __syncthreads();
    }
}

// Block-wide exclusive prefix sum of one int per thread (SORT_THREADS
// threads); returns the thread's offset, *total the sum.
__device__ int block_excl_scan(int v, int *wsum, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(LAGP_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int off = 0, tot = 0;
    for (int i = 0; i < SORT_THREADS / 32; i++) {
        off += i < w ? wsum[i] : 0;
        tot += wsum[i];
    }
    __syncthreads();
    *total = tot;
    return off + incl - v;
}

// Bound Delta on |s - r^2| for the direct-form FP32 value s of a row whose
// FP32 value is at most tau (its exact distance r is then at most
// Rm = sqrt(tau) (1-u)^(-(p+4)/2) + e2, e2 = 2uB sqrt(p)):
//     |s - r^2| <= ((1+u)^(p+4) - 1) (Rm + e2)^2 + 2 Rm e2 + e2^2,
// widened by 1e-6 relative, plus 2e-15 Rm^2 for the rounding of the FP64
// sums that define the order.  Two rows whose FP32 values differ by more
// than 2 Delta are in the same order by their FP64 distances, strictly.
// g_half >= (1 - u)^-(p+4)/2, g_full >= (1 + u)^(p+4), e2 = 2uB sqrt(p)
__device__ __forceinline__ double tie_bound(float tau, double g_half, double g_full, double e2) {
    const double Rm = sqrt((double)tau) * g_half * (1.0 + 1e-13) + e2;
    const double d0 = (g_full - 1.0) * (Rm + e2) * (Rm + e2) + 2.0 * Rm * e2 + e2 * e2;
    return d0 * (1.0 + 1e-6) + 2e-15 * Rm * Rm;
}

__device__ __forceinline__ bool pair_less(double da, uint32_t ra, double db, uint32_t rb) {
    return da < db || (da == db && ra < rb);
}

// One CTA per query.
//  (1) direct-form FP32 value s = sum (y_x - y_q)^2 of every collected row;
//  (2) radix selection of the N'-th smallest, v_k;
//  (3) survivors: rows with s <= screen_margin(v_k), which hold the exact
//      FP64 top N' (at least N' collected rows have s <= v_k, so the N'-th
//      exact distance is bounded as in the screen);
//  (4) bitonic sort of the survivors on (s, row) as one 64-bit key;
//  (5) runs of neighbours closer than 2 tie_bound get their exact FP64
//      distances (separately rounded subtract/multiply/add in coordinate
//      order, on the original coordinates) and are re-ordered on (d2, row)
//      within the run; outside the runs the FP32 order is the FP64 order.
//      A run longer than 32 sends the query to a full FP64 sort instead;
//  (6) the first N' rows.
// Ascending bitonic sort of sk[0, S) (S <= 1,024; the keys past S act as
// +infinity) by 256 threads, four keys a thread in registers: element e =
// 128 warp + 4 lane + r.  Compare-exchanges at distance 1, 2 stay in the
// thread, 4..64 go through warp shuffles, 128..512 through shared memory
// (two alternating buffers of 1,024 keys, sk and alt: one barrier a step).
// The sorted keys end in sk[0, 1024).
__device__ void sort1024_registers(unsigned long long *sk, int S, unsigned long long *alt) {
    static_assert(SORT_THREADS == 256, "four keys a thread for 1,024");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = warp * 128 + lane * 4;
    unsigned long long x[4];
#pragma unroll
    for (int r = 0; r < 4; r++) x[r] = base + r < S ? sk[base + r] : ~0ull;
    __syncthreads();  // every key is read before sk serves as an exchange buffer
    int buf = 0;
    for (int size = 2; size <= 1024; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 128) {
                unsigned long long *b = buf ? alt : sk;
                buf ^= 1;
#pragma unroll
                for (int r = 0; r < 4; r++) b[base + r] = x[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int e = base + r;
                    const unsigned long long y = b[e ^ stride];
                    // take y when it belongs here: smaller for the low end of an
                    // ascending pair (or the high end of a descending one)
                    if ((y < x[r]) == (((e & stride) == 0) == ((e & size) == 0))) x[r] = y;
                }
            } else if (stride >= 4) {
                const int lm = stride >> 2;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int e = base + r;
                    const unsigned long long y = __shfl_xor_sync(LAGP_FULL_MASK, x[r], lm);
                    if ((y < x[r]) == (((lane & lm) == 0) == ((e & size) == 0))) x[r] = y;
                }
            } else {
                // within the thread: pairs (0, 2), (1, 3) at distance 2, (0, 1),
                // (2, 3) at distance 1 (constant register indices)
                auto cx = [&](unsigned long long &a, unsigned long long &c, int e) {
                    const bool asc = (e & size) == 0;
                    if (asc ? c < a : a < c) {
                        const unsigned long long t = a;
                        a = c;
                        c = t;
                    }
                };
                if (stride == 2) {
                    cx(x[0], x[2], base);
                    cx(x[1], x[3], base + 1);
                } else {
                    cx(x[0], x[1], base);
                    cx(x[2], x[3], base + 2);
                }
            }
        }
    }
    __syncthreads();  // the last exchange buffer is read before sk is written
#pragma unroll
    for (int r = 0; r < 4; r++) sk[base + r] = x[r];
    __syncthreads();
}

__global__ void __launch_bounds__(SORT_THREADS)
knn_sort(const void *__restrict__ X, const float *__restrict__ Yv, int p, lagp_dtype dt,
         const void *__restrict__ Xref, int64_t M, const int32_t *__restrict__ Np, int32_t Npmax,
         const unsigned long long *__restrict__ kmax, const unsigned long long *__restrict__ kmin,
         const int32_t *__restrict__ cand, const int32_t *__restrict__ cand_count, int32_t Cmax,
         int32_t *__restrict__ idx, const KnnConst *__restrict__ kc, const float *__restrict__ rcol,
         int32_t *__restrict__ retry, int32_t *__restrict__ bigf, int big) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t q = blockIdx.x;
    // Two launches.  The first (big = 0, shared memory for up to 1,024
    // survivors) sorts every query but those flagged for the exact retry, and
    // flags (bigf) the ones with more survivors; the second (big = 1, shared
    // memory for any count) sorts the flagged ones of either kind.
    const bool flagged = (retry && retry[q] != 0) || (big && bigf[q] != 0);
    (void)kmax;
    (void)kmin;
    if (flagged != (big != 0)) return;
    const int C = cand_count[q];
    const int k = Np ? Np[q] : Npmax;
    int32_t *out = idx + q * Npmax;
    if (C < k || C > Cmax || k < 1 || k > Npmax) {  // invalid or overflowed: empty row
        for (int t = threadIdx.x; t < Npmax; t += SORT_THREADS) out[t] = -1;
        return;
    }
    int Cp = 1;
    while (Cp < Cmax) Cp <<= 1;
    // region 1 (R1 doubles): FP32 keys and rows for steps 1-3, then FP64 keys;
    // region 2 (R2 words of 64 bits): the survivors' (s, row) keys
    const int R1 = big ? Cp : (Cmax + 1) & ~1, R2 = big ? Cp : SORT_SMALL;
    uint32_t *key32 = reinterpret_cast<uint32_t *>(smem_raw);           // Cmax
    int32_t *rowA = reinterpret_cast<int32_t *>(key32 + R1);            // Cmax
    double *dk = reinterpret_cast<double *>(smem_raw);                  // R1
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem_raw + (size_t)R1 * 8);  // R2
    __shared__ double xq[64];
    __shared__ float yq[64];
    __shared__ float s_d2f;
    __shared__ uint32_t hist[256];
    __shared__ int wsum[SORT_THREADS / 32];
    __shared__ uint32_t s_prefix;
    __shared__ int s_kk, s_big, s_fail;
    __shared__ float s_tauf;
    __shared__ uint32_t tied[CAND_CAP / 32];
    if (threadIdx.x < p) {
        xq[threadIdx.x] = load_coord64(Xref, q, p, threadIdx.x, dt);
        yq[threadIdx.x] = (float)(xq[threadIdx.x] - kc->c[threadIdx.x]);
    }
    if (threadIdx.x == 0) {
        s_prefix = 0u;
        s_kk = k;
        s_big = 0;
    }
    __syncthreads();
    // (1) direct-form FP32 values (non-negative floats order like their
    // bits); four rows a thread in flight
    const int pv = (p + 3) & ~3;  // row stride of Yv
#pragma unroll 4
    for (int e = threadIdx.x; e < C; e += SORT_THREADS) {
        const int32_t r = cand[q * Cmax + e];
        const float4 *yr = reinterpret_cast<const float4 *>(Yv + (int64_t)r * pv);
        float sv = 0.f;
        for (int i4 = 0; i4 < pv; i4 += 4) {
            const float4 v = yr[i4 >> 2];
            const float t[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (i4 + j < p) {  // coordinate order, as the direct form defines
                    const float df = t[j] - yq[i4 + j];
                    sv = fmaf(df, df, sv);
                }
        }
        key32[e] = __float_as_uint(sv);  // NaN keeps the largest keys
        rowA[e] = r;
    }
    // (2) radix selection of the k-th smallest key, 8 bits at a time
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += SORT_THREADS) hist[b] = 0u;
        __syncthreads();
        const uint32_t prefix = s_prefix;
        const uint32_t hmask = shift == 24 ? 0u : (0xffffffffu << (shift + 8));
        // one atomic per distinct bin of a warp (most keys share their top bits)
        const int lane = threadIdx.x & 31;
        for (int e0 = threadIdx.x - lane; e0 < C; e0 += SORT_THREADS) {
            uint32_t bin = 0xFFFFFFFFu;
            if (e0 + lane < C) {
                const uint32_t kv = key32[e0 + lane];
                if ((kv & hmask) == prefix) bin = (kv >> shift) & 255u;
            }
            const unsigned peers = __match_any_sync(LAGP_FULL_MASK, bin);
            if (bin != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int kk = s_kk;
            uint32_t sub = 0;
            for (int b = 0; b < 8; b++) sub += hist[lane * 8 + b];
            uint32_t incl = sub;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(LAGP_FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned ball = __ballot_sync(LAGP_FULL_MASK, incl >= (uint32_t)kk);
            const int L = __ffs(ball) - 1;  // the k-th key is in lane L's bins
            if (lane == L) {
                uint32_t cum = incl - sub;
                int b = 0;
                for (; b < 7; b++) {
                    if (cum + hist[lane * 8 + b] >= (uint32_t)kk) break;
                    cum += hist[lane * 8 + b];
                }
                s_prefix = prefix | ((uint32_t)(lane * 8 + b) << shift);
                s_kk = kk - (int)cum;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // the margins with the launch's constants
        const double g = kc->g_half, e2 = kc->e2;
        const float vk = __uint_as_float(s_prefix);
        const double rk = sqrt((double)vk) * g * (1.0 + 1e-13) + e2;  // >= exact N'-th distance
        const float tauf = __double2float_rd(screen_margin_c(vk, g, e2));
        s_tauf = tauf;
        s_d2f = __double2float_ru(2.0 * tie_bound(tauf, g, kc->g_full, e2));
        // rows collected on the tensor cores: the N'-th of them must lie
        // within the radius collected in full, else the query goes to the
        // exact retry
        s_fail = rcol ? !(rk <= (double)rcol[q]) : 0;
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) retry[q] = 1;
        for (int t = threadIdx.x; t < Npmax; t += SORT_THREADS) out[t] = -1;
        return;
    }
    const float tauf = s_tauf;
    // (3) survivors, in candidate order, as (s, row) keys
    int mine = 0;
    for (int e = threadIdx.x; e < C; e += SORT_THREADS) mine += __uint_as_float(key32[e]) <= tauf;
    int S = 0;
    int pos = block_excl_scan(mine, wsum, &S);  // S is block-uniform
    int Sp = 1;
    while (Sp < S) Sp <<= 1;
    if (Sp > R2) {  // more survivors than this launch holds: the second launch sorts it
        if (threadIdx.x == 0) bigf[q] = 1;
        return;
    }
    for (int e = threadIdx.x; e < C; e += SORT_THREADS)
        if (__uint_as_float(key32[e]) <= tauf)
            sk[pos++] = ((unsigned long long)key32[e] << 32) | (uint32_t)rowA[e];
    for (int e = S + threadIdx.x; e < Sp; e += SORT_THREADS) sk[e] = ~0ull;
    __syncthreads();
    // (4) bitonic sort on (s, row): up to 1,024 keys in registers (four a
    // thread), else in shared memory
    if (Sp <= 4 * SORT_THREADS) {
        sort1024_registers(sk, S, reinterpret_cast<unsigned long long *>(smem_raw));
    } else {
        for (int size = 2; size <= Sp; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int e = threadIdx.x; e < (Sp >> 1); e += SORT_THREADS) {
                    const int lo = 2 * e - (e & (stride - 1)), hi = lo + stride;
                    const bool up = ((lo & size) == 0);
                    const unsigned long long ka = sk[lo], kb = sk[hi];
                    if (up ? kb < ka : ka < kb) {
                        sk[lo] = kb;
                        sk[hi] = ka;
                    }
                }
                __syncthreads();
            }
        }
    }
    // (5) runs of near-equal FP32 values: FP64 keys, ordered within the run
    const float d2f = s_d2f;  // twice the tie bound, rounded up
    auto gap_ok = [&](int i) {  // rows i and i + 1 are in a certain FP64 order
        // the FP32 difference rounded down never exceeds the true one
        const float a = __uint_as_float((uint32_t)(sk[i] >> 32));
        const float b = __uint_as_float((uint32_t)(sk[i + 1] >> 32));
        return __fsub_rd(b, a) > d2f;
    };
    auto fp64_key = [&](int i) {
        const int32_t r = (int32_t)(uint32_t)sk[i];
        double sd = 0.0;
        for (int t = 0; t < p; t++) {
            const double diff = __dsub_rn(xq[t], load_coord64(X, r, p, t, dt));
            sd = __dadd_rn(sd, __dmul_rn(diff, diff));
        }
        return sd;
    };
    // tie flags first (bit i: rows i and i + 1 need their FP64 order), so that
    // no run is re-ordered while another thread still reads its FP32 keys
    for (int w = threadIdx.x; w < (Sp + 31) / 32; w += SORT_THREADS) tied[w] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i + 1 < S; i += SORT_THREADS)
        if (!gap_ok(i)) atomicOr(&tied[i >> 5], 1u << (i & 31));
    __syncthreads();
    auto is_tied = [&](int i) { return (tied[i >> 5] >> (i & 31)) & 1u; };
    for (int i = threadIdx.x; i < S; i += SORT_THREADS) {
        if (!is_tied(i) || (i > 0 && is_tied(i - 1))) continue;  // not the start of a run
        int end = i + 1;  // the run is [i, end]
        while (is_tied(end) && end - i < 32) end++;
        if (end - i >= 32) {
            s_big = 1;
            continue;
        }
        for (int t = i; t <= end; t++) dk[t] = fp64_key(t);
        for (int t = i + 1; t <= end; t++) {  // insertion sort on (d2, row)
            const double dv = dk[t];
            const unsigned long long kv = sk[t];
            int u = t - 1;
            while (u >= i && pair_less(dv, (uint32_t)kv, dk[u], (uint32_t)sk[u])) {
                dk[u + 1] = dk[u];
                sk[u + 1] = sk[u];
                u--;
            }
            dk[u + 1] = dv;
            sk[u + 1] = kv;
        }
    }
    __syncthreads();
    if (s_big) {
        // a long run: exact FP64 keys for every survivor and a full sort on (d2, row)
        for (int i = threadIdx.x; i < Sp; i += SORT_THREADS) dk[i] = i < S ? fp64_key(i) : CUDART_INF;
        __syncthreads();
        for (int size = 2; size <= Sp; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int e = threadIdx.x; e < (Sp >> 1); e += SORT_THREADS) {
                    const int lo = 2 * e - (e & (stride - 1)), hi = lo + stride;
                    const bool up = ((lo & size) == 0);
                    const double da = dk[lo], db = dk[hi];
                    const unsigned long long ka = sk[lo], kb = sk[hi];
                    const bool swap = up ? pair_less(db, (uint32_t)kb, da, (uint32_t)ka)
                                         : pair_less(da, (uint32_t)ka, db, (uint32_t)kb);
                    if (swap) {
                        dk[lo] = db;
                        dk[hi] = da;
                        sk[lo] = kb;
                        sk[hi] = ka;
                    }
                }
                __syncthreads();
            }
        }
    }
    // (6)
    for (int t = threadIdx.x; t < Npmax; t += SORT_THREADS) out[t] = t < k ? (int32_t)(uint32_t)sk[t] : -1;
}

// The screen's first launch: the sampled threshold and the collection on the
// norm expansion (CUDA cores), or with tau0 the sampled threshold only (the
// collection then runs on the tensor cores); and the exact retry of the
// flagged queries on the direct form.
template <int P>
void launch_screen(lagp_ctx *ctx, bool retry_pass, dim3 grid, size_t smem, const float *Y32, const float *Ys,
                   int64_t N, int p, const void *Xref, lagp_dtype dt, int64_t M, const int32_t *Np, int32_t Npmax,
                   const unsigned long long *kmax, const unsigned long long *kmin, int32_t *cand, int32_t Cmax,
                   int32_t *cc, int32_t *status, int64_t stride, int32_t *retry, int *counters, float *tau0) {
    cudaStream_t st = ctx->stream;
    if (!retry_pass) {
        cudaFuncSetAttribute(knn_screen<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        knn_screen<P, true><<<grid, SCREEN_THREADS, smem, st>>>(Y32, Ys, N, p, Xref, dt, M, Np, Npmax, kmax, kmin,
                                                                cand, Cmax, cc, status, stride, retry, 0,
                                                                counters, tau0);
    } else {
        cudaFuncSetAttribute(knn_screen<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        knn_screen<P, false><<<grid, SCREEN_THREADS, smem, st>>>(Y32, Y32, N, p, Xref, dt, M, Np, Npmax, kmax,
                                                                 kmin, cand, Cmax, cc, status, 1, retry, 1,
                                                                 counters + 1, nullptr);
    }
    ctx->launches++;
}

}  // namespace

lagp_status launch_knn(lagp_ctx *ctx, const void *X, int64_t N, int p, lagp_dtype dtype,
                       const void *Xref, int64_t M, const int32_t *Np, int32_t Npmax,
                       int32_t *idx, int32_t *status) {
    cudaStream_t st = ctx->stream;
    ctx->knn_last_M = M;
    // sample stride: about 8 N' sampled rows per candidate set, 1 (exact) for small designs
    const int64_t stride = std::max<int64_t>(1, std::min<int64_t>(64, N / (8 * (int64_t)Npmax)));
    const int64_t nsamp = (N + stride - 1) / stride;
    // candidate capacity: the sampled threshold (the rtarget-th smallest of
    // every stride-th row, rtarget ~ 1.3 N' / stride + 16) collects about
    // rtarget stride rows with a spread of about sqrt(rtarget) stride; six of
    // those spreads above (and 512 rows for the error margins) leave an
    // overflow, and so an exact retry over the whole design (one CTA's pass
    // over all N rows: at N = 4M it sets the pass's duration), to about one
    // query in 1e9.  At least 2 N' + 1024, and no more than the power of two
    // at or above that (the second sort launch's shared memory, sized by
    // that power of two, keeps its resident CTAs), nor than the sort holds.
    int32_t Cmax = std::min(2 * Npmax + 1024, CAND_CAP);
    if (stride > 1) {
        int32_t pow2 = 1;
        while (pow2 < Cmax) pow2 <<= 1;
        const int64_t rt = std::min<int64_t>((13 * (int64_t)Npmax + 10 * stride - 1) / (10 * stride) + 16, nsamp);
        const double want = (double)rt * stride + 6.0 * std::sqrt((double)rt) * stride + 512.0;
        Cmax = (int32_t)std::min<double>(std::max<double>(Cmax, std::ceil(want)), std::min(pow2, CAND_CAP));
    }
    char *meta = static_cast<char *>(lagp_ws(ctx, WS_KNN_META, META_HEAD + (size_t)M * 12));
    int32_t *cand = static_cast<int32_t *>(lagp_ws(ctx, WS_KNN_CAND, (size_t)M * Cmax * 4));
    const int pp = row_stride(p);
    const int64_t Npad = round_up(N, 32);
    const int64_t nsamp_pad = stride > 1 ? round_up(nsamp, 32) : 0;
    const int pv = (p + 3) & ~3;
    float *Y32 = static_cast<float *>(lagp_ws(ctx, WS_KNN_X32, ((size_t)(Npad + nsamp_pad) * pp + (size_t)Npad * pv) * 4));
    if (!meta || !cand || !Y32) return LAGP_ENOMEM;
    float *Ys = stride > 1 ? Y32 + Npad * pp : Y32;
    float *Yv = Y32 + (Npad + nsamp_pad) * pp;  // 16-byte aligned: Npad is a multiple of 32
    int *counters = reinterpret_cast<int *>(meta + 64);
    unsigned long long *kmax = reinterpret_cast<unsigned long long *>(meta + 256);
    unsigned long long *kmin = reinterpret_cast<unsigned long long *>(meta + 768);
    int32_t *cc = reinterpret_cast<int32_t *>(meta + META_HEAD);
    int32_t *retry = cc + M;
    int32_t *bigf = retry + M;  // queries with more survivors than the first sort holds
    LAGP_CUDA(ctx, cudaMemsetAsync(meta, 0, META_HEAD, st));
    LAGP_CUDA(ctx, cudaMemsetAsync(bigf, 0, (size_t)M * 4, st));
    const int blocks = ctx->num_sms * 4;
    knn_bounds<<<blocks, 256, 0, st>>>(X, N, Xref, M, p, dtype, kmax, kmin);
    KnnConst *kc = reinterpret_cast<KnnConst *>(meta + META_CONST);
    knn_prep<<<blocks, 256, 0, st>>>(X, N, p, dtype, kmax, kmin, Y32, Npad, stride > 1 ? Ys : nullptr,
                                     nsamp_pad, stride, kc, Yv);
    ctx->launches += 2;
    LAGP_CUDA(ctx, cudaGetLastError());
    // collection on the tensor cores unless the tuning asks for CUDA cores
    void *tc_ws = nullptr;
    float *tau0 = nullptr, *rcol = nullptr;
    if (ctx->tuning.knn_path == 0 && knn_tc_supported(p)) {
        tc_ws = lagp_ws(ctx, WS_KNN_TC, knn_tc_workspace(N, M, p));
        if (!tc_ws) return LAGP_ENOMEM;
        LAGP_TRY(launch_knn_tc_prep(ctx, tc_ws, X, N, p, dtype, Xref, M, kmax, kmin, &tau0, &rcol));
    }
    int *tc_err = reinterpret_cast<int *>(meta);

    size_t smem = (size_t)QB * HB * 4 + 2 * (size_t)tile_len(pp) * pp * 4 + (size_t)(QB + 1) * pp * 4;
    // persistent grid: two CTAs per SM, blocks of QB queries from a counter
    const int64_t nblk = (M + QB - 1) / QB;
    dim3 grid((unsigned)std::min<int64_t>(nblk, (int64_t)ctx->num_sms * 2));
    int Cp = 1;
    while (Cp < Cmax) Cp <<= 1;
    // the first sort launch: up to SORT_SMALL survivors (more CTAs per SM);
    // the second: any count
    const size_t smem_small = (size_t)((Cmax + 1) & ~1) * 8 + (size_t)SORT_SMALL * 8;
    const size_t smem_big = (size_t)Cp * 16;
    if (smem_big > ctx->smem_optin) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: N' too large for the sort");
    cudaFuncSetAttribute(knn_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_big);
    auto screen = [&](bool retry_pass) {
        switch (p) {
            case 2: launch_screen<2>(ctx, retry_pass, grid, smem, Y32, Ys, N, p, Xref, dtype, M, Np, Npmax, kmax, kmin, cand, Cmax, cc, status, stride, retry, counters, tau0); break;
            case 3: launch_screen<3>(ctx, retry_pass, grid, smem, Y32, Ys, N, p, Xref, dtype, M, Np, Npmax, kmax, kmin, cand, Cmax, cc, status, stride, retry, counters, tau0); break;
            case 8: launch_screen<8>(ctx, retry_pass, grid, smem, Y32, Ys, N, p, Xref, dtype, M, Np, Npmax, kmax, kmin, cand, Cmax, cc, status, stride, retry, counters, tau0); break;
            default: launch_screen<0>(ctx, retry_pass, grid, smem, Y32, Ys, N, p, Xref, dtype, M, Np, Npmax, kmax, kmin, cand, Cmax, cc, status, stride, retry, counters, tau0); break;
        }
    };
    auto sort = [&](const float *rc, int32_t *rflags, int big) {
        knn_sort<<<(unsigned)M, SORT_THREADS, big ? smem_big : smem_small, st>>>(
            X, Yv, p, dtype, Xref, M, Np, Npmax, kmax, kmin, cand, cc, Cmax, idx, kc, rc, rflags, bigf, big);
        ctx->launches++;
    };
    screen(false);
    LAGP_CUDA(ctx, cudaGetLastError());
    if (tc_ws) {
        // collection on the tensor cores, the sort (which checks each query's
        // collection), the exact retry of the flagged queries and their sort
        LAGP_TRY(launch_knn_tc_collect(ctx, tc_ws, N, p, M, Np, Npmax, kmax, kmin, cand, Cmax, cc, status, retry,
                                       tc_err, rcol, nullptr));
        sort(rcol, retry, 0);
        screen(true);
        sort(nullptr, retry, 1);
    } else {
        screen(true);
        sort(nullptr, nullptr, 0);
        sort(nullptr, nullptr, 1);
    }
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

// Diagnostic: the tensor-core values s of every (query, design row) pair, as
// the collection pass computes them (out: M x N floats).
lagp_status launch_knn_tc_dist(lagp_ctx *ctx, const void *X, int64_t N, int p, lagp_dtype dtype,
                               const void *Xref, int64_t M, float *out) {
    if (!knn_tc_supported(p)) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn_tc_dist: p > 20");
    cudaStream_t st = ctx->stream;
    char *meta = static_cast<char *>(lagp_ws(ctx, WS_KNN_META, META_HEAD + (size_t)M * 12));
    void *tc_ws = lagp_ws(ctx, WS_KNN_TC, knn_tc_workspace(N, M, p));
    if (!meta || !tc_ws) return LAGP_ENOMEM;
    unsigned long long *kmax = reinterpret_cast<unsigned long long *>(meta + 256);
    unsigned long long *kmin = reinterpret_cast<unsigned long long *>(meta + 768);
    int32_t *cc = reinterpret_cast<int32_t *>(meta + META_HEAD);
    int32_t *retry = cc + M;
    LAGP_CUDA(ctx, cudaMemsetAsync(meta, 0, META_HEAD, st));
    knn_bounds<<<ctx->num_sms * 4, 256, 0, st>>>(X, N, Xref, M, p, dtype, kmax, kmin);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    float *tau0 = nullptr, *rcol = nullptr;
    LAGP_TRY(launch_knn_tc_prep(ctx, tc_ws, X, N, p, dtype, Xref, M, kmax, kmin, &tau0, &rcol));
    return launch_knn_tc_collect(ctx, tc_ws, N, p, M, nullptr, 1, kmax, kmin, nullptr, 1, cc, nullptr, retry,
                                 reinterpret_cast<int *>(meta), rcol, out);
}

// Diagnostic: of the last kNN call on the context, the queries that went to
// the exact retry and whether the tensor-core pass gave up on a wait.
lagp_status knn_last_stats(lagp_ctx *ctx, int64_t *n_retry, int32_t *tc_failed) {
    const int64_t M = ctx->knn_last_M;
    char *meta = static_cast<char *>(ctx->ws[WS_KNN_META]);
    if (!meta || M <= 0) {
        *n_retry = 0;
        *tc_failed = 0;
        return LAGP_OK;
    }
    std::vector<int32_t> r((size_t)M);
    int32_t f = 0;
    LAGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    LAGP_CUDA(ctx, cudaMemcpy(r.data(), meta + META_HEAD + (size_t)M * 4, (size_t)M * 4, cudaMemcpyDeviceToHost));
    LAGP_CUDA(ctx, cudaMemcpy(&f, meta, 4, cudaMemcpyDeviceToHost));
    int64_t n = 0;
    for (int32_t v : r) n += v != 0;
    *n_retry = n;
    *tc_failed = f;
    return LAGP_OK;
}
