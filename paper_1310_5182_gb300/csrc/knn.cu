// a1: exact N'-nearest-neighbour candidate sets (Sec. 3.1 of the paper: the
// ALC search runs over the N' nearest neighbours of x; Fig. 1 step 2(a)).
//
// Design (GB300): distances are screened in FP32 (74 TFLOP/s) and only the
// few candidates near the N'-th distance are re-ranked in FP64 (1.2 TFLOP/s).
//   knn_prep    FP32 copy of an FP64 design, and R = max |coordinate|.
//   knn_screen  persistent; 16 queries per CTA, two per warp, sharing every
//               design tile in shared memory:
//               (A, B) 2-level histogram (FP32 distance bits [30:21], then
//               [20:11] inside the boundary bin) over a strided sample of the
//               design, giving a threshold tau0 expected to bound about 1.3 N'
//               rows (with stride 1, exactly the N'-th smallest distance);
//               (C) one pass over the whole design collecting every row below
//               tau0 widened by a rigorous FP32-vs-FP64 error margin (see
//               screen_margin) and counting the rows below tau0.  A query
//               whose count is short of N', or whose buffer overflowed, is
//               redone by a second launch with stride 1 (the exact method).
//   knn_sort    one CTA per query: exact FP64 distances of the collected rows
//               (separately rounded subtract/multiply/add in coordinate order),
//               bitonic sort on (d2, row), first N' rows written out.
// The collected set provably contains the exact FP64 top-N', so the result
// equals an FP64 sort of all N rows bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "lagp_internal.h"

namespace {

constexpr int QPW = 2;                // queries per warp
constexpr int SCREEN_THREADS = 256;
constexpr int QB = QPW * SCREEN_THREADS / 32;  // 16 queries per CTA
constexpr int HB = 1024;              // histogram bins per level (10 bits)
constexpr int L1_SHIFT = 21;          // level 1: FP32 distance bits [30:21]
constexpr int L2_SHIFT = 11;          // level 2: bits [20:11] inside the boundary bin
constexpr uint32_t L2_LOW = (1u << L2_SHIFT) - 1;
constexpr int TILE_FLOATS = 4096;     // floats of one design tile (tile length x p)
constexpr int STAGE = TILE_FLOATS / SCREEN_THREADS;  // floats a thread stages per tile

// Design points per tile: a multiple of 32 with tile length x p <= TILE_FLOATS,
// at most 512.
__host__ __device__ inline int tile_len(int p) {
    int t = (TILE_FLOATS / p) & ~31;
    return t > 512 ? 512 : (t < 32 ? 32 : t);
}
constexpr int CAND_CAP = 8192;        // candidate capacity cap (sort in shared memory)
constexpr int SORT_THREADS = 256;

__global__ void knn_prep(const double *__restrict__ X, int64_t nX, const double *__restrict__ Xr,
                         int64_t nR, float *__restrict__ X32, unsigned long long *Rbits) {
    double mx = 0.0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nX; i += stride) {
        double v = X[i];
        X32[i] = static_cast<float>(v);
        mx = fmax(mx, fabs(v));
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nR; i += stride)
        mx = fmax(mx, fabs(Xr[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(LAGP_FULL_MASK, mx, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(Rbits, (unsigned long long)__double_as_longlong(mx));
}

// Widened threshold for the collection pass.  With u = 2^-24, coordinates
// rounded to FP32 with absolute error <= u R (R = 0 for FP32 inputs), FP32
// differences, squares and sums each rounded once, the FP32 screen value s of
// a row at exact distance r satisfies
//     (1-u)^((p+4)/2) (r - 2uR sqrt(p)) <= sqrt(s) <= (1+u)^((p+4)/2) (r + 2uR sqrt(p)).
// Every row with s <= tau then has r <= r_hi = sqrt(tau) (1-u)^(-(p+4)/2) + 2uR sqrt(p),
// so the N'-th exact distance is <= r_hi, and every row of the exact top-N' has
// sqrt(s) <= (r_hi + 2uR sqrt(p)) (1+u)^((p+4)/2).  The final factor covers the
// rounding of the FP64 reference distances and of this computation.
__device__ double screen_margin(float tau, int p, double R) {
    const double u = 5.9604644775390625e-08;  // 2^-24
    double e2 = 2.0 * u * R * sqrt((double)p);
    double r = sqrt((double)tau);
    double r_hi = r * pow(1.0 - u, -0.5 * (p + 4)) + e2;
    double r_col = (r_hi + e2) * pow(1.0 + u, 0.5 * (p + 4));
    return r_col * r_col * (1.0 + 1e-12);
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

// One design tile against a warp's QPW queries.  PASS 0: level-1 histogram;
// PASS 1: level-2 histogram inside the boundary bin; PASS 2: collection.
template <int P, int PASS>
__device__ __forceinline__ void screen_tile(const float *t, int TS, int cnt, int lane, int p,
                                            const float (&qr)[QPW][P > 0 ? P : 1],
                                            const float *qsw, const bool (&ok)[QPW], uint32_t *histw,
                                            const uint32_t (&b1)[QPW], const float (&tau0)[QPW],
                                            const float (&tau2f)[QPW], int32_t *cntw, int32_t *cnt0w,
                                            int32_t *__restrict__ cand, const int64_t (&q)[QPW],
                                            int32_t Cmax, int64_t base) {
    for (int pt = lane; pt < cnt; pt += 32) {
        float sd[QPW] = {};
        if constexpr (P > 0) {
#pragma unroll
            for (int i = 0; i < P; i++) {
                const float x = t[i * TS + pt];
#pragma unroll
                for (int h = 0; h < QPW; h++) {
                    const float df = x - qr[h][i];
                    sd[h] = fmaf(df, df, sd[h]);
                }
            }
        } else {
            for (int i = 0; i < p; i++) {
                const float x = t[i * TS + pt];
#pragma unroll
                for (int h = 0; h < QPW; h++) {
                    const float df = x - qsw[h * p + i];
                    sd[h] = fmaf(df, df, sd[h]);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < QPW; h++) {
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
//   Pass C: every row whose FP32 distance is <= screen_margin(tau0) is
//   collected, and the rows <= tau0 are counted; when that count reaches N'
//   the collected set provably holds the exact FP64 top N' (see
//   screen_margin).  Otherwise (a sample that underestimated the threshold)
//   or when the buffer overflows, the query is flagged for the exact retry.
template <int P>
__global__ void __launch_bounds__(SCREEN_THREADS, 2)
knn_screen(const float *__restrict__ X32, int64_t N, int p, const void *__restrict__ Xref,
           lagp_dtype dt, int64_t M, const int32_t *__restrict__ Np, int32_t Npmax,
           const unsigned long long *__restrict__ Rbits, int32_t *__restrict__ cand, int32_t Cmax,
           int32_t *__restrict__ cand_count, int32_t *__restrict__ status, int64_t stride,
           int32_t *__restrict__ retry, int retry_pass, int *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TT = tile_len(p), TS = TT + 1;  // tile length and padded stride
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_raw);   // QB x HB
    float *tiles = reinterpret_cast<float *>(hist + QB * HB);  // 2 x p x TS
    float *qs = tiles + 2 * (size_t)p * TS;                      // QB x p
    __shared__ int32_t s_count[QB], s_count0[QB];
    __shared__ int64_t s_blk;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double R = __longlong_as_double((long long)*Rbits);
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
            for (int i = lane; i < p; i += 32) qs[ql * p + i] = active[h] ? load_coord32(Xref, q[h], p, i, dt) : 0.f;
            for (int b = lane; b < HB; b += 32) hist[ql * HB + b] = 0;
            if (lane == 0) s_count[ql] = s_count0[ql] = 0;
        }
        if (!__syncthreads_or(mine_any)) continue;  // nothing to do in this block
        float qr[QPW][P > 0 ? P : 1] = {};
        if constexpr (P > 0) {
#pragma unroll
            for (int h = 0; h < QPW; h++)
#pragma unroll
                for (int i = 0; i < P; i++) qr[h][i] = qs[(w * QPW + h) * p + i];
        }

        uint32_t b1[QPW] = {}, before[QPW] = {};
        // thresholds as floats: for a float distance s, s <= t (t real) holds
        // exactly when s <= t rounded down to a float, so the hot loop compares
        // in FP32 (an FP64 compare per point would occupy the slow FP64 unit)
        float tau0[QPW] = {}, tau2f[QPW] = {};
        for (int pass = 0; pass < 3; pass++) {
            const int64_t rstride = pass < 2 ? stride : 1;  // passes A, B: sampled rows
            const int64_t nrows = pass < 2 ? nsamp : N;
            const int64_t ntiles = (nrows + TT - 1) / TT;
            float stage[STAGE];
            auto load_stage = [&](int64_t tile) {
                const int64_t base = tile * TT;
                const int cnt = (int)min((int64_t)TT, nrows - base);
#pragma unroll
                for (int u = 0; u < STAGE; u++) {
                    const int e = threadIdx.x + u * SCREEN_THREADS;
                    if (e < cnt * p) {
                        const int pt = (P > 0) ? e / P : e / p, i = e - pt * p;
                        stage[u] = X32[(base + pt) * rstride * p + i];
                    } else {
                        stage[u] = 0.f;
                    }
                }
            };
            auto store_stage = [&](int buf) {
                float *t = tiles + (size_t)buf * p * TS;
#pragma unroll
                for (int u = 0; u < STAGE; u++) {
                    const int e = threadIdx.x + u * SCREEN_THREADS;
                    if (e < TT * p) {
                        const int pt = (P > 0) ? e / P : e / p, i = e - pt * p;
                        t[i * TS + pt] = stage[u];
                    }
                }
            };
            load_stage(0);
            store_stage(0);
            __syncthreads();
            for (int64_t tile = 0; tile < ntiles; tile++) {
                const int buf = (int)(tile & 1);
                if (tile + 1 < ntiles) load_stage(tile + 1);  // in flight during the screen
                const int64_t base = tile * TT;
                const int cnt = (int)min((int64_t)TT, nrows - base);
                const float *t = tiles + (size_t)buf * p * TS;
                if (pass == 0)
                    screen_tile<P, 0>(t, TS, cnt, lane, p, qr, qs + w * QPW * p, ok, hist + w * QPW * HB,
                                      b1, tau0, tau2f, s_count + w * QPW, s_count0 + w * QPW, cand, q,
                                      Cmax, base);
                else if (pass == 1)
                    screen_tile<P, 1>(t, TS, cnt, lane, p, qr, qs + w * QPW * p, ok, hist + w * QPW * HB,
                                      b1, tau0, tau2f, s_count + w * QPW, s_count0 + w * QPW, cand, q,
                                      Cmax, base);
                else
                    screen_tile<P, 2>(t, TS, cnt, lane, p, qr, qs + w * QPW * p, ok, hist + w * QPW * HB,
                                      b1, tau0, tau2f, s_count + w * QPW, s_count0 + w * QPW, cand, q,
                                      Cmax, base);
                __syncthreads();  // every warp is done with the other buffer
                if (tile + 1 < ntiles) store_stage(buf ^ 1);
                __syncthreads();
            }
#pragma unroll
            for (int h = 0; h < QPW; h++) {
                if (!ok[h]) continue;
                uint32_t *hh = hist + (w * QPW + h) * HB;
                if (pass == 0) {
                    find_bin(hh, (uint32_t)rtarget[h], lane, b1[h], before[h]);
                    __syncwarp();
                    for (int b = lane; b < HB; b += 32) hh[b] = 0;
                } else if (pass == 1) {
                    uint32_t b2, before2;
                    find_bin(hh, (uint32_t)rtarget[h] - before[h], lane, b2, before2);
                    tau0[h] = __uint_as_float((b1[h] << L1_SHIFT) | (b2 << L2_SHIFT) | L2_LOW);
                    tau2f[h] = __double2float_rd(screen_margin(tau0[h], p, R));
                }
                __syncwarp();
            }
            __syncthreads();
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

__device__ __forceinline__ bool key_less(unsigned long long ka, int32_t ra, unsigned long long kb,
                                         int32_t rb) {
    return ka < kb || (ka == kb && ra < rb);
}

__global__ void __launch_bounds__(SORT_THREADS)
knn_sort(const void *__restrict__ X, int p, lagp_dtype dt, const void *__restrict__ Xref,
         int64_t M, const int32_t *__restrict__ Np, int32_t Npmax, const int32_t *__restrict__ cand,
         const int32_t *__restrict__ cand_count, int32_t Cmax, int32_t *__restrict__ idx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t q = blockIdx.x;
    const int C = cand_count[q];
    const int k = Np ? Np[q] : Npmax;
    int32_t *out = idx + q * Npmax;
    if (C < k || C > Cmax || k < 1 || k > Npmax) {  // invalid or overflowed: empty row
        for (int t = threadIdx.x; t < Npmax; t += SORT_THREADS) out[t] = -1;
        return;
    }
    int Cp = 1;
    while (Cp < C) Cp <<= 1;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem_raw);
    int32_t *rows = reinterpret_cast<int32_t *>(keys + Cp);
    double *xq = reinterpret_cast<double *>(rows + Cp + (Cp & 1));
    for (int i = threadIdx.x; i < p; i += SORT_THREADS) xq[i] = load_coord64(Xref, q, p, i, dt);
    __syncthreads();
    for (int e = threadIdx.x; e < Cp; e += SORT_THREADS) {
        if (e < C) {
            int32_t r = cand[q * Cmax + e];
            double s = 0.0;
            for (int i = 0; i < p; i++) {
                double diff = __dsub_rn(xq[i], load_coord64(X, r, p, i, dt));
                s = __dadd_rn(s, __dmul_rn(diff, diff));
            }
            keys[e] = (unsigned long long)__double_as_longlong(s);
            rows[e] = r;
        } else {
            keys[e] = ~0ull;
            rows[e] = INT32_MAX;
        }
    }
    __syncthreads();
    // bitonic sort, ascending (key, row)
    for (int size = 2; size <= Cp; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int e = threadIdx.x; e < (Cp >> 1); e += SORT_THREADS) {
                int lo = 2 * e - (e & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                unsigned long long ka = keys[lo], kb = keys[hi];
                int32_t ra = rows[lo], rb = rows[hi];
                bool swap = up ? key_less(kb, rb, ka, ra) : key_less(ka, ra, kb, rb);
                if (swap) {
                    keys[lo] = kb;
                    keys[hi] = ka;
                    rows[lo] = rb;
                    rows[hi] = ra;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < Npmax; t += SORT_THREADS) out[t] = t < k ? rows[t] : -1;
}

template <int P>
void launch_screen(dim3 grid, size_t smem, cudaStream_t st, const float *X32, int64_t N, int p,
                   const void *Xref, lagp_dtype dt, int64_t M, const int32_t *Np, int32_t Npmax,
                   const unsigned long long *Rb, int32_t *cand, int32_t Cmax, int32_t *cc,
                   int32_t *status, int64_t stride, int32_t *retry, int *counters) {
    cudaFuncSetAttribute(knn_screen<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // sampled threshold, then the exact retry of the flagged queries
    knn_screen<P><<<grid, SCREEN_THREADS, smem, st>>>(X32, N, p, Xref, dt, M, Np, Npmax, Rb, cand,
                                                      Cmax, cc, status, stride, retry, 0, counters);
    knn_screen<P><<<grid, SCREEN_THREADS, smem, st>>>(X32, N, p, Xref, dt, M, Np, Npmax, Rb, cand,
                                                      Cmax, cc, status, 1, retry, 1, counters + 1);
}

}  // namespace

lagp_status launch_knn(lagp_ctx *ctx, const void *X, int64_t N, int p, lagp_dtype dtype,
                       const void *Xref, int64_t M, const int32_t *Np, int32_t Npmax,
                       int32_t *idx, int32_t *status) {
    cudaStream_t st = ctx->stream;
    const int32_t Cmax = std::min(2 * Npmax + 1024, CAND_CAP);
    // meta: R bits (8 bytes) and two block counters, then per-query candidate
    // counts and retry flags
    char *meta = static_cast<char *>(lagp_ws(ctx, WS_KNN_META, 256 + (size_t)M * 8));
    int32_t *cand = static_cast<int32_t *>(lagp_ws(ctx, WS_KNN_CAND, (size_t)M * Cmax * 4));
    if (!meta || !cand) return LAGP_ENOMEM;
    unsigned long long *Rbits = reinterpret_cast<unsigned long long *>(meta);
    int32_t *cc = reinterpret_cast<int32_t *>(meta + 256);
    int32_t *retry = cc + M;
    int *counters = reinterpret_cast<int *>(meta + 64);
    LAGP_CUDA(ctx, cudaMemsetAsync(meta, 0, 256, st));
    const float *X32;
    if (dtype == LAGP_F64) {
        float *x32 = static_cast<float *>(lagp_ws(ctx, WS_KNN_X32, (size_t)N * p * 4));
        if (!x32) return LAGP_ENOMEM;
        int blocks = ctx->num_sms * 4;
        knn_prep<<<blocks, 256, 0, st>>>(static_cast<const double *>(X), N * p,
                                         static_cast<const double *>(Xref), M * p, x32, Rbits);
        ctx->launches++;
        X32 = x32;
    } else {
        X32 = static_cast<const float *>(X);  // FP32 inputs: exact, R term not needed
    }
    LAGP_CUDA(ctx, cudaGetLastError());

    size_t smem = (size_t)QB * HB * 4 + 2 * (size_t)p * (tile_len(p) + 1) * 4 + (size_t)QB * p * 4;
    // persistent grid: two CTAs per SM, blocks of QB queries from a counter
    const int64_t nblk = (M + QB - 1) / QB;
    dim3 grid((unsigned)std::min<int64_t>(nblk, (int64_t)ctx->num_sms * 2));
    // sample stride: about 8 N' sampled rows per candidate set, 1 (exact) for small designs
    const int64_t stride = std::max<int64_t>(1, std::min<int64_t>(64, N / (8 * (int64_t)Npmax)));
    switch (p) {
        case 2: launch_screen<2>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status, stride, retry, counters); break;
        case 3: launch_screen<3>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status, stride, retry, counters); break;
        case 8: launch_screen<8>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status, stride, retry, counters); break;
        default: launch_screen<0>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status, stride, retry, counters); break;
    }
    ctx->launches += 2;
    LAGP_CUDA(ctx, cudaGetLastError());

    int Cp = 1;
    while (Cp < Cmax) Cp <<= 1;
    size_t smem_sort = (size_t)Cp * 12 + 8 + (size_t)p * 8 + 16;
    if (smem_sort > ctx->smem_optin) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: N' too large for the sort");
    cudaFuncSetAttribute(knn_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sort);
    knn_sort<<<(unsigned)M, SORT_THREADS, smem_sort, st>>>(X, p, dtype, Xref, M, Np, Npmax, cand, cc,
                                                           Cmax, idx);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
