// a1: exact N'-nearest-neighbour candidate sets (Sec. 3.1 of the paper: the
// ALC search runs over the N' nearest neighbours of x; Fig. 1 step 2(a)).
//
// Design (GB300): distances are screened in FP32 (74 TFLOP/s) and only the
// few candidates near the N'-th distance are re-ranked in FP64 (1.2 TFLOP/s).
//   knn_prep    FP32 copy of an FP64 design, and R = max |coordinate|.
//   knn_screen  one warp per query, eight queries per CTA sharing each design
//               tile in shared memory; three passes over the design:
//               (1) 2048-bin histogram of the FP32 distance bits [30:20],
//               (2) 2048-bin histogram of bits [19:9] inside the boundary bin,
//               giving tau >= the N'-th smallest FP32 distance,
//               (3) collect every row whose FP32 distance is below tau widened
//               by a rigorous FP32-vs-FP64 error margin (see screen_margin).
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

constexpr int QB = 8;                 // queries per CTA, one warp each
constexpr int SCREEN_THREADS = QB * 32;
constexpr int HB = 2048;              // histogram bins per level
constexpr int TILE_FLOATS = 8192;     // shared floats for one design tile
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

// FP32 screen distance of design tile point t to the warp's query (held in
// registers for the compile-time dimensions, in shared memory otherwise).
template <int P>
__device__ __forceinline__ float screen_d2(const float *tile, int stride, int t, const float (&qr)[P > 0 ? P : 1],
                                           const float *qsm, int p) {
    float s = 0.f;
    if constexpr (P > 0) {
#pragma unroll
        for (int i = 0; i < P; i++) {
            float df = tile[t * stride + i] - qr[i];
            s = fmaf(df, df, s);
        }
    } else {
        for (int i = 0; i < p; i++) {
            float df = tile[t * stride + i] - qsm[i];
            s = fmaf(df, df, s);
        }
    }
    return s;
}

template <int P>
__global__ void __launch_bounds__(SCREEN_THREADS, 2)
knn_screen(const float *__restrict__ X32, int64_t N, int p, const void *__restrict__ Xref,
           lagp_dtype dt, int64_t M, const int32_t *__restrict__ Np, int32_t Npmax,
           const unsigned long long *__restrict__ Rbits, int32_t *__restrict__ cand, int32_t Cmax,
           int32_t *__restrict__ cand_count, int32_t *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_raw);
    float *tile = reinterpret_cast<float *>(hist + QB * HB);
    float *qs = tile + TILE_FLOATS;
    __shared__ int32_t s_count[QB];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * QB + w;
    const bool active = q < M;
    const int k = active ? (Np ? Np[q] : Npmax) : 0;
    const bool ok = active && k >= 1 && k <= Npmax;
    const int stride = p + 1;  // odd stride: conflict-free per-lane rows
    int T = (TILE_FLOATS / stride) & ~31;
    if (T > 1024) T = 1024;

    float qreg[P > 0 ? P : 1] = {};
    for (int i = lane; i < p; i += 32) qs[w * p + i] = active ? load_coord32(Xref, q, p, i, dt) : 0.f;
    for (int b = lane; b < HB; b += 32) hist[w * HB + b] = 0;
    if (lane == 0) s_count[w] = 0;
    __syncthreads();
    if constexpr (P > 0) {
#pragma unroll
        for (int i = 0; i < P; i++) qreg[i] = qs[w * p + i];
    }
    const double R = __longlong_as_double((long long)*Rbits);

    uint32_t b1 = 0, before = 0;
    double tau2 = 0.0;
    for (int pass = 0; pass < 3; pass++) {
        for (int64_t base = 0; base < N; base += T) {
            const int cnt = (int)min((int64_t)T, N - base);
            __syncthreads();
            const float *src = X32 + base * p;
            for (int e = threadIdx.x; e < cnt * p; e += SCREEN_THREADS) {
                int t = e / p, i = e - t * p;
                tile[t * stride + i] = src[e];
            }
            __syncthreads();
            if (ok) {
                for (int t = lane; t < cnt; t += 32) {
                    float s = screen_d2<P>(tile, stride, t, qreg, qs + w * p, p);
                    uint32_t bits = __float_as_uint(s);
                    uint32_t hi = (bits >> 20) & 0x7FFu;
                    if (pass == 0) {
                        atomicAdd(&hist[w * HB + hi], 1u);
                    } else if (pass == 1) {
                        if (hi == b1) atomicAdd(&hist[w * HB + ((bits >> 9) & 0x7FFu)], 1u);
                    } else if ((double)s <= tau2) {
                        int pos = atomicAdd(&s_count[w], 1);
                        if (pos < Cmax) cand[q * Cmax + pos] = (int32_t)(base + t);
                    }
                }
            }
        }
        __syncthreads();
        if (ok && pass == 0) {
            find_bin(hist + w * HB, (uint32_t)k, lane, b1, before);
            __syncwarp();
            for (int b = lane; b < HB; b += 32) hist[w * HB + b] = 0;
        } else if (ok && pass == 1) {
            uint32_t b2, before2;
            find_bin(hist + w * HB, (uint32_t)k - before, lane, b2, before2);
            float tau = __uint_as_float((b1 << 20) | (b2 << 9) | 0x1FFu);
            tau2 = screen_margin(tau, p, R);
        }
        __syncthreads();
    }
    if (active && lane == 0) {
        cand_count[q] = ok ? s_count[w] : 0;
        // fewer rows than N' under the threshold only happens with non-finite
        // distances (NaN or overflowing coordinates)
        if (status)
            status[q] = !ok || s_count[w] < k ? LAGP_EINVAL
                                              : (s_count[w] > Cmax ? LAGP_ENOMEM : LAGP_OK);
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
                   int32_t *status) {
    cudaFuncSetAttribute(knn_screen<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    knn_screen<P><<<grid, SCREEN_THREADS, smem, st>>>(X32, N, p, Xref, dt, M, Np, Npmax, Rb, cand,
                                                      Cmax, cc, status);
}

}  // namespace

lagp_status launch_knn(lagp_ctx *ctx, const void *X, int64_t N, int p, lagp_dtype dtype,
                       const void *Xref, int64_t M, const int32_t *Np, int32_t Npmax,
                       int32_t *idx, int32_t *status) {
    cudaStream_t st = ctx->stream;
    const int32_t Cmax = std::min(2 * Npmax + 1024, CAND_CAP);
    // meta: R bits (8 bytes), then per-query candidate counts
    char *meta = static_cast<char *>(lagp_ws(ctx, WS_KNN_META, 256 + (size_t)M * 4));
    int32_t *cand = static_cast<int32_t *>(lagp_ws(ctx, WS_KNN_CAND, (size_t)M * Cmax * 4));
    if (!meta || !cand) return LAGP_ENOMEM;
    unsigned long long *Rbits = reinterpret_cast<unsigned long long *>(meta);
    int32_t *cc = reinterpret_cast<int32_t *>(meta + 256);
    LAGP_CUDA(ctx, cudaMemsetAsync(Rbits, 0, 8, st));
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

    size_t smem = (size_t)QB * HB * 4 + (size_t)TILE_FLOATS * 4 + (size_t)QB * p * 4;
    dim3 grid((unsigned)((M + QB - 1) / QB));
    switch (p) {
        case 2: launch_screen<2>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status); break;
        case 3: launch_screen<3>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status); break;
        case 8: launch_screen<8>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status); break;
        default: launch_screen<0>(grid, smem, st, X32, N, p, Xref, dtype, M, Np, Npmax, Rbits, cand, Cmax, cc, status); break;
    }
    ctx->launches++;
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
