// a1, collection pass of the exact N'-nearest-neighbour screen on the
// tensor cores (Sec. 3.1: the candidate set of a location is its N' nearest
// design points).
//
// The squared distances s = |y_q|^2 + |y_x|^2 - 2 y_q . y_x between centred
// FP32 coordinates form a dense (design x queries) contraction over the p
// coordinates, here one tcgen05.mma chain (kind::f16, FP32 accumulation) per
// 128 design rows.  The coordinates are scaled by the power of two 2^-e that
// brings them into [-1, 1] (exact), and every FP32 value v enters as a
// two-term FP16 split v = v_h + v_l, the dot product as the three products
//   y_qh . y_xh + y_ql . y_xh + y_qh . y_xl        (y_ql . y_xl dropped),
// each exact in FP32; the two squared norms enter split the same way against
// unit entries.  Operand rows (K FP16 values each, K = 3p + 4 rounded up to
// 16, one MMA instruction per 16):
//   design x: ( y_xh, y_xh, y_xl, 1, 1, n_xh, n_xl, 0 ... )
//   query q:  ( -2 y_qh, -2 y_ql, -2 y_qh, n_qh, n_ql, 1, 1, 0 ... )
// so that the accumulator holds s 2^-2e for every (design row, query) pair.
//
// Exactness: the rows with s <= tau2 are collected, tau2 a rigorous widening
// (tc_margin) of the sampled threshold tau0 (itself widened by 2 E_tc so that
// rows at the sample's boundary fall inside whatever the rounding of either
// pass).  The sort then checks that the N'-th collected row lies within the
// radius that tau2 guarantees collected (tc_collected_radius, stored per
// query); a query that
// fails, or whose buffer overflows, goes to the exact CUDA-core retry.  E_tc
// (knn_common.cuh) assumes that one tensor-core instruction adds its products
// and accumulator with an error of at most TC_ACC_ULPS = 64 units of 2^-24
// times the sum of their magnitudes, several times what a truncating
// alignment of its seventeen addends can lose.
//
// Kernel layout (one CTA per SM, persistent over blocks of up to 128
// queries): warp 0 streams the design operand into a ring of shared-memory
// stages with bulk asynchronous copies, warp 1 owns the tensor memory and
// issues the MMAs (one thread) into four accumulators of 128 columns, and
// four groups of four epilogue warps (one per TMEM lane quarter; group g
// takes the design blocks it = g mod 4, accumulator g) read the distances
// back.  A lane compares its design row's distances with the queries'
// thresholds into a bit mask, two columns per FP16 x 2 compare (values
// rounded down, thresholds up: no hit is lost); only the set bits (about
// 1.5% of the pairs) are visited to append the row to the query's candidate
// list.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "device_util.cuh"
#include "knn_common.cuh"
#include "lagp_internal.h"
#include "tc_sm100.cuh"

namespace {

constexpr int TC_EPI_GROUPS = 4;  // epilogue groups of four warps (one per TMEM lane quarter)
constexpr int TC_THREADS = 64 + 128 * TC_EPI_GROUPS;  // warp 0: copies, warp 1: TMEM + MMA, then the epilogue
constexpr int TC_MROWS = 128;    // design rows per MMA (M)
constexpr int TC_STAGES_MAX = 8; // design stages in flight (fewer for wide rows)
constexpr int TC_NACC = 4;       // TMEM accumulators (128 columns each)
constexpr int TC_ACC_COLS = 128;
constexpr int TC_TMEM_COLS = TC_NACC * TC_ACC_COLS;  // 512: the whole tensor memory of the SM
constexpr int TC_QMAX = 128;     // queries per block (MMA N <= 128)
constexpr int TC_QUE = 32 * (TC_QMAX / 16);  // hit-queue entries of an epilogue warp: one a lane and chunk

// Half offset of element k of operand row r in the no-swizzle K-major
// layout: 8-row groups of K / 8 core matrices (8 rows x 8 halves, 128 bytes),
// the core matrices of a group adjacent along K.
__device__ __forceinline__ int64_t tc_off(int64_t r, int k, int K) {
    return (r >> 3) * (8 * (int64_t)K) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// Two FP32 values as FP16 x 2, rounded toward zero with negatives clamped to
// zero (never above the value they stand for, for a value >= 0; NaN stays
// NaN): x in the low half, y in the high half.
__device__ __forceinline__ uint32_t f16x2_rz_relu(float x, float y) {
    uint32_t r;
    asm("cvt.rz.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(y), "f"(x));
    return r;
}
// per half: 0xFFFF when a <= b, else 0 (NaN: 0)
__device__ __forceinline__ uint32_t le_mask_h2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("set.le.u32.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// v = h + l with h, l FP16 (round to nearest): |v - h - l| <= max(2^-22 |v|, 2^-25)
// for |v| <= 2
__device__ __forceinline__ void f16_split(float v, __half &h, __half &l) {
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
}

// The centred FP32 coordinates y and squared norm n of row r of A, exactly as
// the CUDA-core screen computes them (the norm an FMA chain in coordinate
// order).
__device__ __forceinline__ float centred_coords(const void *A, int64_t r, int p, lagp_dtype dt,
                                                const double *c, float *y) {
    float n2 = 0.f;
    for (int i = 0; i < p; i++) {
        y[i] = (float)(load_coord64(A, r, p, i, dt) - c[i]);
        n2 = fmaf(y[i], y[i], n2);
    }
    return n2;
}

// Design operand (Npad rows, blocked layout; rows past N are zero) and query
// operand rows (M x K, row-major), FP16.
__global__ void knn_tc_prep(const void *__restrict__ X, int64_t N, int64_t Npad, const void *__restrict__ Xr,
                            int64_t M, int p, lagp_dtype dt, const unsigned long long *kmax,
                            const unsigned long long *kmin, __half *__restrict__ A, __half *__restrict__ Q) {
    __shared__ double c[64];
    __shared__ double sB;
    if (threadIdx.x == 0) centre_and_bound(kmax, kmin, p, c, sB);
    __syncthreads();
    const int K = tc_k(p);
    const float scale = ldexpf(1.f, -tc_scale_exp(sB));
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float y[20];
    __half row[64];  // p <= 20, K <= 64 (knn_tc_supported)
    const __half one = __float2half_rn(1.f), zero = __float2half_rn(0.f);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < Npad + M; r += stride) {
        const bool des = r < Npad;
        const int64_t rr = des ? r : r - Npad;
        for (int k = 0; k < K; k++) row[k] = zero;
        if (!des || rr < N) {
            centred_coords(des ? X : Xr, rr, p, dt, c, y);
            float n2 = 0.f;  // |y 2^-e|^2: the FP32 chain of the unscaled norm, scaled exactly
            for (int i = 0; i < p; i++) {
                y[i] *= scale;
                n2 = fmaf(y[i], y[i], n2);
            }
            __half nh, nl;
            f16_split(n2, nh, nl);
            for (int i = 0; i < p; i++) {
                __half vh, vl;
                f16_split(des ? y[i] : -2.f * y[i], vh, vl);  // -2 y_q: an exact scaling
                row[i] = vh;
                row[p + i] = des ? vh : vl;
                row[2 * p + i] = des ? vl : vh;
            }
            row[3 * p] = des ? one : nh;
            row[3 * p + 1] = des ? one : nl;
            row[3 * p + 2] = des ? nh : one;
            row[3 * p + 3] = des ? nl : one;
        }
        __half *dst = des ? A : Q + rr * K;
        for (int k = 0; k < K; k += 8) {
            uint4 v;
            __half *hv = reinterpret_cast<__half *>(&v);
            for (int j = 0; j < 8; j++) hv[j] = row[k + j];
            *reinterpret_cast<uint4 *>(des ? dst + tc_off(rr, k, K) : dst + k) = v;
        }
    }
}

struct TcArgs {
    const __half *A;  // design operand, nmb * 128 rows
    const __half *Q;  // query operand rows, M x K
    int64_t N, M;
    int p, K, nmb;
    const float *tau0;  // per query: sampled threshold, NaN = not screened
    float *rcol;        // per query out: the radius collected in full (rounded down; NaN: not collected)
    const int32_t *Np;
    int32_t Npmax;
    const unsigned long long *kmax, *kmin;
    int32_t *cand, Cmax;
    int32_t *cand_count, *status, *retry;
    int nq, nblocks;  // queries per block, blocks
    int stages;       // shared-memory stages of the design ring
    float *dump;      // diagnostic: every value s (M x N) instead of the collection
    int stall;        // test hook: the producer stops after the first design block
    int *err;         // raised when a bounded wait gave up (the block's queries go to the retry)
};

__global__ void __launch_bounds__(TC_THREADS, 1) knn_screen_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int K = a.K, S = a.stages;
    const int stage_halves = TC_MROWS * K;
    __half *sA = reinterpret_cast<__half *>(smem_raw);         // S stages x 128 rows
    __half *sQ = sA + (size_t)S * stage_halves;                // TC_QMAX rows
    float *s_tau2 = reinterpret_cast<float *>(sQ + (size_t)TC_QMAX * K);  // TC_QMAX
    uint32_t *s_t2h = reinterpret_cast<uint32_t *>(s_tau2 + TC_QMAX);  // TC_QMAX/2: FP16 x 2, rounded up
    int *s_cnt = reinterpret_cast<int *>(s_t2h + TC_QMAX / 2);       // TC_QMAX
    uint2 *s_que = reinterpret_cast<uint2 *>(s_cnt + TC_QMAX);  // per epilogue warp: TC_QUE entries
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_que + TC_QUE * 4 * TC_EPI_GROUPS);
    uint64_t *full = bar, *empty = bar + S, *tfull = bar + 2 * S, *tempty = bar + 2 * S + TC_NACC;
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    __shared__ double s_c[64], s_B;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int c = 0; c < TC_NACC; c++) {
            mbar_init(tfull + c, 1);
            mbar_init(tempty + c, 4);  // the four warps of the group that reads it (group c)
        }
        mbar_init_fence();
        s_err = 0;
        centre_and_bound(a.kmax, a.kmin, a.p, s_c, s_B);
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(&s_tmem, TC_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = s_tmem;
    volatile int *err = &s_err;
    const uint32_t stage_bytes = (uint32_t)stage_halves * 2u;
    const uint32_t sbo = 8u * (uint32_t)K * 2u;  // bytes between 8-row groups
    // the operands carry 2^-e, the accumulators 2^-2e
    const float s2 = ldexpf(1.f, -2 * tc_scale_exp(s_B));

    long long it0 = 0;  // design blocks processed by this CTA so far (ring positions)
    for (int blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x) {
        const int64_t q0 = (int64_t)blk * a.nq;
        const int nqb = (int)min((int64_t)a.nq, a.M - q0);
        const int nmma = (nqb + 15) & ~15;  // MMA N: a multiple of 16
        // query operand and thresholds of this block
        for (int e = tid; e < nmma * K; e += TC_THREADS) {
            const int r = e / K, k = e - r * K;
            sQ[tc_off(r, k, K)] = r < nqb ? a.Q[(q0 + r) * K + k] : __float2half_rn(0.f);
        }
        for (int c = tid; c < TC_QMAX; c += TC_THREADS) {
            float t2 = CUDART_NAN_F;  // NaN: no row ever compares below
            if (c < nqb) {
                const int64_t q = q0 + c;
                const int k = a.Np ? a.Np[q] : a.Npmax;
                const float tq = a.tau0[q];
                if (k >= 1 && k <= a.Npmax && tq == tq) {
                    // the sampled threshold widened by 2 E_tc (rows at the
                    // sample's boundary fall inside whatever the rounding of
                    // either pass), then by the collection margin
                    const float t0 = __double2float_ru((double)tq + 2.0 * tc_error_bound(a.p, K, s_B));
                    t2 = __double2float_rd(tc_margin(t0, a.p, K, s_B));
                }
            }
            s_tau2[c] = t2 * s2;  // an exact scaling
            s_cnt[c] = 0;
        }
        __syncthreads();
        // the thresholds in FP16, rounded up (so that a value below a threshold
        // stays below it after both roundings), two a word
        for (int c2 = tid; c2 < TC_QMAX / 2; c2 += TC_THREADS) {
            const float ta = s_tau2[2 * c2], tb = s_tau2[2 * c2 + 1];
            const __half ha = __float2half_ru(ta), hb = __float2half_ru(tb);
            s_t2h[c2] = (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {  // producer: design blocks into the stage ring
                int issued = 0;
                for (int mb = 0; mb < a.nmb && !*err; mb++) {
                    if (a.stall && mb == 1) break;  // the MMA's wait on this block then runs out
                    const long long it = it0 + mb;
                    const int s = (int)(it % S);
                    const uint32_t round = (uint32_t)(it / S);
                    if (!mbar_wait(empty + s, (round & 1u) ^ 1u, err, 128)) break;
                    mbar_arrive_expect_tx(full + s, stage_bytes);
                    bulk_g2s(sA + (size_t)s * stage_halves, a.A + (size_t)mb * stage_halves, stage_bytes, full + s);
                    issued = mb + 1;
                }
                if (*err && issued > 0) {  // let the copies in flight land before the CTA moves on
                    for (int mb = max(0, issued - S); mb < issued; mb++) {
                        const long long it = it0 + mb;
                        int quiet = 0;
                        mbar_wait(full + (int)(it % S), (uint32_t)(it / S) & 1u, &quiet);
                    }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {  // MMA issuer
                const uint32_t idesc = idesc_f16_f32(TC_MROWS, nmma);
                const uint32_t qaddr = smem_u32(sQ);
                long long last = -1;
                for (int mb = 0; mb < a.nmb && !*err; mb++) {
                    const long long it = it0 + mb;
                    const int s = (int)(it % S);
                    const int ac = (int)(it % TC_NACC);
                    if (!mbar_wait(full + s, (uint32_t)(it / S) & 1u, err, 32)) break;
                    if (!mbar_wait(tempty + ac, ((uint32_t)(it / TC_NACC) & 1u) ^ 1u, err, 32)) break;
                    tc_fence_after_sync();
                    const uint32_t aaddr = smem_u32(sA + (size_t)s * stage_halves);
                    for (int ks = 0; ks < K / 16; ks++)  // 16 halves (two core matrices) per MMA
                        mma_f16(tmem + (uint32_t)(ac * TC_ACC_COLS), smem_desc_kmajor(aaddr + ks * 256u, 128u, sbo),
                                smem_desc_kmajor(qaddr + ks * 256u, 128u, sbo), idesc, ks > 0 ? 1u : 0u);
                    mma_commit(empty + s);    // the stage may be overwritten once these MMAs are done
                    mma_commit(tfull + ac);   // the accumulator is ready
                    last = it;
                }
                if (*err && last >= 0) {  // the MMAs issued finish before the TMEM is released
                    int quiet = 0;
                    mbar_wait(tfull + (int)(last % TC_NACC), (uint32_t)(last / TC_NACC) & 1u, &quiet);
                }
            }
        } else {
            // epilogue: group g reads accumulator g, of the design blocks with
            // it = g (mod 4); each warp its TMEM lane quarter (32 design rows)
            const int g = (warp - 2) >> 2, quarter = warp & 3;
            uint2 *que = s_que + (size_t)(warp - 2) * TC_QUE;
            const uint32_t lt_mask = (1u << lane) - 1u;
            for (int mb = 0; mb < a.nmb; mb++) {
                const long long it = it0 + mb;
                if ((int)(it % TC_NACC) != g) continue;
                // every lane waits; the warp goes on only together (the TMEM
                // loads are warp-collective)
                const bool ready = mbar_wait(tfull + g, (uint32_t)(it / TC_NACC) & 1u, err, 64);
                if (!__all_sync(LAGP_FULL_MASK, ready)) break;
                tc_fence_after_sync();
                const int64_t row = (int64_t)mb * TC_MROWS + quarter * 32 + lane;
                const bool live = row < a.N;
                int qn = 0;  // hit-queue entries of this design block
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * TC_ACC_COLS);
                for (int cb = 0; cb < nmma; cb += 64) {
                    // up to four chunks of 16 columns in flight, one wait
                    uint32_t v[4][16];
#pragma unroll
                    for (int h = 0; h < 4; h++)
                        if (cb + 16 * h < nmma) tmem_ld16(taddr + (uint32_t)(cb + 16 * h), v[h]);
#pragma unroll
                    for (int h = 0; h < 4; h++)
                        if (cb + 16 * h < nmma) tmem_wait_ld16(v[h]);
                    if (cb + 64 >= nmma) {  // every column read: release the accumulator
                        tc_fence_before_sync();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tempty + g);
                    }
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        const int c0 = cb + 16 * h;
                        if (c0 >= nmma) break;
                        if (a.dump) {
                            if (live)
#pragma unroll
                                for (int i = 0; i < 16; i++)
                                    if (c0 + i < nqb)
                                        a.dump[(q0 + c0 + i) * a.N + row] = __uint_as_float(v[h][i]) / s2;
                            continue;
                        }
                        // hit mask, compared two columns a time in FP16 (values
                        // rounded down, thresholds up: no hit is lost; the
                        // rounding admits at most a few extra rows): column
                        // c0 + 2i sets bit i, column c0 + 2i + 1 bit 16 + i
                        const uint4 *t4 = reinterpret_cast<const uint4 *>(s_t2h + c0 / 2);
                        uint32_t m2 = 0;
#pragma unroll
                        for (int i4 = 0; i4 < 2; i4++) {
                            const uint4 t = t4[i4];
                            const uint32_t tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                            for (int q2 = 0; q2 < 4; q2++) {
                                const int i = 4 * i4 + q2;  // the pair of columns c0 + 2i, c0 + 2i + 1
                                const uint32_t hv = f16x2_rz_relu(__uint_as_float(v[h][2 * i]), __uint_as_float(v[h][2 * i + 1]));
                                m2 |= le_mask_h2(hv, tt[q2]) & (0x00010001u << i);
                            }
                        }
                        if (!live) m2 = 0u;
                        // a lane with hits queues (chunk and lane, mask); the
                        // queue is drained lane-parallel after the block
                        const uint32_t b = __ballot_sync(LAGP_FULL_MASK, m2 != 0u);
                        if (m2) que[qn + __popc(b & lt_mask)] = make_uint2(((uint32_t)(c0 >> 4) << 5) | (uint32_t)lane, m2);
                        qn += __popc(b);
                    }
                }
                __syncwarp();
                for (int e = lane; e < qn; e += 32) {
                    const uint2 w = que[e];
                    const int cb0 = (int)(w.x >> 5) * 16;
                    const int32_t hrow = (int32_t)(mb * TC_MROWS + quarter * 32 + (w.x & 31u));
                    uint32_t mm = w.y;  // bit i: column cb0 + 2i; bit 16 + i: column cb0 + 2i + 1
                    while (mm) {
                        const int bit = __ffs(mm) - 1;
                        const int c = cb0 + (bit < 16 ? 2 * bit : 2 * (bit - 16) + 1);
                        mm &= mm - 1u;
                        const int pos = atomicAdd(&s_cnt[c], 1);
                        if (pos < a.Cmax) a.cand[(q0 + c) * a.Cmax + pos] = hrow;
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // per-query results: the collected rows and the threshold they were
        // collected under (the sort checks that the N'-th of them lies within
        // the radius that threshold guarantees); an overflowing or
        // unscreened query goes to the exact retry
        const bool failed = *err != 0;
        for (int c = tid; c < nqb; c += TC_THREADS) {
            const int64_t q = q0 + c;
            const int k = a.Np ? a.Np[q] : a.Npmax;
            const bool kvalid = k >= 1 && k <= a.Npmax;
            const bool ok = kvalid && s_tau2[c] == s_tau2[c];
            const bool done = !failed && ok && s_cnt[c] >= k && s_cnt[c] <= a.Cmax;
            a.retry[q] = (kvalid && !done) ? 1 : 0;
            a.cand_count[q] = done ? s_cnt[c] : 0;
            a.rcol[q] = done ? __double2float_rd(tc_collected_radius(s_tau2[c] / s2, a.p, K, s_B)) : CUDART_NAN_F;
            if (a.status) a.status[q] = kvalid ? LAGP_OK : LAGP_EINVAL;
        }
        it0 += a.nmb;
        __syncthreads();
        if (failed) {
            // this and the CTA's remaining blocks go to the exact retry
            for (int b2 = blk + gridDim.x; b2 < a.nblocks; b2 += gridDim.x)
                for (int c = tid; c < a.nq && (int64_t)b2 * a.nq + c < a.M; c += TC_THREADS) {
                    const int64_t q = (int64_t)b2 * a.nq + c;
                    const int k = a.Np ? a.Np[q] : a.Npmax;
                    const bool kvalid = k >= 1 && k <= a.Npmax;
                    a.retry[q] = kvalid ? 1 : 0;
                    a.cand_count[q] = 0;
                    a.rcol[q] = CUDART_NAN_F;
                    if (a.status) a.status[q] = kvalid ? LAGP_OK : LAGP_EINVAL;
                }
            break;
        }
    }
    if (tid == 0 && *err) atomicExch(a.err, 1);
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after_sync();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

}  // namespace

bool knn_tc_supported(int p) { return p >= 1 && tc_k(p) <= 64; }

size_t knn_tc_workspace(int64_t N, int64_t M, int p) {
    const int K = tc_k(p);
    const int64_t Npad = round_up(std::max<int64_t>(N, 1), TC_MROWS);
    return (size_t)(Npad + M) * K * 2 + (size_t)M * 8 + 256;
}

// Design and query operands, the sampled thresholds (tau0, filled by the
// CUDA-core screen's passes A and B between the two launches), and the
// collection pass.  ws: knn_tc_workspace(N, M, p) bytes.
lagp_status launch_knn_tc_prep(lagp_ctx *ctx, void *ws, const void *X, int64_t N, int p, lagp_dtype dtype,
                               const void *Xref, int64_t M, const unsigned long long *kmax,
                               const unsigned long long *kmin, float **tau0, float **rcol) {
    const int K = tc_k(p);
    const int64_t Npad = round_up(std::max<int64_t>(N, 1), TC_MROWS);
    __half *A = static_cast<__half *>(ws);
    __half *Q = A + Npad * K;
    *tau0 = reinterpret_cast<float *>(Q + M * K);
    *rcol = *tau0 + M;
    knn_tc_prep<<<ctx->num_sms * 4, 128, 0, ctx->stream>>>(X, N, Npad, Xref, M, p, dtype, kmax, kmin, A, Q);
    ctx->launches++;
    return lagp_cuda_check(ctx, cudaGetLastError(), "knn_tc_prep");
}

lagp_status launch_knn_tc_collect(lagp_ctx *ctx, void *ws, int64_t N, int p, int64_t M, const int32_t *Np,
                                  int32_t Npmax, const unsigned long long *kmax, const unsigned long long *kmin,
                                  int32_t *cand, int32_t Cmax, int32_t *cand_count, int32_t *status,
                                  int32_t *retry, int *err, float *rcol, float *dump) {
    const int K = tc_k(p);
    const int64_t Npad = round_up(std::max<int64_t>(N, 1), TC_MROWS);
    TcArgs a;
    a.A = static_cast<const __half *>(ws);
    a.Q = a.A + Npad * K;
    a.N = N;
    a.M = M;
    a.p = p;
    a.K = K;
    a.nmb = (int)(Npad / TC_MROWS);
    a.tau0 = reinterpret_cast<const float *>(a.Q + M * K);
    a.rcol = rcol;
    a.Np = Np;
    a.Npmax = Npmax;
    a.kmax = kmax;
    a.kmin = kmin;
    a.cand = cand;
    a.Cmax = Cmax;
    a.cand_count = cand_count;
    a.status = status;
    a.retry = retry;
    a.err = err;
    a.dump = dump;
    a.stall = ctx->knn_tc_stall;
    ctx->knn_tc_stall = 0;
    // blocks: a multiple of the SM count (balanced waves), at most TC_QMAX queries each
    const int64_t sms = ctx->num_sms;
    const int64_t nb_min = (M + TC_QMAX - 1) / TC_QMAX;
    const int64_t nb = std::min<int64_t>(M, round_up(nb_min, sms));
    a.nq = (int)((M + nb - 1) / nb);
    a.nblocks = (int)((M + a.nq - 1) / a.nq);
    // as many stages as fit (at most TC_STAGES_MAX): the CTA then has the SM
    // (and its tensor memory) to itself
    const size_t fixed = (size_t)TC_QMAX * K * 2 + (2 * TC_QMAX + TC_QMAX / 2 + 2 * TC_QUE * 4 * TC_EPI_GROUPS) * 4 +
                         (2 * TC_STAGES_MAX + 2 * TC_NACC) * 8 + 1024;
    const size_t stage_bytes = (size_t)TC_MROWS * K * 2;
    a.stages = (int)std::min<size_t>(TC_STAGES_MAX, (ctx->smem_optin - fixed) / stage_bytes);
    if (a.stages < 2) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: tensor-core screen exceeds shared memory");
    size_t smem = (size_t)a.stages * stage_bytes + (size_t)TC_QMAX * K * 2 +
                  (2 * TC_QMAX + TC_QMAX / 2 + 2 * TC_QUE * 4 * TC_EPI_GROUPS) * 4 +
                  (2 * (size_t)a.stages + 2 * TC_NACC) * 8;
    // more than half of the SM's shared memory: one CTA per SM, which then
    // holds the whole tensor memory
    smem = std::max(smem, ctx->smem_optin / 2 + 4096);
    LAGP_CUDA(ctx, cudaFuncSetAttribute(knn_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>(a.nblocks, sms);
    knn_screen_tc<<<grid, TC_THREADS, smem, ctx->stream>>>(a);
    ctx->launches++;
    return lagp_cuda_check(ctx, cudaGetLastError(), "knn_screen_tc");
}
