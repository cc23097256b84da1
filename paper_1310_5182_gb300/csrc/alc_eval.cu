// The ALC criterion of Eq. (dxy) for many candidates at one location and a
// fixed design — the computation the paper times in Sec. 4.1 (one reference
// location, N' = 60,000 candidates, designs of n = 16..512).
//
// Given the design X_n and the location x:
//   prep   K_n = exp(-D/d) + g I, its Cholesky factor L (FP64), z = L^{-1} k_n(x),
//          1/diag(L); padded to a multiple of 32 rows with identity rows.
//   cands  per candidate c: u_c = L^{-1} k_n(x_c) by blocked forward
//          substitution, s_c = |u_c|^2 = k_c^T K_n^{-1} k_c,
//          q_c = z^T u_c = k_n(x)^T K_n^{-1} k_c, and
//          Delta_c = (K(x_c, x) - q_c)^2 / (1 + g - s_c)
//          (Eq. (dxy) with Eq. (piedef) after simplification).
// The candidate kernel is one thread per candidate, 32-row blocks: the
// off-diagonal blocks L_IJ are staged in shared memory (read as broadcasts),
// the current block's 32 values live in registers, earlier solved blocks
// stream from a global panel W[i][c] (coalesced across the candidates).  Per
// candidate n^2/2 FP64 FMAs with every lane busy: the FP64 unit bounds it.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "exp64.cuh"
#include "lagp_internal.h"

namespace {

constexpr int EV_THREADS = 128;  // candidates per CTA
constexpr int EV_B = 32;         // rows per block of the substitution
constexpr int PREP_THREADS = 256;

// One CTA: L (np x np, np = n rounded up to 32, identity padding), rd, z.
__global__ void __launch_bounds__(PREP_THREADS)
eval_prep_kernel(const void *X, int p, lagp_dtype dt, const double *x, const int32_t *design, int n,
                 int np, double d, double g, double *L, double *rd, double *z, int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *xd = reinterpret_cast<double *>(smem_raw);  // n x p design coordinates
    double *kx = xd + (size_t)n * p;                    // np
    __shared__ int s_ok;
    __shared__ double etab[EXP64_TABLE_SIZE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < EXP64_TABLE_SIZE; i += PREP_THREADS) etab[i] = exp64_table_g[i];
    if (tid == 0) s_ok = 1;
    for (int e = tid; e < n * p; e += PREP_THREADS) xd[e] = load_coord64(X, design[e / p], p, e % p, dt);
    __syncthreads();
    const double ninv_d = -1.0 / d;
    for (int e = tid; e < np * np; e += PREP_THREADS) {
        const int i = e / np, k = e - i * np;
        double v;
        if (i < n && k < n) {
            double s = 0.0;
            for (int t = 0; t < p; t++) {
                const double df = xd[(size_t)i * p + t] - xd[(size_t)k * p + t];
                s = fma(df, df, s);
            }
            v = exp64_tang(s * ninv_d, etab) + (i == k ? g : 0.0);
        } else {
            v = i == k ? 1.0 : 0.0;  // identity padding
        }
        L[(size_t)i * np + k] = v;
    }
    for (int i = tid; i < np; i += PREP_THREADS) {
        double s = 0.0;
        if (i < n)
            for (int t = 0; t < p; t++) {
                const double df = xd[(size_t)i * p + t] - x[t];
                s = fma(df, df, s);
            }
        kx[i] = i < n ? exp64_tang(s * ninv_d, etab) : 0.0;
    }
    __syncthreads();
    // in-place left-looking Cholesky of the lower triangle
    for (int c = 0; c < np; c++) {
        if (warp == 0) {
            double s = 0.0;
            for (int k = lane; k < c; k += 32) s = fma(L[(size_t)c * np + k], L[(size_t)c * np + k], s);
            s = warp_sum(s);
            if (lane == 0) {
                const double piv = L[(size_t)c * np + c] - s;
                if (!(piv > 0.0)) s_ok = 0;
                const double lcc = piv > 0.0 ? sqrt(piv) : 1.0;
                L[(size_t)c * np + c] = lcc;
                rd[c] = 1.0 / lcc;
            }
        }
        __syncthreads();
        const double rcc = rd[c];
        for (int i = c + 1 + tid; i < np; i += PREP_THREADS) {
            double s0 = L[(size_t)i * np + c], s1 = 0.0;
            int k = 0;
            for (; k + 2 <= c; k += 2) {
                s0 = fma(-L[(size_t)i * np + k], L[(size_t)c * np + k], s0);
                s1 = fma(-L[(size_t)i * np + k + 1], L[(size_t)c * np + k + 1], s1);
            }
            if (k < c) s0 = fma(-L[(size_t)i * np + k], L[(size_t)c * np + k], s0);
            L[(size_t)i * np + c] = (s0 + s1) * rcc;
        }
        __syncthreads();
    }
    // z = L^{-1} k_n(x)
    if (warp == 0) {
        for (int i = 0; i < np; i++) {
            double s = 0.0;
            for (int k = lane; k < i; k += 32) s = fma(L[(size_t)i * np + k], z[k], s);
            s = warp_sum(s);
            if (lane == 0) z[i] = (kx[i] - s) * rd[i];
            __syncwarp();
        }
    }
    if (tid == 0) *status = s_ok ? LAGP_OK : LAGP_ENOTPD;
}

__global__ void __launch_bounds__(EV_THREADS)
eval_cands_kernel(const void *X, int p, lagp_dtype dt, const double *x, const int32_t *design, int n,
                  int np, const int32_t *cands, int64_t Nc, double d, double g, const double *L,
                  const double *rd, const double *z, double *W, double *delta, const int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *blk = reinterpret_cast<double *>(smem_raw);  // EV_B x EV_B block of L
    double *xd = blk + EV_B * EV_B;                       // n x p design coordinates
    double *xc = xd + (size_t)n * p;                      // EV_THREADS x p candidate coordinates
    __shared__ double etab[EXP64_TABLE_SIZE];
    const int tid = threadIdx.x;
    const int64_t c = (int64_t)blockIdx.x * EV_THREADS + tid;
    const bool live = c < Nc;
    for (int i = tid; i < EXP64_TABLE_SIZE; i += EV_THREADS) etab[i] = exp64_table_g[i];
    for (int e = tid; e < n * p; e += EV_THREADS) xd[e] = load_coord64(X, design[e / p], p, e % p, dt);
    const int32_t crow = live ? cands[c] : 0;
    for (int i = 0; i < p; i++) xc[(size_t)tid * p + i] = load_coord64(X, crow, p, i, dt);
    __syncthreads();
    if (*status != LAGP_OK) {  // the design's K_n was not positive definite
        if (live) delta[c] = CUDART_NAN;
        return;
    }
    const double ninv_d = -1.0 / d;
    const double *mx = xc + (size_t)tid * p;
    double s = 0.0, q = 0.0;
    const int nb = np / EV_B;
    for (int I = 0; I < nb; I++) {
        double acc[EV_B];
#pragma unroll
        for (int r = 0; r < EV_B; r++) {  // k_n(x_c) for rows of block I
            const int row = I * EV_B + r;
            double sd = 0.0;
            if (row < n)
                for (int t = 0; t < p; t++) {
                    const double df = mx[t] - xd[(size_t)row * p + t];
                    sd = fma(df, df, sd);
                }
            acc[r] = row < n ? exp64_tang(sd * ninv_d, etab) : 0.0;
        }
        for (int J = 0; J < I; J++) {  // acc -= L_IJ w_J
            __syncthreads();
            for (int e = tid; e < EV_B * EV_B; e += EV_THREADS)
                blk[e] = L[(size_t)(I * EV_B + e / EV_B) * np + J * EV_B + (e % EV_B)];
            __syncthreads();
            const double *Wj = W + (size_t)J * EV_B * Nc + c;
#pragma unroll 4
            for (int k = 0; k < EV_B; k++) {
                const double w = live ? Wj[(size_t)k * Nc] : 0.0;
#pragma unroll
                for (int r = 0; r < EV_B; r++) acc[r] = fma(-blk[r * EV_B + k], w, acc[r]);
            }
        }
        __syncthreads();
        for (int e = tid; e < EV_B * EV_B; e += EV_THREADS)
            blk[e] = L[(size_t)(I * EV_B + e / EV_B) * np + I * EV_B + (e % EV_B)];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < EV_B; r++) {  // the diagonal block, in place
            double t = acc[r];
#pragma unroll
            for (int k = 0; k < r; k++) t = fma(-blk[r * EV_B + k], acc[k], t);
            acc[r] = t * rd[I * EV_B + r];
            s = fma(acc[r], acc[r], s);
            q = fma(z[I * EV_B + r], acc[r], q);
        }
        if (live && I + 1 < nb) {
            double *Wi = W + (size_t)I * EV_B * Nc + c;
#pragma unroll
            for (int r = 0; r < EV_B; r++) Wi[(size_t)r * Nc] = acc[r];
        }
    }
    if (live) {
        double sk = 0.0;
        for (int t = 0; t < p; t++) {
            const double df = mx[t] - x[t];
            sk = fma(df, df, sk);
        }
        const double kap = exp64_tang(sk * ninv_d, etab);  // K(x_c, x)
        const double minv = (1.0 + g) - s;                  // m^{-1}(x_c), Eq. (piedef)
        const double r = kap - q;
        delta[c] = minv > 0.0 ? r * r / minv : CUDART_NAN;
    }
}

}  // namespace

extern "C" lagp_status lagp_alc_eval(lagp_ctx *ctx, const void *X, int64_t N, int32_t p,
                                     lagp_dtype dtype, const double *x, const int32_t *design,
                                     int32_t n, const int32_t *cands, int64_t Nc, double d, double g,
                                     double *delta, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    if (!X || !x || !design || !status || (Nc > 0 && (!cands || !delta)))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_eval: NULL required array");
    if (N < 1 || N >= (int64_t)INT32_MAX || p < 1 || p > 64 || (dtype != LAGP_F64 && dtype != LAGP_F32))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_eval: need 1 <= N < 2^31, 1 <= p <= 64, dtype F64/F32");
    if (n < 1 || n > 1024 || Nc < 0 || !(d > 0.0) || !(g >= 0.0))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_eval: need 1 <= n <= 1024, Nc >= 0, d > 0, g >= 0");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int np = (n + EV_B - 1) / EV_B * EV_B;
    const size_t wbytes = (size_t)np * np * 8 + 2 * (size_t)np * 8 + (size_t)np * (Nc > 0 ? Nc : 1) * 8;
    double *Lm = static_cast<double *>(lagp_ws(ctx, WS_ALC_STATE, wbytes + 256));
    if (!Lm) return LAGP_ENOMEM;
    double *rd = Lm + (size_t)np * np, *z = rd + np, *W = z + np;
    const size_t smem_prep = ((size_t)n * p + np) * 8;
    if (smem_prep > ctx->smem_optin) return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_eval: n x p too large");
    cudaFuncSetAttribute(eval_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_prep);
    eval_prep_kernel<<<1, PREP_THREADS, smem_prep, ctx->stream>>>(X, p, dtype, x, design, n, np, d, g, Lm,
                                                                   rd, z, status);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    if (Nc == 0) return LAGP_OK;
    const size_t smem = ((size_t)EV_B * EV_B + (size_t)n * p + (size_t)EV_THREADS * p) * 8;
    if (smem > ctx->smem_optin) return lagp_fail(ctx, LAGP_EINVAL, "lagp_alc_eval: n x p too large");
    cudaFuncSetAttribute(eval_cands_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t grid = (Nc + EV_THREADS - 1) / EV_THREADS;
    eval_cands_kernel<<<(unsigned)grid, EV_THREADS, smem, ctx->stream>>>(X, p, dtype, x, design, n, np, cands,
                                                                         Nc, d, g, Lm, rd, z, W, delta,
                                                                         status);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
