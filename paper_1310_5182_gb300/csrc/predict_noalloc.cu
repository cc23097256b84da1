// lagp_predict_noalloc: the local predictive equations (Eqs. predgp, preds2)
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose own allocator owns
// every byte of device memory after start-up, services that run under a
// device-memory budget fixed when they start, and latency-critical paths for
// which cudaMalloc's implicit device synchronisation is not acceptable.
// lagp_predict draws its per-CTA matrices from the context's workspace, which
// may grow with cudaMalloc; this entry point instead keeps that scratch in a
// file-scope device array of fixed size, so it never allocates.
//
// Scratch: NA_CTAS CTAs, each owning one NA_NMAX x NA_NMAX FP64 matrix (the
// local covariance, factorised in place), after a 256-byte block holding the
// work counter: 64 * 64 * 64 * 8 bytes + 256 bytes = 2 MiB + 256 bytes, held
// by every GPU that loads the library until the process exits.  Every call
// shares this array and finds the previous call's contents in it; the
// counter is cleared at the start of each call and everything else is
// written before it is read.  Calls that overlap on the GPU (on different
// streams, or from different contexts on the same device) race on it, so the
// caller must order them.  The first call on a device looks up the array's
// device address with that device current; make that first call before any
// stream capture begins.
#include <cuda_runtime.h>

#include <mutex>

#include "device_util.cuh"
#include "lagp_internal.h"

namespace {

constexpr int NA_NMAX = 64;   // largest n_max the static scratch holds
constexpr int NA_CTAS = 64;   // persistent CTAs, one matrix each
constexpr int NA_THREADS = 256;
constexpr int NA_WARPS = NA_THREADS / 32;
constexpr size_t NA_COUNTER_DOUBLES = 32;  // 256 bytes
constexpr size_t NA_MAT = (size_t)NA_NMAX * NA_NMAX;

// The static scratch.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double lagp_noalloc_scratch[NA_COUNTER_DOUBLES + NA_CTAS * NA_MAT];

__device__ double na_block_sum(double v, double *red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NA_WARPS; w++) s += red[w];
    return s;
}

__global__ void __launch_bounds__(NA_THREADS)
predict_noalloc_kernel(GpArgs a, const double *__restrict__ dv, double *scratch, double *mean,
                       double *s2, double *df, int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.nmax, p = a.p, ld = NA_NMAX;
    double *xd = reinterpret_cast<double *>(smem_raw);  // nmax x p
    double *y = xd + (size_t)nmax * p;                   // nmax
    double *kx = y + nmax;                               // nmax
    double *z = kx + nmax;                               // nmax: L^{-1} y
    double *w = z + nmax;                                // nmax: L^{-1} kx
    double *xq = w + nmax;                               // p
    __shared__ int s_loc, s_flag;
    __shared__ double red[NA_WARPS];
    int *counter = reinterpret_cast<int *>(scratch);
    double *A = scratch + NA_COUNTER_DOUBLES + (size_t)blockIdx.x * NA_MAT;  // this CTA's matrix
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) s_loc = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t loc = s_loc;
        __syncthreads();
        if (loc >= a.M) break;
        const int nm = a.n ? a.n[loc] : nmax;
        const double d = dv[loc], g = a.g;
        const int32_t *s = a.sel + loc * nmax;
        if (tid == 0) s_flag = (nm < 1 || nm > nmax || !(d > 0.0) || !isfinite(d)) ? LAGP_EINVAL : LAGP_OK;
        __syncthreads();
        if (s_flag == LAGP_OK)
            for (int t = tid; t < nm; t += NA_THREADS)
                if (s[t] < 0 || s[t] >= a.N) s_flag = LAGP_EINVAL;
        __syncthreads();
        int st = s_flag;
        double mu = CUDART_NAN, sv = CUDART_NAN, dfv = CUDART_NAN;
        if (st == LAGP_OK) {
            for (int e = tid; e < nm * p; e += NA_THREADS) {
                int t = e / p, i = e - t * p;
                xd[e] = load_coord64(a.X, s[t], p, i, a.dtype);
            }
            for (int i = tid; i < p; i += NA_THREADS) xq[i] = load_coord64(a.Xref, loc, p, i, a.dtype);
            for (int t = tid; t < nm; t += NA_THREADS)
                y[t] = a.dtype == LAGP_F64 ? static_cast<const double *>(a.Y)[s[t]]
                                           : (double)static_cast<const float *>(a.Y)[s[t]];
            __syncthreads();
            // K_n (lower triangle): exp(-||x_i - x_k||^2 / d) + g on the diagonal
            for (int e = tid; e < nm * nm; e += NA_THREADS) {
                int i = e / nm, k = e - i * nm;
                if (k <= i) {
                    double q = 0.0;
                    for (int c = 0; c < p; c++) {
                        double df2 = xd[(size_t)i * p + c] - xd[(size_t)k * p + c];
                        q = fma(df2, df2, q);
                    }
                    A[(size_t)i * ld + k] = exp(-q / d) + (i == k ? g : 0.0);
                }
            }
            for (int t = tid; t < nm; t += NA_THREADS) {
                double q = 0.0;
                for (int c = 0; c < p; c++) {
                    double df2 = xq[c] - xd[(size_t)t * p + c];
                    q = fma(df2, df2, q);
                }
                kx[t] = exp(-q / d);
            }
            if (tid == 0) s_flag = 1;
            __syncthreads();
            // in-place left-looking Cholesky, K_n = L L^T
            for (int c = 0; c < nm; c++) {
                if (warp == 0) {
                    double q = 0.0;
                    for (int k = lane; k < c; k += 32) q = fma(A[(size_t)c * ld + k], A[(size_t)c * ld + k], q);
                    q = warp_sum(q);
                    if (lane == 0) {
                        double piv = A[(size_t)c * ld + c] - q;
                        if (!(piv > 0.0)) s_flag = 0;
                        A[(size_t)c * ld + c] = piv > 0.0 ? sqrt(piv) : 1.0;
                    }
                }
                __syncthreads();
                const double lcc = A[(size_t)c * ld + c];
                for (int i = c + 1 + tid; i < nm; i += NA_THREADS) {
                    double q = A[(size_t)i * ld + c];
                    for (int k = 0; k < c; k++) q = fma(-A[(size_t)i * ld + k], A[(size_t)c * ld + k], q);
                    A[(size_t)i * ld + c] = q / lcc;
                }
                __syncthreads();
            }
            if (!s_flag) {
                st = LAGP_ENOTPD;
            } else {
                // z = L^{-1} y (warp 0) and w = L^{-1} kx (warp 1)
                if (warp < 2) {
                    const double *rhs = warp == 0 ? y : kx;
                    double *x = warp == 0 ? z : w;
                    for (int i = 0; i < nm; i++) {
                        double q = 0.0;
                        for (int k = lane; k < i; k += 32) q = fma(A[(size_t)i * ld + k], x[k], q);
                        q = warp_sum(q);
                        if (lane == 0) x[i] = (rhs[i] - q) / A[(size_t)i * ld + i];
                        __syncwarp();
                    }
                }
                __syncthreads();
                double m_p = 0.0, psi_p = 0.0, kk_p = 0.0;
                for (int i = tid; i < nm; i += NA_THREADS) {
                    m_p = fma(w[i], z[i], m_p);
                    psi_p = fma(z[i], z[i], psi_p);
                    kk_p = fma(w[i], w[i], kk_p);
                }
                mu = na_block_sum(m_p, red);
                const double psi = na_block_sum(psi_p, red);
                const double kk = na_block_sum(kk_p, red);
                sv = psi * ((1.0 + g) - kk) / nm;
                dfv = nm;
            }
        }
        if (tid == 0) {
            mean[loc] = mu;
            s2[loc] = sv;
            df[loc] = dfv;
            status[loc] = st;
        }
        __syncthreads();
    }
}

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
double *na_scratch[NA_MAX_DEVICES] = {};

// Device address of the static scratch for the current device, looked up
// once per device (with that device current).
lagp_status na_scratch_for(lagp_ctx *ctx, double **out) {
    if (ctx->device < 0 || ctx->device >= NA_MAX_DEVICES)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_scratch[ctx->device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, lagp_noalloc_scratch);
        if (e != cudaSuccess) return lagp_cuda_check(ctx, e, "cudaGetSymbolAddress(lagp_noalloc_scratch)");
        na_scratch[ctx->device] = static_cast<double *>(ptr);
    }
    *out = na_scratch[ctx->device];
    return LAGP_OK;
}

}  // namespace

extern "C" lagp_status lagp_predict_noalloc(lagp_ctx *ctx, const void *X, const void *Y, int64_t N,
                                            int32_t p, lagp_dtype dtype, const void *Xref, int64_t M,
                                            const int32_t *sel, const int32_t *n, int32_t n_max,
                                            const double *d, double g, double *mean, double *s2,
                                            double *df, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    if (!X || !Y || (M > 0 && (!Xref || !sel || !d || !mean || !s2 || !df || !status)))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict_noalloc: NULL required array");
    if (N < 1 || N >= (int64_t)INT32_MAX || p < 1 || p > 64 || (dtype != LAGP_F64 && dtype != LAGP_F32))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict_noalloc: need 1 <= N < 2^31, 1 <= p <= 64, dtype F64/F32");
    // (its work counter is a 32-bit atomic that runs up to M + NA_CTAS)
    if (M < 0 || M >= ((int64_t)1 << 30))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict_noalloc: need 0 <= M < 2^30");
    if (n_max < 1 || n_max > NA_NMAX)
        return lagp_fail(ctx, LAGP_EINVAL,
                         "lagp_predict_noalloc: n_max must be in [1, 64], the size of the static scratch");
    if (!(g >= 0.0) || !isfinite(g))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict_noalloc: g must be finite and >= 0");
    if (M == 0) return LAGP_OK;
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    double *scratch = nullptr;
    LAGP_TRY(na_scratch_for(ctx, &scratch));
    // the work counter must start at zero; everything else is written before it is read
    LAGP_CUDA(ctx, cudaMemsetAsync(scratch, 0, NA_COUNTER_DOUBLES * sizeof(double), ctx->stream));
    const size_t smem = ((size_t)n_max * p + 4 * (size_t)n_max + (size_t)p) * sizeof(double) + 16;
    LAGP_CUDA(ctx, cudaFuncSetAttribute(predict_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    GpArgs a{X, Y, N, p, dtype, Xref, M, sel, n, n_max, g};
    const int grid = (int)(M < NA_CTAS ? M : NA_CTAS);
    predict_noalloc_kernel<<<grid, NA_THREADS, smem, ctx->stream>>>(a, d, scratch, mean, s2, df, status);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
