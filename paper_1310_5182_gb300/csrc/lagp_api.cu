// C ABI entry points of liblagp.so: context management, argument checking,
// workspace, and the whole-method host-buffer call (lagp_agp).
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "lagp_internal.h"

// ------------------------------------------------------------- status/errors

lagp_status lagp_fail(lagp_ctx *ctx, lagp_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return s;
}

lagp_status lagp_cuda_check(lagp_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LAGP_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return lagp_fail(ctx, e == cudaErrorMemoryAllocation ? LAGP_ENOMEM : LAGP_ECUDA, m);
}

void *lagp_ws(lagp_ctx *ctx, WsSlot slot, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (ctx->ws_bytes[slot] >= bytes) return ctx->ws[slot];
    // grow geometrically to limit reallocations
    size_t want = bytes + bytes / 4;
    if (ctx->ws[slot]) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws[slot]);
        ctx->ws[slot] = nullptr;
        ctx->ws_bytes[slot] = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "workspace slot %d: cudaMalloc(%zu) failed: %s", (int)slot, want,
                 cudaGetErrorString(e));
        ctx->err = buf;
        return nullptr;
    }
    ctx->ws[slot] = p;
    ctx->ws_bytes[slot] = want;
    return p;
}

lagp_status alc_counters(lagp_ctx *ctx, int **counter, unsigned long long **work) {
    char *base = static_cast<char *>(lagp_ws(ctx, WS_ALC_COUNTER, 256));
    if (!base) return LAGP_ENOMEM;
    *counter = reinterpret_cast<int *>(base);
    *work = reinterpret_cast<unsigned long long *>(base + 128);
    if (!ctx->work_zeroed) {
        // the ALC words (offset 128) and the MLE words (offset 192)
        LAGP_CUDA(ctx, cudaMemsetAsync(*work, 0, 128, ctx->stream));
        ctx->work_zeroed = true;
    }
    return LAGP_OK;
}

extern "C" {

const char *lagp_status_string(lagp_status s) {
    switch (s) {
        case LAGP_OK: return "LAGP_OK";
        case LAGP_EINVAL: return "LAGP_EINVAL";
        case LAGP_ENOTPD: return "LAGP_ENOTPD";
        case LAGP_ECUDA: return "LAGP_ECUDA";
        case LAGP_ETIMEOUT: return "LAGP_ETIMEOUT";
        case LAGP_ENOMEM: return "LAGP_ENOMEM";
    }
    return "LAGP_UNKNOWN";
}

lagp_status lagp_create(lagp_ctx **out, int device, void *cuda_stream) {
    if (!out) return LAGP_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return LAGP_ECUDA;
    }
    if (device < 0 || device >= ndev) return LAGP_EINVAL;
    lagp_ctx *ctx = new (std::nothrow) lagp_ctx();
    if (!ctx) return LAGP_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaDeviceProp pr;
    if (cudaSetDevice(device) != cudaSuccess || cudaGetDeviceProperties(&pr, device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return LAGP_ECUDA;
    }
    ctx->num_sms = pr.multiProcessorCount;
    ctx->smem_optin = pr.sharedMemPerBlockOptin;
    *out = ctx;
    return LAGP_OK;
}

lagp_status lagp_destroy(lagp_ctx *ctx) {
    if (!ctx) return LAGP_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (int s = 0; s < WS_NSLOTS; s++)
        if (ctx->ws[s]) cudaFree(ctx->ws[s]);
    if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
    delete ctx;
    return LAGP_OK;
}

lagp_status lagp_set_stream(lagp_ctx *ctx, void *cuda_stream) {
    if (!ctx) return LAGP_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return LAGP_OK;
}

const char *lagp_last_error(const lagp_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

lagp_status lagp_get_tuning(const lagp_ctx *ctx, lagp_tuning *out) {
    if (!ctx || !out) return LAGP_EINVAL;
    *out = ctx->tuning;
    return LAGP_OK;
}

lagp_status lagp_set_tuning(lagp_ctx *ctx, const lagp_tuning *in) {
    if (!ctx || !in) return LAGP_EINVAL;
    if (in->ctas_per_sm < 0 || in->ctas_per_sm > 32 || in->block_threads < 0 ||
        in->block_threads > 1024 || (in->block_threads % 32) != 0 || in->rescore_max < 0 ||
        in->rescore_max > 32 || !(in->rescore_rel >= 0.0) || !(in->rescore_rel < 1.0) ||
        in->knn_path < 0 || in->knn_path > 1)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_set_tuning: field out of range");
    ctx->tuning = *in;
    return LAGP_OK;
}

int64_t lagp_launch_count(const lagp_ctx *ctx) { return ctx ? ctx->launches : 0; }

lagp_status lagp_alc_work(lagp_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return LAGP_EINVAL;
    ctx->err.clear();
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    int *counter = nullptr;
    unsigned long long *work = nullptr;
    LAGP_TRY(alc_counters(ctx, &counter, &work));
    unsigned long long h[4] = {0, 0, 0, 0};
    LAGP_CUDA(ctx, cudaMemcpyAsync(h, work, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    LAGP_CUDA(ctx, cudaMemsetAsync(work, 0, sizeof h, ctx->stream));
    LAGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 4; i++) out[i] = h[i];
    return LAGP_OK;
}

lagp_status lagp_mle_work(lagp_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return LAGP_EINVAL;
    ctx->err.clear();
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    int *counter = nullptr;
    unsigned long long *work = nullptr;
    LAGP_TRY(alc_counters(ctx, &counter, &work));
    unsigned long long h[2] = {0, 0};
    LAGP_CUDA(ctx, cudaMemcpyAsync(h, work + 8, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    LAGP_CUDA(ctx, cudaMemsetAsync(work + 8, 0, sizeof h, ctx->stream));
    LAGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 2; i++) out[i] = h[i];
    return LAGP_OK;
}

// --------------------------------------------------------------------- kNN

// d0 everywhere, on the device (no host staging, no synchronisation)
__global__ void fill_f64_kernel(double *p, int64_t n, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// The persistent kernels hand out locations through a 32-bit atomic counter
// that runs up to M plus the grid size: M stays below 2^30.
constexpr int64_t LAGP_M_LIMIT = (int64_t)1 << 30;

static lagp_status check_design(lagp_ctx *ctx, const void *X, int64_t N, int32_t p,
                                lagp_dtype dtype, const char *fn) {
    if (!X) return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": X is NULL");
    if (N < 1 || N >= (int64_t)INT32_MAX)
        return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": N must be in [1, 2^31-1)");
    if (p < 1 || p > 64) return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": p must be in [1, 64]");
    if (dtype != LAGP_F64 && dtype != LAGP_F32)
        return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": unknown dtype");
    return LAGP_OK;
}

lagp_status lagp_knn(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                     const void *Xref, int64_t M, const int32_t *Nprime, int32_t Nprime_max,
                     int32_t *idx, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    LAGP_TRY(check_design(ctx, X, N, p, dtype, "lagp_knn"));
    if (M < 0 || M >= LAGP_M_LIMIT) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: need 0 <= M < 2^30");
    if (M == 0) return LAGP_OK;
    if (!Xref || !idx) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: NULL Xref or idx");
    if (Nprime_max < 1 || Nprime_max > N)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: need 1 <= Nprime_max <= N");
    if (Nprime_max > 4096)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn: Nprime_max above the supported 4096");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_knn(ctx, X, N, p, dtype, Xref, M, Nprime, Nprime_max, idx, status);
}

lagp_status lagp_knn_tc_dist(lagp_ctx *ctx, const void *X, int64_t N, int32_t p, lagp_dtype dtype,
                             const void *Xref, int64_t M, float *out) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    LAGP_TRY(check_design(ctx, X, N, p, dtype, "lagp_knn_tc_dist"));
    if (M < 1 || !Xref || !out) return lagp_fail(ctx, LAGP_EINVAL, "lagp_knn_tc_dist: need M >= 1, Xref, out");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_knn_tc_dist(ctx, X, N, p, dtype, Xref, M, out);
}

lagp_status lagp_knn_tc_stall(lagp_ctx *ctx) {
    if (!ctx) return LAGP_EINVAL;
    ctx->knn_tc_stall = 1;
    return LAGP_OK;
}

lagp_status lagp_knn_stats(lagp_ctx *ctx, int64_t *n_retry, int32_t *tc_failed) {
    if (!ctx || !n_retry || !tc_failed) return LAGP_EINVAL;
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return knn_last_stats(ctx, n_retry, tc_failed);
}

// --------------------------------------------------------------- ALC search

static lagp_status alc_common(lagp_ctx *ctx, const char *fn, const void *X, int64_t N, int32_t p,
                              lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *idx,
                              const int32_t *Nprime, int32_t Nprime_max, int32_t n0, const int32_t *n,
                              int32_t n_max, const double *d, double g, lagp_precision prec,
                              int32_t *sel, double *alc, int32_t *status, const void *Y,
                              double *mean, double *s2, double *df) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    const std::string f(fn);
    LAGP_TRY(check_design(ctx, X, N, p, dtype, fn));
    if (M < 0 || M >= LAGP_M_LIMIT) return lagp_fail(ctx, LAGP_EINVAL, f + ": need 0 <= M < 2^30");
    if (M == 0) return LAGP_OK;
    if (!Xref || !idx || !d || !sel || !status)
        return lagp_fail(ctx, LAGP_EINVAL, f + ": NULL required array");
    if (Nprime_max < 1 || Nprime_max > N || Nprime_max > 4096)
        return lagp_fail(ctx, LAGP_EINVAL, f + ": need 1 <= Nprime_max <= min(N, 4096)");
    if (n0 < 1 || n_max < n0 || n_max > Nprime_max || n_max > 128)
        return lagp_fail(ctx, LAGP_EINVAL, f + ": need 1 <= n0 <= n_max <= min(Nprime_max, 128)");
    if (!(g >= 0.0) || !std::isfinite(g)) return lagp_fail(ctx, LAGP_EINVAL, f + ": g must be >= 0");
    if (prec != LAGP_PREC_F64 && prec != LAGP_PREC_F32BULK && prec != LAGP_PREC_F64SCHUR &&
        prec != LAGP_PREC_F32BULK_F64)
        return lagp_fail(ctx, LAGP_EINVAL, f + ": unknown precision");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    AlcArgs a{X, N, p, dtype, Xref, M, idx, Nprime, Nprime_max, n0, n, n_max, d, g, sel, alc, status,
              Y, mean, s2, df};
    if (prec == LAGP_PREC_F64) return launch_alc_f64(ctx, a);
    if (prec == LAGP_PREC_F64SCHUR) return launch_alc_f64schur(ctx, a);
    // FP32-bulk (either re-score): the locations where the FP32 screen broke
    // down (no contender with m^{-1} > 0: near-singular local matrices) are
    // redone by the FP64 Schur form in a second launch that returns at once
    // when there are none
    int *cnt = nullptr;
    unsigned long long *wk = nullptr;
    LAGP_TRY(alc_counters(ctx, &cnt, &wk));
    int *fails = reinterpret_cast<int *>(reinterpret_cast<char *>(cnt) + 64);
    LAGP_CUDA(ctx, cudaMemsetAsync(fails, 0, sizeof(int), ctx->stream));
    a.fail_count = fails;
    LAGP_TRY(prec == LAGP_PREC_F32BULK ? launch_alc_f32(ctx, a) : launch_alc_f32x64(ctx, a));
    const std::string key = ctx->last_alc_key;  // (the autotuner records under the FP32-bulk key)
    AlcArgs r = a;
    r.fail_count = nullptr;
    r.retry_count = fails;
    const lagp_status rc = launch_alc_f64schur(ctx, r);
    ctx->last_alc_key = key;
    return rc;
}

lagp_status lagp_alc_select(lagp_ctx *ctx, const void *X, int64_t N, int32_t p,
                            lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *idx,
                            const int32_t *Nprime, int32_t Nprime_max, int32_t n0,
                            const int32_t *n, int32_t n_max, const double *d, double g,
                            lagp_precision prec, int32_t *sel, double *alc, int32_t *status) {
    return alc_common(ctx, "lagp_alc_select", X, N, p, dtype, Xref, M, idx, Nprime, Nprime_max, n0, n,
                      n_max, d, g, prec, sel, alc, status, nullptr, nullptr, nullptr, nullptr);
}

lagp_status lagp_alc_predict(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                             lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *idx,
                             const int32_t *Nprime, int32_t Nprime_max, int32_t n0,
                             const int32_t *n, int32_t n_max, const double *d, double g,
                             lagp_precision prec, int32_t *sel, double *alc, double *mean,
                             double *s2, double *df, int32_t *status) {
    if (ctx && M > 0 && (!Y || !mean || !s2 || !df)) {
        ctx->err = "lagp_alc_predict: NULL Y or prediction output";
        return LAGP_EINVAL;
    }
    return alc_common(ctx, "lagp_alc_predict", X, N, p, dtype, Xref, M, idx, Nprime, Nprime_max, n0,
                      n, n_max, d, g, prec, sel, alc, status, Y, mean, s2, df);
}

// --------------------------------------------------------- predict / MLE

static lagp_status check_gp(lagp_ctx *ctx, const GpArgs &a, const char *fn, bool need_ref) {
    LAGP_TRY(check_design(ctx, a.X, a.N, a.p, a.dtype, fn));
    if (a.M < 0 || a.M >= LAGP_M_LIMIT) return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": need 0 <= M < 2^30");
    if (a.M == 0) return LAGP_OK;
    if (!a.Y || !a.sel || (need_ref && !a.Xref))
        return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": NULL required array");
    if (a.nmax < 1 || a.nmax > 256)
        return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": need 1 <= n_max <= 256");
    if (!(a.g >= 0.0) || !std::isfinite(a.g))
        return lagp_fail(ctx, LAGP_EINVAL, std::string(fn) + ": g must be >= 0");
    return LAGP_OK;
}

lagp_status lagp_predict(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                         lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *sel,
                         const int32_t *n, int32_t n_max, const double *d, double g,
                         double *mean, double *s2, double *df, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    GpArgs a{X, Y, N, p, dtype, Xref, M, sel, n, n_max, g};
    LAGP_TRY(check_gp(ctx, a, "lagp_predict", true));
    if (M == 0) return LAGP_OK;
    if (!d || !mean || !s2 || !df || !status)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict: NULL output or d");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_predict(ctx, a, d, mean, s2, df, status);
}

lagp_status lagp_mle_step(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                          lagp_dtype dtype, int64_t M, const int32_t *sel, const int32_t *n,
                          int32_t n_max, double *d, double g, double dmin, double dmax,
                          int32_t max_iter, double *llik, double *dllik, double *d2llik,
                          int32_t *iters, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    GpArgs a{X, Y, N, p, dtype, nullptr, M, sel, n, n_max, g};
    LAGP_TRY(check_gp(ctx, a, "lagp_mle_step", false));
    if (M == 0) return LAGP_OK;
    if (!d || !status) return lagp_fail(ctx, LAGP_EINVAL, "lagp_mle_step: NULL d or status");
    if (!(dmin > 0.0) || !(dmax >= dmin) || !std::isfinite(dmax) || max_iter < 0 || max_iter > 1000)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_mle_step: need 0 < dmin <= dmax, 0 <= max_iter <= 1000");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_mle(ctx, a, d, dmin, dmax, max_iter, llik, dllik, d2llik, iters, status);
}

lagp_status lagp_predict_grad(lagp_ctx *ctx, const void *X, const void *Y, int64_t N,
                              int32_t p, lagp_dtype dtype, const void *Xref, int64_t M,
                              const int32_t *sel, const int32_t *n, int32_t n_max,
                              const double *d, double g, double *dmean_dd, double *dmean_dg,
                              double *ds2_dd, double *ds2_dg, double *dllik_dd,
                              double *dllik_dg, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    GpArgs a{X, Y, N, p, dtype, Xref, M, sel, n, n_max, g};
    LAGP_TRY(check_gp(ctx, a, "lagp_predict_grad", true));
    if (M == 0) return LAGP_OK;
    if (!d || !status) return lagp_fail(ctx, LAGP_EINVAL, "lagp_predict_grad: NULL d or status");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_predict_grad(ctx, a, d, dmean_dd, dmean_dg, ds2_dd, ds2_dg, dllik_dd, dllik_dg,
                               status);
}

// ------------------------------------------------- whole method, host buffers

lagp_status lagp_agp(lagp_ctx *ctx, const void *X, const void *Y, int64_t N, int32_t p,
                     lagp_dtype dtype, const void *Xref, int64_t M, const int32_t *Nprime,
                     int32_t Nprime_max, int32_t n0, const int32_t *n, int32_t n_max,
                     double d0, double g, lagp_precision prec, int32_t mle_rounds, double dmin,
                     double dmax, int32_t max_iter, double *mean, double *s2, double *df,
                     double *d_out, int32_t *status) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    LAGP_TRY(check_design(ctx, X, N, p, dtype, "lagp_agp"));
    if (M < 0 || M >= LAGP_M_LIMIT) return lagp_fail(ctx, LAGP_EINVAL, "lagp_agp: need 0 <= M < 2^30");
    if (M == 0) return LAGP_OK;
    if (!Y || !Xref || !mean || !s2 || !df || !status)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_agp: NULL required array");
    if (!(d0 > 0.0)) return lagp_fail(ctx, LAGP_EINVAL, "lagp_agp: d0 must be > 0");
    if (mle_rounds < 0 || mle_rounds > LAGP_MAX_MLE_ROUNDS)
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_agp: mle_rounds must be in [0, 16]");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));

    const size_t es = dtype == LAGP_F64 ? 8 : 4;
    // device layout inside one workspace slot, each region 256-byte aligned
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t oX = 0, oY = oX + al(N * p * es), oR = oY + al(N * es), oNp = oR + al(M * p * es);
    size_t on = oNp + al(M * 4), oIdx = on + al(M * 4), oSel = oIdx + al(M * (size_t)Nprime_max * 4);
    size_t od = oSel + al(M * (size_t)n_max * 4), oMean = od + al(M * 8), oS2 = oMean + al(M * 8);
    // statuses: kNN, then (selection, MLE) per round (one selection without
    // MLE), then prediction
    const int nst = 2 + 2 * (mle_rounds > 0 ? mle_rounds : 1);
    size_t oDf = oS2 + al(M * 8), oSt = oDf + al(M * 8), total = oSt + (size_t)nst * al(M * 4);
    char *base = static_cast<char *>(lagp_ws(ctx, WS_AGP_IO, total));
    if (!base) return LAGP_ENOMEM;
    void *dX = base + oX, *dY = base + oY, *dR = base + oR;
    int32_t *dNp = Nprime ? reinterpret_cast<int32_t *>(base + oNp) : nullptr;
    int32_t *dn = n ? reinterpret_cast<int32_t *>(base + on) : nullptr;
    int32_t *dIdx = reinterpret_cast<int32_t *>(base + oIdx);
    int32_t *dSel = reinterpret_cast<int32_t *>(base + oSel);
    double *dd = reinterpret_cast<double *>(base + od);
    double *dMean = reinterpret_cast<double *>(base + oMean);
    double *dS2 = reinterpret_cast<double *>(base + oS2);
    double *dDf = reinterpret_cast<double *>(base + oDf);
    auto dSt = [&](int i) { return reinterpret_cast<int32_t *>(base + oSt + (size_t)i * al(M * 4)); };
    cudaStream_t st = ctx->stream;

    LAGP_CUDA(ctx, cudaMemcpyAsync(dX, X, N * p * es, cudaMemcpyHostToDevice, st));
    LAGP_CUDA(ctx, cudaMemcpyAsync(dY, Y, N * es, cudaMemcpyHostToDevice, st));
    LAGP_CUDA(ctx, cudaMemcpyAsync(dR, Xref, M * p * es, cudaMemcpyHostToDevice, st));
    if (Nprime) LAGP_CUDA(ctx, cudaMemcpyAsync(dNp, Nprime, M * 4, cudaMemcpyHostToDevice, st));
    if (n) LAGP_CUDA(ctx, cudaMemcpyAsync(dn, n, M * 4, cudaMemcpyHostToDevice, st));
    // d starts at d0 everywhere
    fill_f64_kernel<<<(unsigned)std::min<int64_t>((M + 255) / 256, 1024), 256, 0, st>>>(dd, M, d0);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    LAGP_TRY(lagp_knn(ctx, dX, N, p, dtype, dR, M, dNp, Nprime_max, dIdx, dSt(0)));
    if (mle_rounds > 0) {
        // Fig. 1 steps 2-3, repeated (step 4): design at the current d, MLE of
        // d on that design starting from the current d; then prediction (step
        // 5) with the last design and estimate
        for (int r = 0; r < mle_rounds; r++) {
            LAGP_TRY(lagp_alc_select(ctx, dX, N, p, dtype, dR, M, dIdx, dNp, Nprime_max, n0, dn, n_max,
                                     dd, g, prec, dSel, nullptr, dSt(1 + 2 * r)));
            LAGP_TRY(lagp_mle_step(ctx, dX, dY, N, p, dtype, M, dSel, dn, n_max, dd, g, dmin, dmax,
                                   max_iter, nullptr, nullptr, nullptr, nullptr, dSt(2 + 2 * r)));
        }
        LAGP_TRY(lagp_predict(ctx, dX, dY, N, p, dtype, dR, M, dSel, dn, n_max, dd, g, dMean, dS2,
                              dDf, dSt(nst - 1)));
    } else {
        // prediction carried by the search itself (one kernel)
        LAGP_TRY(lagp_alc_predict(ctx, dX, dY, N, p, dtype, dR, M, dIdx, dNp, Nprime_max, n0, dn,
                                  n_max, dd, g, prec, dSel, nullptr, dMean, dS2, dDf, dSt(1)));
        LAGP_CUDA(ctx, cudaMemsetAsync(dSt(2), 0, M * 4, st));
        LAGP_CUDA(ctx, cudaMemsetAsync(dSt(3), 0, M * 4, st));
    }
    LAGP_CUDA(ctx, cudaMemcpyAsync(mean, dMean, M * 8, cudaMemcpyDeviceToHost, st));
    LAGP_CUDA(ctx, cudaMemcpyAsync(s2, dS2, M * 8, cudaMemcpyDeviceToHost, st));
    LAGP_CUDA(ctx, cudaMemcpyAsync(df, dDf, M * 8, cudaMemcpyDeviceToHost, st));
    if (d_out) LAGP_CUDA(ctx, cudaMemcpyAsync(d_out, dd, M * 8, cudaMemcpyDeviceToHost, st));
    // the stages' statuses through the context's pinned staging buffer
    const size_t sv_bytes = (size_t)nst * M * 4;
    if (ctx->host_pin_bytes < sv_bytes) {
        if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
        ctx->host_pin = nullptr;
        ctx->host_pin_bytes = 0;
        LAGP_CUDA(ctx, cudaHostAlloc(&ctx->host_pin, sv_bytes, cudaHostAllocDefault));
        ctx->host_pin_bytes = sv_bytes;
    }
    int32_t *sv = static_cast<int32_t *>(ctx->host_pin);
    for (int i = 0; i < nst; i++)
        LAGP_CUDA(ctx, cudaMemcpyAsync(sv + (size_t)i * M, dSt(i), M * 4, cudaMemcpyDeviceToHost, st));
    LAGP_CUDA(ctx, cudaStreamSynchronize(st));
    // first failing stage wins: kNN, then each round's selection and MLE, then prediction
    for (int64_t m = 0; m < M; m++) {
        int32_t v = LAGP_OK;
        for (int i = 0; i < nst && v == LAGP_OK; i++) v = sv[(size_t)i * M + m];
        status[m] = v;
    }
    return LAGP_OK;
}

}  // extern "C"
