// Autotuner for the persistent ALC kernels: times the search on a sample of
// the caller's problem for every admissible count of resident CTAs per SM
// (and, for the FP32-bulk kernel, two double-float re-score batch sizes) and
// records the fastest for that problem shape on the context.
#include <cuda_runtime.h>
#include <stdio.h>

#include <string>

#include "lagp_internal.h"

std::string alc_shape_key(const char *kernel, int cpt, int nmax, int p, bool fused) {
    char buf[96];
    snprintf(buf, sizeof buf, "%s/cpt%d/n%d/p%d/%s", kernel, cpt, nmax, p, fused ? "pred" : "sel");
    return buf;
}

int alc_ctas_per_sm(lagp_ctx *ctx, const std::string &key, int default_cps) {
    ctx->last_alc_key = key;
    if (ctx->tune_override > 0) return ctx->tune_override;
    if (ctx->tuning.ctas_per_sm > 0) return ctx->tuning.ctas_per_sm;
    auto it = ctx->tuned_ctas.find(key);
    return it != ctx->tuned_ctas.end() ? it->second : default_cps;
}

int alc_rescore_batch(lagp_ctx *ctx, const std::string &key) {
    if (ctx->tune_tmax_override > 0) return ctx->tune_tmax_override;
    if (ctx->tuning.rescore_max > 0) return ctx->tuning.rescore_max;
    auto it = ctx->tuned_tmax.find(key);
    return it != ctx->tuned_tmax.end() ? it->second : 8;
}

extern "C" lagp_status lagp_autotune(lagp_ctx *ctx, const void *X, int64_t N, int32_t p,
                                     lagp_dtype dtype, const void *Xref, int64_t M,
                                     const int32_t *idx, const int32_t *Nprime, int32_t Nprime_max,
                                     int32_t n0, const int32_t *n, int32_t n_max, const double *d,
                                     double g, lagp_precision prec, const void *Y,
                                     int32_t *best_ctas_per_sm, int32_t *best_rescore_max) {
    if (!ctx) return LAGP_EINVAL;
    if (M <= 0) return lagp_fail(ctx, LAGP_EINVAL, "lagp_autotune: M must be > 0");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    // a sample large enough to keep every candidate grid busy for several waves
    const int64_t Ms = M < (int64_t)ctx->num_sms * 16 ? M : (int64_t)ctx->num_sms * 16;
    const size_t al = 256;
    auto up = [&](size_t b) { return (b + al - 1) / al * al; };
    const size_t bsel = up((size_t)Ms * n_max * 4), bst = up((size_t)Ms * 4), bd = up((size_t)Ms * 8);
    char *ws = static_cast<char *>(lagp_ws(ctx, WS_TUNE, bsel + bst + 3 * bd));
    if (!ws) return LAGP_ENOMEM;
    int32_t *sel = reinterpret_cast<int32_t *>(ws);
    int32_t *st = reinterpret_cast<int32_t *>(ws + bsel);
    double *mean = reinterpret_cast<double *>(ws + bsel + bst);
    double *s2 = mean + bd / 8, *df = s2 + bd / 8;
    cudaEvent_t e0, e1;
    LAGP_CUDA(ctx, cudaEventCreate(&e0));
    LAGP_CUDA(ctx, cudaEventCreate(&e1));
    const int max_cps = (prec == LAGP_PREC_F32BULK || prec == LAGP_PREC_F32BULK_F64) ? 4 : 3;
    // the FP32-bulk kernel's re-score batch too (unless the user fixed it)
    const bool tune_b = prec == LAGP_PREC_F32BULK && ctx->tuning.rescore_max == 0;
    const int batches[3] = {16, 8, 4};
    float best_ms = 1e30f;
    int best = 0, best_b = 0;
    std::string key;
    lagp_status rc = LAGP_OK;
    for (int trial = 0; trial < max_cps * (tune_b ? 3 : 1) && rc == LAGP_OK; trial++) {
        const int cps = 1 + trial % max_cps, tb = tune_b ? batches[trial / max_cps] : 0;
        ctx->tune_override = cps;
        ctx->tune_tmax_override = tb;
        float ms_sum = 0.f;
        for (int rep = 0; rep < 3 && rc == LAGP_OK; rep++) {
            cudaEventRecord(e0, ctx->stream);
            rc = Y ? lagp_alc_predict(ctx, X, Y, N, p, dtype, Xref, Ms, idx, Nprime, Nprime_max, n0, n,
                                      n_max, d, g, prec, sel, nullptr, mean, s2, df, st)
                   : lagp_alc_select(ctx, X, N, p, dtype, Xref, Ms, idx, Nprime, Nprime_max, n0, n,
                                     n_max, d, g, prec, sel, nullptr, st);
            cudaEventRecord(e1, ctx->stream);
            if (rc != LAGP_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = lagp_cuda_check(ctx, cudaGetLastError(), "lagp_autotune: trial");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_sum += ms;  // the first repetition warms caches and workspaces
        }
        if (rc == LAGP_OK && ms_sum < best_ms) {
            best_ms = ms_sum;
            best = cps;
            best_b = tb;
        }
        key = ctx->last_alc_key;  // the launcher's own key for this shape
    }
    ctx->tune_override = 0;
    ctx->tune_tmax_override = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LAGP_OK) return rc;
    // recorded under the key the launcher looked up during the trials
    ctx->tuned_ctas[key] = best;
    if (tune_b) ctx->tuned_tmax[key] = best_b;
    if (best_ctas_per_sm) *best_ctas_per_sm = best;
    if (best_rescore_max) *best_rescore_max = tune_b ? best_b : alc_rescore_batch(ctx, key);
    return LAGP_OK;
}
