// Internal declarations shared by the translation units of liblagp.so:
// the context, its workspace, and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>

#include "lagp.h"

// Workspace slots owned by a context; each grows on demand.
enum WsSlot {
    WS_KNN_X32 = 0,   // FP32 copy of the design for kNN screening
    WS_KNN_CAND,      // kNN per-query candidate rows
    WS_KNN_META,      // kNN per-query counters / thresholds / flags
    WS_KNN_TC,        // kNN tensor-core operands and sampled thresholds
    WS_ALC_PANEL,     // ALC per-CTA candidate panel (F64 kernel values or F32 whitened U)
    WS_ALC_STATE,     // ALC per-CTA FP64 state (K^{-1}, vectors)
    WS_ALC_COUNTER,   // persistent-grid work counters
    WS_GP_MAT,        // predict / MLE per-CTA matrices
    WS_AGP_IO,        // lagp_agp device copies of inputs and outputs
    WS_TUNE,          // autotuner trial outputs
    WS_NSLOTS
};

struct lagp_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    void *ws[WS_NSLOTS] = {};
    size_t ws_bytes[WS_NSLOTS] = {};
    std::string err;
    lagp_tuning tuning = {0, 0, 0, 0.5, 0};
    int64_t launches = 0;
    // autotuned resident CTAs per SM, keyed by the ALC problem shape
    std::map<std::string, int> tuned_ctas;
    std::map<std::string, int> tuned_tmax;  // FP32-bulk re-score batch by shape
    int tune_override = 0;       // set by the autotuner while it times a candidate
    int tune_tmax_override = 0;  // (the batch size of the candidate)
    std::string last_alc_key;    // shape key of the last ALC launch (the tuner records under it)
    bool work_zeroed = false;  // ALC work counters cleared once after allocation
    int64_t knn_last_M = 0;    // queries of the last lagp_knn call (for lagp_knn_stats)
    int knn_tc_stall = 0;      // test hook for the next tensor-core kNN pass (lagp_knn_tc_stall)
    void *host_pin = nullptr;  // pinned host staging (lagp_agp's statuses), grown on demand
    size_t host_pin_bytes = 0;
};

// Shape key of an ALC launch for the autotuner's table.
std::string alc_shape_key(const char *kernel, int cpt, int nmax, int p, bool fused);
// Resident CTAs per SM for an ALC launch: the autotuner's trial value, the
// user's tuning, the tuned table, or the kernel's default.
int alc_ctas_per_sm(lagp_ctx *ctx, const std::string &key, int default_cps);
// The FP32-bulk re-score batch for a shape: the autotuner's candidate, the
// user's tuning.rescore_max, the tuned choice, or 8.
int alc_rescore_batch(lagp_ctx *ctx, const std::string &key);

// The persistent kernels' work counter (offset 0) and the ALC work counters
// (4 x uint64 at offset 128; the MLE's 2 x uint64 follow at offset 192) of
// the WS_ALC_COUNTER slot.
lagp_status alc_counters(lagp_ctx *ctx, int **counter, unsigned long long **work);

// status helpers (lagp_api.cu)
lagp_status lagp_fail(lagp_ctx *ctx, lagp_status s, const std::string &msg);
lagp_status lagp_cuda_check(lagp_ctx *ctx, cudaError_t e, const char *what);
// returns nullptr and sets the error on failure
void *lagp_ws(lagp_ctx *ctx, WsSlot slot, size_t bytes);

#define LAGP_TRY(expr)                       \
    do {                                     \
        lagp_status _s = (expr);             \
        if (_s != LAGP_OK) return _s;        \
    } while (0)
#define LAGP_CUDA(ctx, expr) LAGP_TRY(lagp_cuda_check((ctx), (expr), #expr))

// ----------------------------------------------------------------- launchers
// Each launcher validates nothing (lagp_api.cu does), enqueues on ctx->stream,
// adds its kernel count to ctx->launches and returns a CUDA error status.

lagp_status launch_knn(lagp_ctx *ctx, const void *X, int64_t N, int p, lagp_dtype dtype,
                       const void *Xref, int64_t M, const int32_t *Np, int32_t Npmax,
                       int32_t *idx, int32_t *status);

// kNN collection pass on the tensor cores (knn_tc.cu)
bool knn_tc_supported(int p);
size_t knn_tc_workspace(int64_t N, int64_t M, int p);
lagp_status launch_knn_tc_prep(lagp_ctx *ctx, void *ws, const void *X, int64_t N, int p, lagp_dtype dtype,
                               const void *Xref, int64_t M, const unsigned long long *kmax,
                               const unsigned long long *kmin, float **tau0, float **rcol);
lagp_status launch_knn_tc_collect(lagp_ctx *ctx, void *ws, int64_t N, int p, int64_t M, const int32_t *Np,
                                  int32_t Npmax, const unsigned long long *kmax, const unsigned long long *kmin,
                                  int32_t *cand, int32_t Cmax, int32_t *cand_count, int32_t *status,
                                  int32_t *retry, int *err, float *rcol, float *dump);
lagp_status launch_knn_tc_dist(lagp_ctx *ctx, const void *X, int64_t N, int p, lagp_dtype dtype,
                               const void *Xref, int64_t M, float *out);
lagp_status knn_last_stats(lagp_ctx *ctx, int64_t *n_retry, int32_t *tc_failed);

struct AlcArgs {
    const void *X;
    int64_t N;
    int p;
    lagp_dtype dtype;
    const void *Xref;
    int64_t M;
    const int32_t *idx;
    const int32_t *Np;  // may be null
    int32_t Npmax;
    int32_t n0;
    const int32_t *n;   // may be null
    int32_t nmax;
    const double *d;
    double g;
    int32_t *sel;
    double *alc;        // may be null
    int32_t *status;
    // fused local prediction (Eqs. predgp, preds2) on the selected design;
    // all four null for a plain search
    const void *Y;
    double *mean, *s2, *df;
    // FP32-bulk: counts the locations that end LAGP_ENOTPD (device int)
    int *fail_count = nullptr;
    // FP64 Schur retry of those: when set, only locations whose status is
    // LAGP_ENOTPD are redone, and nothing at all when *retry_count is 0
    const int *retry_count = nullptr;
};

lagp_status launch_alc_f64(lagp_ctx *ctx, const AlcArgs &a);
lagp_status launch_alc_f32(lagp_ctx *ctx, const AlcArgs &a);
lagp_status launch_alc_f64schur(lagp_ctx *ctx, const AlcArgs &a);
lagp_status launch_alc_f32x64(lagp_ctx *ctx, const AlcArgs &a);

struct GpArgs {
    const void *X;
    const void *Y;
    int64_t N;
    int p;
    lagp_dtype dtype;
    const void *Xref;   // predict / grad only
    int64_t M;
    const int32_t *sel;
    const int32_t *n;   // may be null
    int32_t nmax;
    double g;
};

lagp_status launch_predict(lagp_ctx *ctx, const GpArgs &a, const double *d, double *mean,
                           double *s2, double *df, int32_t *status);
lagp_status launch_mle(lagp_ctx *ctx, const GpArgs &a, double *d, double dmin, double dmax,
                       int32_t max_iter, double *llik, double *dllik, double *d2llik,
                       int32_t *iters, int32_t *status);
lagp_status launch_predict_grad(lagp_ctx *ctx, const GpArgs &a, const double *d,
                                double *dmean_dd, double *dmean_dg, double *ds2_dd,
                                double *ds2_dg, double *dllik_dd, double *dllik_dg,
                                int32_t *status);
