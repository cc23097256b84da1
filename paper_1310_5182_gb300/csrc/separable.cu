// Separable lengthscales (Sec. 3.1: the correlation "via a vectorized theta
// parameter").  K(x,x') = exp(-sum_i (x_i - x'_i)^2 / theta_i) is the
// isotropic correlation with d = 1 of the inputs scaled column by column,
// y_i = x_i / sqrt(theta_i); this entry point writes that scaling, after
// which every search and prediction entry point evaluates the separable
// correlation when called on the scaled inputs with d = 1.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "lagp_internal.h"

namespace {

__global__ void scale_kernel(const void *X, int64_t N, int p, lagp_dtype dt, const double *theta,
                             double *Xs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * p; e += stride) {
        const int i = (int)(e % p);
        Xs[e] = load_coord64(X, e / p, p, i, dt) / sqrt(theta[i]);
    }
}

}  // namespace

extern "C" lagp_status lagp_scale_inputs(lagp_ctx *ctx, const void *X, int64_t N, int32_t p,
                                         lagp_dtype dtype, const double *theta, double *Xs) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    if (N < 0 || p < 1 || p > 64 || (dtype != LAGP_F64 && dtype != LAGP_F32))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_scale_inputs: need N >= 0, 1 <= p <= 64, dtype F64/F32");
    if (N == 0) return LAGP_OK;
    if (!X || !theta || !Xs) return lagp_fail(ctx, LAGP_EINVAL, "lagp_scale_inputs: NULL array");
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t blocks = (N * p + 255) / 256;
    scale_kernel<<<(unsigned)(blocks < 4L * ctx->num_sms ? blocks : 4L * ctx->num_sms), 256, 0, ctx->stream>>>(
        X, N, p, dtype, theta, Xs);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
