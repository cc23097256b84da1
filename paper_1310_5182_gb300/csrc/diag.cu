// Diagnostic entry points: the kernels' own FP64 exponential, evaluated
// beside the CUDA library's exp on the same arguments, and the double-float
// split of a double and double-float exponential (for their accuracy tests).
#include <cuda_runtime.h>

#include "df64.cuh"
#include "device_util.cuh"
#include "exp64.cuh"
#include "lagp_internal.h"

namespace {

__global__ void exp64_check_kernel(const double *a, int64_t n, double *out_tang, double *out_lib) {
    __shared__ double tab[EXP64_TABLE_SIZE];
    for (int i = threadIdx.x; i < EXP64_TABLE_SIZE; i += blockDim.x) tab[i] = exp64_table_g[i];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out_tang[i] = exp64_tang(a[i], tab);
        out_lib[i] = exp(a[i]);
    }
}

__global__ void df_check_kernel(const double *a, int64_t n, float *split, float *ex) {
    __shared__ float2 tab[EXP64_TABLE_SIZE];
    for (int i = threadIdx.x; i < EXP64_TABLE_SIZE; i += blockDim.x) {
        const dfl t = df_from_double(exp64_table_g[i]);
        tab[i] = make_float2(t.hi, t.lo);
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const dfl x = df_from_double(a[i]);
        split[2 * i] = x.hi;
        split[2 * i + 1] = x.lo;
        const dfl e = df_exp(x, tab);
        ex[2 * i] = e.hi;
        ex[2 * i + 1] = e.lo;
    }
}

}  // namespace

extern "C" lagp_status lagp_df_check(lagp_ctx *ctx, const double *a, int64_t n, float *split, float *ex) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!a || !split || !ex)))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_df_check: NULL array or n < 0");
    if (n == 0) return LAGP_OK;
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < 4L * ctx->num_sms ? want : 4L * ctx->num_sms);
    df_check_kernel<<<grid, 256, 0, ctx->stream>>>(a, n, split, ex);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}

extern "C" lagp_status lagp_exp64_check(lagp_ctx *ctx, const double *a, int64_t n, double *out_tang,
                                        double *out_lib) {
    if (!ctx) return LAGP_EINVAL;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!a || !out_tang || !out_lib)))
        return lagp_fail(ctx, LAGP_EINVAL, "lagp_exp64_check: NULL array or n < 0");
    if (n == 0) return LAGP_OK;
    LAGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < 4L * ctx->num_sms ? want : 4L * ctx->num_sms);
    exp64_check_kernel<<<grid, 256, 0, ctx->stream>>>(a, n, out_tang, out_lib);
    ctx->launches++;
    LAGP_CUDA(ctx, cudaGetLastError());
    return LAGP_OK;
}
