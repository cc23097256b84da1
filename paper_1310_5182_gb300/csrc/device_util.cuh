// Device helpers shared by the kernels of liblagp.so.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "lagp.h"

#define LAGP_FULL_MASK 0xffffffffu

// Coordinate i of row r of a row-major N x p array of either dtype, as double.
__device__ __forceinline__ double load_coord64(const void *A, int64_t r, int p, int i,
                                               lagp_dtype dt) {
    return dt == LAGP_F64 ? static_cast<const double *>(A)[r * p + i]
                          : static_cast<double>(static_cast<const float *>(A)[r * p + i]);
}

__device__ __forceinline__ float load_coord32(const void *A, int64_t r, int p, int i,
                                              lagp_dtype dt) {
    return dt == LAGP_F64 ? static_cast<float>(static_cast<const double *>(A)[r * p + i])
                          : static_cast<const float *>(A)[r * p + i];
}

// Squared distance in FP64, coordinates summed in order 0..p-1, each term a
// separately rounded subtract, multiply and add (no contraction), so that the
// result is bit-identical to any IEEE FP64 evaluation in the same order.
__device__ __forceinline__ double sqdist64_exact(const double *a, const double *b, int p) {
    double s = 0.0;
    for (int i = 0; i < p; i++) {
        double diff = __dsub_rn(a[i], b[i]);
        s = __dadd_rn(s, __dmul_rn(diff, diff));
    }
    return s;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LAGP_FULL_MASK, v, o);
    return v;
}

// (value, row) argmax with ties to the lower row; rows < 0 mean "empty".
struct ArgBest {
    double v;
    int32_t row;   // design row (tie-break key)
    int32_t slot;  // candidate slot within the location
};

__device__ __forceinline__ bool better(double va, int32_t ra, double vb, int32_t rb) {
    if (rb < 0) return ra >= 0;
    if (ra < 0) return false;
    return va > vb || (va == vb && ra < rb);
}

__device__ __forceinline__ ArgBest warp_argmax(ArgBest b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(LAGP_FULL_MASK, b.v, o);
        int32_t orow = __shfl_xor_sync(LAGP_FULL_MASK, b.row, o);
        int32_t oslot = __shfl_xor_sync(LAGP_FULL_MASK, b.slot, o);
        if (better(ov, orow, b.v, b.row)) {
            b.v = ov;
            b.row = orow;
            b.slot = oslot;
        }
    }
    return b;
}
