// Device helpers shared by the kNN kernels (CUDA-core screen and sort, and
// the tensor-core collection pass): order-preserving keys of doubles, the
// centre and half-width of the coordinates, and size rounding.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Unsigned keys with the order of the doubles (0 below every key), so that
// zero-initialised buffers work as the identity of atomicMax.
__device__ __forceinline__ unsigned long long dkey(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Centre c_i (midrange of coordinate i) and B = max_i |x_i - c_i| (with a
// relative slack of 2^-50 for the rounding of c_i), from the bounds of the
// finite coordinates (a coordinate with none gets c_i = 0, B unchanged).
__device__ void centre_and_bound(const unsigned long long *kmax, const unsigned long long *kmin,
                                 int p, double *c, double &B) {
    double b = 0.0;
    for (int i = 0; i < p; i++) {
        if (kmax[i] == 0ull) {  // no finite value in this coordinate
            c[i] = 0.0;
            continue;
        }
        const double hi = dkey_inv(kmax[i]), lo = dkey_inv(~kmin[i]);
        const double ci = 0.5 * lo + 0.5 * hi;
        c[i] = ci;
        b = fmax(b, fmax(hi - ci, ci - lo) + 0x1p-52 * fmax(fabs(lo), fabs(hi)));
    }
    B = b * (1.0 + 0x1p-50);
}

// ----------------------------------------- tensor-core collection bounds
// Assumed error of one tensor-core instruction (kind::f16, FP32
// accumulation): at most TC_ACC_ULPS units of 2^-24 times the sum of the
// magnitudes of its products and accumulator.
constexpr double TC_ACC_ULPS = 64.0;

// FP16 values per operand row for p coordinates (3p split products and four
// norm terms, in multiples of 16: one MMA instruction takes 16)
__host__ __device__ inline int tc_k(int p) { return (3 * p + 4 + 15) & ~15; }

// The operands are the centred coordinates scaled by 2^-e, the power of two
// with B <= 2^e (|y 2^-e| <= 1; an exact scaling), and s carries 2^-2e.
__host__ __device__ inline int tc_scale_exp(double B) {
    int e = 0;
    frexp(B, &e);
    return e;
}

// The error E_tc of a tensor-core value s against |y_q - y_x|^2 (original
// units).  With S = 2^e, u = 2^-24 (widened by 2^-27 for the FP64 centring),
// each scaled value v split into FP16 parts with |v - v_h - v_l| <=
// max(2^-22 |v|, 2^-25), and the products of the parts exact in FP32:
//   per coordinate, |A| <= 2 (A = -2 y_q / S), |b| <= 1 (b = y_x / S):
//     |A| |db| + |b| |dA| + |A_l b_l| <= 2^-21 + 2^-21 + 2^-21 (+ 2^-21 slack)
//   E_tc = S^2 [ 4p 2^-21                                  (cross terms)
//              + 2 (gamma_p p + 2^-22 p + 2^-25)           (two norms, splits)
//              + TC_ACC_ULPS (K/16) 2^-24 4p (1 + 2^-9) ]  (accumulation)
// A row with s <= tau0 then has exact distance r <= sqrt(tau0 + E_tc) + e2
// (e2 = 2uB sqrt(p)), and every row of the exact top N' has s <= (r_hi +
// e2)^2 + E_tc.
__device__ inline double tc_error_bound(int p, int K, double B) {
    const double u = 0x1p-24 * (1.0 + 0x1p-27);
    const double S = ldexp(1.0, tc_scale_exp(B));
    const double gp = p * u / (1.0 - p * u);
    return S * S * (4.0 * p * 0x1p-21 + 2.0 * (gp * p + 0x1p-22 * p + 0x1p-25) +
                    TC_ACC_ULPS * (K / 16) * 0x1p-24 * 4.0 * p * (1.0 + 0x1p-9));
}

__device__ inline double tc_margin(float tau, int p, int K, double B) {
    const double u = 0x1p-24 * (1.0 + 0x1p-27);
    const double e2 = 2.0 * u * B * sqrt((double)p);
    const double E = tc_error_bound(p, K, B);
    const double r_hi = sqrt((double)tau + E) * (1.0 + 1e-13) + e2;
    const double r_col = r_hi + e2;
    return (r_col * r_col + E) * (1.0 + 1e-12);
}

// A lower bound on the exact distance R such that every row within R of the
// query has a tensor-core value s <= tau2 (and so was collected):
//   s <= (r + e2)^2 + E_tc <= tau2  whenever  r <= sqrt(tau2 - E_tc) - e2.
__device__ inline double tc_collected_radius(float tau2, int p, int K, double B) {
    const double u = 0x1p-24 * (1.0 + 0x1p-27);
    const double e2 = 2.0 * u * B * sqrt((double)p);
    const double v = ((double)tau2 * (1.0 - 1e-12) - tc_error_bound(p, K, B));
    return v > 0.0 ? sqrt(v) * (1.0 - 1e-13) - e2 : -1.0;
}

}  // namespace
