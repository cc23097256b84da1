// FP64 exponential for the kernel values K(x, x') = exp(-||x - x'||^2 / d).
//
// Method: P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989.  With
// N = round(a * 64 / ln 2) and r = a - N ln2 / 64 (|r| <= ln2 / 128),
//   exp(a) = 2^(N div 64) * 2^((N mod 64) / 64) * exp(r),
// where 2^(k/64) comes from a 64-entry table and exp(r) - 1 from its Taylor
// polynomial of degree 6 (truncation error below r^7/7! < 1e-19).  The
// reduction uses the two-part (Cody-Waite) constant ln2/64 = L_HI + L_LO,
// L_HI holding 36 significant bits so that N * L_HI is exact for |N| < 2^17.
// The power of two is applied by adding N div 64 to the exponent field,
// which is exact while the result stays a normal number; arguments with
// |a| > 700 (and NaN) take the library exp instead.
//
// Cost: 11 FP64 operations and a table read.  Accuracy: the table entries
// and the final fused multiply-add each round once (0.5 ulp each), the
// rest is far below that, so the result is within about 1 ulp of exp(a).
//
// The table and constants are the correctly rounded doubles of 2^(k/64),
// 64/ln 2, 1/k! and the split of ln 2 / 64 described above; a CPU test
// recomputes every one of them in 60-digit decimal arithmetic.
#pragma once
#include <cuda_runtime.h>

#define LAGP_EXP64_TABLE                                                                        \
    {                                                                                           \
        0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0, \
        0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0, \
        0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0, \
        0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0, \
        0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0, \
        0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0, \
        0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0, \
        0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0, \
        0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0, \
        0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0, \
        0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0, \
        0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0, \
        0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0, \
        0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0, \
        0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0, \
        0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0  \
    }

// The table in global memory; kernels copy it to shared memory once.
static __device__ const double exp64_table_g[64] = LAGP_EXP64_TABLE;

constexpr double EXP64_INV_L = 0x1.71547652b82fep+6;  // 64 / ln 2
constexpr double EXP64_L_HI = 0x1.62e42fefa0000p-7;   // ln 2 / 64, leading 36 bits
constexpr double EXP64_L_LO = 0x1.cf79abc9e3b3ap-46;  // ln 2 / 64 - L_HI
constexpr double EXP64_SHIFT = 0x1.8p52;              // rounds to an integer when added
constexpr double EXP64_C2 = 0x1.0000000000000p-1;     // 1/2!
constexpr double EXP64_C3 = 0x1.5555555555555p-3;     // 1/3!
constexpr double EXP64_C4 = 0x1.5555555555555p-5;     // 1/4!
constexpr double EXP64_C5 = 0x1.1111111111111p-7;     // 1/5!
constexpr double EXP64_C6 = 0x1.6c16c16c16c17p-10;    // 1/6!
constexpr long long EXP64_FAST_MAX_BITS = 0x4085e00000000000LL;  // bits of 700.0

// exp(a); `tab` is the 64-entry table above (shared memory in the kernels).
__device__ __forceinline__ double exp64_tang(double a, const double *tab) {
    const long long abits = __double_as_longlong(a) & 0x7fffffffffffffffLL;
    if (abits > EXP64_FAST_MAX_BITS) return exp(a);  // |a| > 700, infinities, NaN
    const double t = fma(a, EXP64_INV_L, EXP64_SHIFT);
    const int N = __double2loint(t);  // low word of SHIFT + N holds N
    const double nd = t - EXP64_SHIFT;
    double r = fma(-nd, EXP64_L_HI, a);
    r = fma(-nd, EXP64_L_LO, r);
    double q = fma(r, EXP64_C6, EXP64_C5);
    q = fma(r, q, EXP64_C4);
    q = fma(r, q, EXP64_C3);
    q = fma(r, q, EXP64_C2);
    const double pm1 = fma(r * r, q, r);  // exp(r) - 1
    const double T = tab[N & 63];
    const double e = fma(T, pm1, T);
    const unsigned long long scale = static_cast<unsigned long long>(static_cast<long long>(N >> 6)) << 52;
    return __longlong_as_double(static_cast<long long>(static_cast<unsigned long long>(__double_as_longlong(e)) + scale));
}
