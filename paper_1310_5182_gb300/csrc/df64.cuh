// Double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers; normalised,
// |lo| <= ulp(hi) / 2, which carries about 48 significant bits.  On this GPU
// an FP64 warp instruction holds its sub-partition's FP64 unit for ~64
// cycles (and so do conversions between double and float), while FP32
// instructions issue every cycle, so a double-float operation of 3..20 FP32
// instructions is several times cheaper than one FP64 instruction.
//
// Building blocks, each exact:
//   TwoSum   (Knuth)   s = fl(a + b), t = (a + b) - s            6 operations
//   Fast2Sum (Dekker)  the same when |a| >= |b| or a = 0         3 operations
//   TwoProd            p = fl(a b), e = fma(a, b, -p) = a b - p  2 operations
// The double-word operations below are those analysed by M. Joldes,
// J.-M. Muller and V. Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44(2), 2017: the sum
// of a double-word and a float, the accurate sum of two double-words
// (relative error below 3u^2 + 13u^3 even under cancellation), the product
// and the quotient of double-words (relative errors a small multiple of u^2),
// with u = 2^-24.  Dot products accumulate the exact product's leading part
// with TwoSum and everything else in the low word, and are normalised once
// at the end (the error stays a small multiple of u^2 times the sum of the
// terms' magnitudes, like a componentwise FP64 bound at 2^-48).
//
// Conversions to and from FP64 are done on the integer pipe, bit by bit,
// never by the hardware's double/float conversions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_make(float h, float l) { return dfl{h, l}; }
__device__ __forceinline__ dfl df_zero() { return dfl{0.f, 0.f}; }
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

// s + t = a + b exactly
__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    const float da = __fsub_rn(a, ap);
    const float db = __fsub_rn(b, bp);
    return dfl{s, __fadd_rn(da, db)};
}

// s + t = a + b exactly, provided |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return dfl{s, __fsub_rn(b, z)};
}

// p + e = a b exactly (barring underflow)
__device__ __forceinline__ dfl two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return dfl{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_normalize(dfl a) { return fast_two_sum(a.hi, a.lo); }

// x + b, x double-word, b float (relative error <= 2u^2)
__device__ __forceinline__ dfl df_add_f(dfl x, float b) {
    const dfl s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

// x + y, accurate also under cancellation (relative error <= 3u^2 + 13u^3)
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    const dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }

// x + y when no cancellation is expected (same signs, or terms of a sum whose
// error may be relative to the sum of magnitudes): error <= ~2u^2 (|x| + |y|)
__device__ __forceinline__ dfl df_add_sloppy(dfl x, dfl y) {
    const dfl s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// x y, both double-words (relative error a few u^2)
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    dfl c = two_prod(x.hi, y.hi);
    const float t = __fmul_rn(x.hi, y.lo);
    const float l = __fmaf_rn(x.lo, y.hi, t);
    return fast_two_sum(c.hi, __fadd_rn(c.lo, l));
}

// x b, b float
__device__ __forceinline__ dfl df_mul_f(dfl x, float b) {
    dfl c = two_prod(x.hi, b);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, b, c.lo));
}

__device__ __forceinline__ dfl df_sqr(dfl x) {
    dfl c = two_prod(x.hi, x.hi);
    return fast_two_sum(c.hi, __fmaf_rn(x.hi + x.hi, x.lo, c.lo));
}

// acc += x y, acc left unnormalised (the low word collects every rounding
// term); normalise with df_normalize when the sum is complete
__device__ __forceinline__ void df_fma_acc(dfl &acc, dfl x, dfl y) {
    const dfl p = two_prod(x.hi, y.hi);
    float pl = __fmaf_rn(x.hi, y.lo, p.lo);
    pl = __fmaf_rn(x.lo, y.hi, pl);
    const dfl s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, pl));
}

// 1 / y and x / y (y normalised, nonzero): a first quotient from the FP32
// reciprocal, then one correction with the exact remainder
static __device__ __noinline__ dfl df_div(dfl x, dfl y) {
    const float r = __frcp_rn(y.hi);
    const float q1 = __fmul_rn(x.hi, r);
    // remainder x - q1 y, computed as a double-word (q1 y exact by TwoProd)
    const dfl p = two_prod(q1, y.hi);
    const float pl = __fmaf_rn(q1, y.lo, p.lo);
    const dfl rem = df_add(x, dfl{-p.hi, -pl});
    const float q2 = __fmul_rn(rem.hi, r);
    // second correction: the first quotient's error is ~2u, the second
    // term's relative error ~2u, so q1 + q2 is good to a few u^2
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ dfl df_rcp(dfl y) { return df_div(dfl{1.f, 0.f}, y); }

// a > b for normalised double-words
__device__ __forceinline__ bool df_gt(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// ------------------------------------------------------------ conversions

// FP64 -> double-word, on the integer pipe.  hi is the leading 24 significant
// bits rounded to nearest, lo the rest (29 bits, rounded to 24): relative
// error <= 2^-48.  |v| below 2^-74 keeps only hi (relative error 2^-24 of a
// value that small), below 2^-126 (FP32's normal range) becomes 0; |v| at or
// above 2^128 becomes +-inf, NaN stays NaN.
__device__ __forceinline__ dfl df_from_double(double v) {
    const unsigned hw = (unsigned)__double2hiint(v);
    const unsigned lw = (unsigned)__double2loint(v);
    const unsigned sign = hw & 0x80000000u;
    const unsigned ah = hw & 0x7fffffffu;
    const int e = (int)(ah >> 20);  // biased FP64 exponent
    // leading 23 fraction bits, exponent rebiased by 1023 - 127 = 896
    unsigned hb = __funnelshift_l(lw, ah - 0x38000000u, 3);
    const unsigned up = (lw >> 28) & 1u;  // round half up on the 29 dropped bits
    hb += up;                             // a carry moves into the exponent: exact
    // remainder below hi, in units of 2^(e - 1075): [-2^28, 2^28]
    const int rem = (int)(lw & 0x1fffffffu) - (int)(up << 29);
    float lo = __int2float_rn(rem) * __int_as_float((e - 948) << 23);
    float hi = __uint_as_float(hb | sign);
    lo = sign ? -lo : lo;
    if (e < 949) lo = 0.f;
    if (e < 897) hi = __uint_as_float(sign);
    if (e > 1150) {
        hi = (e == 2047 && ((ah & 0xfffffu) | lw)) ? __int_as_float(0x7fc00000) : __uint_as_float(sign | 0x7f800000u);
        lo = 0.f;
    }
    return dfl{hi, lo};
}

// FP32 -> FP64 exactly, on the integer pipe (FP32 subnormals become 0)
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned a = b & 0x7fffffffu;
    if (a < 0x00800000u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (a >= 0x7f800000u)  // inf / NaN
        return __hiloint2double((int)((b & 0x80000000u) | 0x7ff00000u | (a > 0x7f800000u ? 0x80000u : 0u)), 0);
    const unsigned hw = ((a >> 3) + 0x38000000u) | (b & 0x80000000u);
    return __hiloint2double((int)hw, (int)(b << 29));
}

// double-word -> FP64 (one FP64 add)
__device__ __forceinline__ double df_to_double(dfl x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

// ------------------------------------------------------ exponential
// exp(a) for a <= 0 in double-word arithmetic by Tang's table-driven method
// (P. T. P. Tang, ACM TOMS 15(2), 1989), the same reduction as the FP64
// exponential of the library:
//   N = round(a 1024 / ln 2),  r = a - N ln2/1024 (|r| <= ~ln2 / 2048),
//   exp(a) = 2^(N div 1024) 2^((N mod 1024)/1024) (1 + p(r)),
//   p(r) = r + r^2/2 + r^3/6 + r^4/24  (truncation < r^5/120 < 4e-20).
// N ln2/1024 is formed exactly from the double-word ln2/1024 and the
// reduction is an accurate double-word subtraction, so r carries a relative
// error of a few u^2 plus |a| u^2 from the constant (the rounding of a itself
// already costs |a| u^2); r^2/2 is a double-word, r^3/6 + r^4/24 a float.
// tab holds 2^(k/1024), k = 0..1023, as double-words.  a < -87 (results below
// FP32's normal range) gives 0.
constexpr float DF_EXP_INV_L = 0x1.715476p+10f;  // 1024 / ln 2, rounded to FP32
constexpr float DF_EXP_L_HI = 0x1.62e430p-11f;   // ln 2 / 1024 = L_HI + L_LO
constexpr float DF_EXP_L_LO = -0x1.05c610p-39f;  //   to 1.3e-16 relative
constexpr float DF_EXP_SHIFT = 0x1.8p23f;        // rounds to an integer when added

static __device__ __noinline__ dfl df_exp(dfl a, const float2 *tab) {
    if (!(a.hi >= -87.0f)) return df_zero();  // also NaN -> 0 (never produced by the kernels)
    const float t = __fmaf_rn(a.hi, DF_EXP_INV_L, DF_EXP_SHIFT);
    const int N = __float_as_int(t) - __float_as_int(DF_EXP_SHIFT);
    const float nf = __fsub_rn(t, DF_EXP_SHIFT);  // exact
    // N ln2/1024 as an (unnormalised) double-word: exact product with L_HI,
    // N L_LO rounded once
    const dfl p = two_prod(nf, DF_EXP_L_HI);
    const float pl = __fmaf_rn(nf, DF_EXP_L_LO, p.lo);
    const dfl r = df_add(a, dfl{-p.hi, -pl});
    // p(r) = r + r^2/2 + (r^3/6 + r^4/24)
    const dfl r2 = df_sqr(r);
    const float c34 = __fmul_rn(__fmul_rn(r2.hi, r.hi), __fmaf_rn(r.hi, 1.f / 24.f, 1.f / 6.f));
    dfl pm1 = df_add_sloppy(r, dfl{0.5f * r2.hi, 0.5f * r2.lo});
    pm1.lo = __fadd_rn(pm1.lo, c34);
    const float2 T2 = tab[N & 1023];
    const dfl T{T2.x, T2.y};
    dfl e = df_add_sloppy(T, df_mul(T, pm1));
    // times 2^(N div 1024): N >= -128,500 here, so the scale stays normal
    const float sc = __int_as_float(((N >> 10) + 127) << 23);
    return dfl{__fmul_rn(e.hi, sc), __fmul_rn(e.lo, sc)};
}
