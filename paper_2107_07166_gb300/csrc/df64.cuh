// Double-float ("double-word") arithmetic on the FP32 units: a value is hi + lo with two
// binary32 words, |lo| <= ulp(hi)/2 when normalised, about 48 significant bits.  On GB300
// the FP32 units issue 58x the binary64 rate (73.4 vs 1.256 TFLOP/s measured), so the
// binary64-accurate mode of the FMM evaluates its pair kernels in this type.
//
// Building blocks (published error-free transformations):
//   TwoSum      Knuth, TAOCP vol. 2 (1969): s + e = a + b exactly, 6 flops
//   FastTwoSum  Dekker (1971), |a| >= |b|:  s + e = a + b exactly, 3 flops
//   TwoProd     with FMA: p + e = a * b exactly, 2 flops
//   add         Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic
//               building blocks of double-word arithmetic", ACM TOMS 44 (2017),
//               Algorithm 6 (AccurateDWPlusDW), relative error <= 3u^2 + 13u^3
//   mul         same paper, Algorithm 12 (DWTimesDW3, FMA), relative error <= 4u^2
//   fma_t       accumulation c + a*b: the product's exact head and its cross terms, the
//               head added to c.hi with TwoSum and every low part gathered in c.lo; c is
//               left unnormalised (|lo| grows like a few ulp(hi) over long sums) and is
//               normalised by norm() before it leaves a kernel
//   rsqrt_t     x^-1/2 from the binary32 estimate y refined by one binary32 Newton step;
//               with the residual e = 1 - x y^2 formed in double-word arithmetic,
//               x^-1/2 = y (1 - e)^-1/2 = y (1 + e/2 + 3e^2/8 + O(e^3)), |e| ~ 2^-23, so the
//               truncation error is ~2^-69 and the result is limited by the format
#pragma once
#include <cuda_runtime.h>

namespace gbfmm {

struct df64 {
    float hi, lo;
    __host__ __device__ constexpr df64() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // exact for every binary32 value; for a binary64 constant it keeps ~48 bits
    __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df64(int i) : hi((float)i), lo(0.f) {}
};

__device__ __forceinline__ df64 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64(s, e);
}

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df64(s, e);
}

__device__ __forceinline__ df64 two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df64(p, e);
}

__device__ __forceinline__ df64 norm(df64 a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
    df64 s = two_sum(x.hi, y.hi);
    df64 t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    df64 v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
    df64 c = two_prod(x.hi, y.hi);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(c.lo, cl2);
    return fast_two_sum(c.hi, cl3);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
    a = a + b;
    return a;
}

// c + a*b, accumulation form (see the header comment)
__device__ __forceinline__ df64 fma_t(df64 a, df64 b, df64 c) {
    float ph = __fmul_rn(a.hi, b.hi);
    float pl = __fmaf_rn(a.hi, b.hi, -ph);
    pl = __fmaf_rn(a.hi, b.lo, pl);
    pl = __fmaf_rn(a.lo, b.hi, pl);
    df64 s = two_sum(c.hi, ph);
    return df64(s.hi, __fadd_rn(__fadd_rn(c.lo, s.lo), pl));
}

__device__ __forceinline__ df64 rsqrt_t(df64 x) {
    // binary32 estimate and one binary32 Newton step: y ~ x^-1/2 to ~2^-23
    float y = rsqrtf(x.hi);
    y = __fmul_rn(y, __fmaf_rn(-0.5f * x.hi, __fmul_rn(y, y), 1.5f));
    // residual e = 1 - x y^2 in double-word arithmetic, then y (1 + e/2 + 3e^2/8)
    df64 yy = two_prod(y, y);
    df64 u = x * yy;
    float e = __fsub_rn(__fsub_rn(1.0f, u.hi), u.lo);
    float corr = __fmaf_rn(__fmul_rn(0.375f, e), e, __fmul_rn(0.5f, e));
    return fast_two_sum(y, __fmul_rn(y, corr));
}

__device__ __forceinline__ df64 to_df(double d) {
    float h = __double2float_rn(d);
    return df64(h, __double2float_rn(d - (double)h));
}

__device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }
// multiplication by a power of two f: both words scale exactly (barring underflow of lo)
__device__ __forceinline__ df64 scale_t(df64 a, float f) { return df64(a.hi * f, a.lo * f); }
// a * f * c for a power of two f and a small integer c: the high word's product is split
// exactly (TwoProd), the low word's carries the usual double-word error (left unnormalised)
__device__ __forceinline__ df64 scale_c_t(df64 a, float f, float c) {
    float h = a.hi * f;
    float p = h * c;
    float e = fmaf(h, c, -p);
    return df64(p, fmaf(a.lo * f, c, e));
}

}  // namespace gbfmm
