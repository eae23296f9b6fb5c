// fd_df64.cuh -- double-word ("double-float") arithmetic on the binary32 pipe.
//
// A value is the unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi)/2, giving about 48 significant bits.  The building blocks are
// the error-free transformations
//   TwoSum      (Knuth 1969):  s + e = a + b exactly, any a, b;
//   FastTwoSum  (Dekker 1971): s + e = a + b exactly, |a| >= |b|;
//   TwoProd     (with FMA):    p + e = a * b exactly;
// and double-word algorithms analysed by Joldes, Muller and Popescu, "Tight
// and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 44, 2017):
//   sums      SloppyDWPlusDW: error below about 2u^2 (|x| + |y|), u = 2^-24,
//             the size of the operands' own 48-bit representation error, which
//             is what the stencil differences need (the accurate variant also
//             bounds the error relative to a cancelled result, at twice the cost);
//   products  DWTimesDW with FMA (relative error below 5u^2), DWTimesFP with
//             FMA for a binary32 factor, and exact scaling by powers of two.
//
// Every step must be evaluated exactly as written: the library is compiled
// with -fmad=false and without fast-math, so no multiply-add is contracted and
// no sum is re-associated.
#pragma once

#include <cuda_runtime.h>

namespace fd {

struct df64 {
    float hi, lo;
    df64() = default;
    // Split of a binary64 constant: exact for the 48 leading bits.  Evaluated at
    // compile time for literals; on the host for run-time constants.
    __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr double to_double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float v = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return df64(s, e);
}

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df64(s, e);
}

// SloppyDWPlusDW
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
    df64 s = two_sum(x.hi, y.hi);
    float v = __fadd_rn(x.lo, y.lo);
    float w = __fadd_rn(s.lo, v);
    return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }
__device__ __forceinline__ df64& operator+=(df64& x, df64 y) { return x = x + y; }

// DWTimesDW with FMA
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
    float ch = __fmul_rn(x.hi, y.hi);
    float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(cl1, cl2);
    return fast_two_sum(ch, cl3);
}

// DWTimesFP with FMA
__device__ __forceinline__ df64 times_fp(df64 x, float y) {
    float ch = __fmul_rn(x.hi, y);
    float cl1 = __fmaf_rn(x.hi, y, -ch);
    float cl3 = __fmaf_rn(x.lo, y, cl1);
    return fast_two_sum(ch, cl3);
}

// x * p for a power of two p: exact, word by word.
__device__ __forceinline__ df64 scale2(df64 x, float p) { return df64(__fmul_rn(x.hi, p), __fmul_rn(x.lo, p)); }

__device__ __forceinline__ bool operator!=(df64 x, df64 y) { return x.hi != y.hi || x.lo != y.lo; }

// a * b + c (a product then a sum; not a fused operation).
__device__ __forceinline__ df64 fmx(df64 a, df64 b, df64 c) { return a * b + c; }

// 1 / x: the binary32 reciprocal of the leading word refined by one Newton
// step r' = r + r (1 - x r) evaluated in double-word arithmetic.
__device__ __forceinline__ df64 recip(df64 x) {
    const df64 r(__frcp_rn(x.hi), 0.0f);
    const df64 e = df64(1.0) - x * r;
    return r + r * e;
}

}  // namespace fd
