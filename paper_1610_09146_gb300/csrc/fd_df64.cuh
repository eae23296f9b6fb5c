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

// ---- binary64 <-> double-word by integer operations ----------------------
// On GB300 every conversion instruction between binary32 and binary64 issues on
// the FP64 pipe at the rate of a DFMA (2 per SM per clock, measured), so the
// kernels that mix binary64 with double-word arithmetic move values between
// the two formats by rearranging the IEEE 754 fields with integer operations.
//
// Bit images of the two formats (binary64: sign, 11-bit exponent E biased by
// 1023, 52-bit fraction M; binary32: sign, 8-bit exponent biased by 127, 23-bit
// fraction).
__host__ __device__ __forceinline__ unsigned f32_bits(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    unsigned u;
    __builtin_memcpy(&u, &x, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float f32_of(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    __builtin_memcpy(&x, &u, 4);
    return x;
#endif
}
__host__ __device__ __forceinline__ unsigned f64_hi(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned)__double2hiint(x);
#else
    unsigned long long u;
    __builtin_memcpy(&u, &x, 8);
    return (unsigned)(u >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned f64_lo(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned)__double2loint(x);
#else
    unsigned long long u;
    __builtin_memcpy(&u, &x, 8);
    return (unsigned)u;
#endif
}
__host__ __device__ __forceinline__ double f64_of(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const unsigned long long u = ((unsigned long long)hi << 32) | lo;
    double x;
    __builtin_memcpy(&x, &u, 8);
    return x;
#endif
}
__host__ __device__ __forceinline__ float i32_to_f32(int i) {
#ifdef __CUDA_ARCH__
    return __int2float_rn(i);  // I2F: integer pipe, not FP64
#else
    return (float)i;
#endif
}

// Double-word of a binary64 value x (about 48 of its 53 significand bits):
//   hi = x rounded to 24 significand bits (half away from zero): the binary64
//        fraction's top 23 bits, incremented when the next bit is set (a carry
//        into the exponent field is the correct rounding), with the exponent
//        re-biased by 1023 - 127 = 896;
//   lo = x - hi, exactly the remaining 29 fraction bits as a signed integer
//        (negative when hi was rounded up), converted to binary32 (rounded to
//        24 bits) and scaled by 2^(E - 1075).
// |x - (hi + lo)| <= 2^-48 |x| for 2^-74 <= |x| < 2^128; below 2^-74 the trailing
// word is dropped and below 2^-126 the result is 0 (absolute error below 2^-74
// resp. 2^-126); |x| >= 2^128, infinities and NaN map to a binary32 infinity or NaN.
__host__ __device__ __forceinline__ df64 dw_of_f64(double x) {
    const unsigned hw = f64_hi(x), lw = f64_lo(x);
    const unsigned sign = hw & 0x80000000u;
    const int E = (int)((hw >> 20) & 0x7ffu);
    // (hw << 3) | (lw >> 29): exponent bits 8..0 over the top 23 fraction bits;
    // adding 128 << 23 maps E mod 512 to E - 896 for 897 <= E <= 1150
    const unsigned top = (hw << 3) | (lw >> 29);
    unsigned hb = (top + 0x40000000u + ((lw >> 28) & 1u)) | sign;
    const int rem = (int)(lw << 3) >> 3;  // the 29 trailing fraction bits, sign-extended from bit 28
    const int se = E - 948 > 0 ? E - 948 : 0;  // binary32 exponent field of 2^(E - 1075), 0 below range
    float lo = i32_to_f32(rem) * f32_of(((unsigned)se << 23) | sign);
    if (E < 897) hb = sign;
    if (E > 1150) {
        const bool nan = E == 2047 && (((hw & 0xfffffu) | lw) != 0u);
        hb = sign | (nan ? 0x7fc00000u : 0x7f800000u);
        lo = 0.0f;
    }
    return df64(f32_of(hb), lo);
}

// Exact binary64 value of a binary32 number (normal numbers, zero, infinities
// and NaN; binary32 subnormals, below 2^-126, become zero): the fraction moves
// to the top of the binary64 fraction and the exponent is re-biased by 896.
__host__ __device__ __forceinline__ double f64_of_f32(float f) {
    const unsigned b = f32_bits(f);
    const unsigned sign = b & 0x80000000u, mag = b & 0x7fffffffu;
    if (mag < 0x00800000u) return f64_of(sign, 0u);
    if (mag >= 0x7f800000u)
        return f64_of(sign | 0x7ff00000u | (mag & 0x007fffffu ? 0x00080000u : 0u), 0u);
    return f64_of(sign | ((mag >> 3) + 0x38000000u), b << 29);
}

// hi + lo of a double-word rounded to binary64 (one DADD).
__host__ __device__ __forceinline__ double f64_of_dw(df64 x) { return f64_of_f32(x.hi) + f64_of_f32(x.lo); }

// ---- unnormalised forms for long stencil sums -----------------------------
// The fused residual sums many products of stencil taps.  There the pair
// (hi, lo) need not be renormalised after every operation: what the result
// needs is an absolute error of ~2^-47 of the operands' scale, and that holds
// for unevaluated sums whose trailing word stays within a few units of the
// leading word's last place (or, after a cancellation in the leading words,
// within that of the operands).  These forms drop the renormalisation:
//   mul_nn(x, y): hi = fl(x.hi y.hi), lo = its exact error (FMA) + x.hi y.lo
//                 + x.lo y.hi; the term x.lo y.lo (below 2^-46 |x y|) is dropped
//                 (4 operations, against 10 for DWTimesDW);
//   add_nn(x, y): TwoSum of the leading words, the trailing words added to its
//                 error (8 operations, against 11 for SloppyDWPlusDW);
//   renorm(x):    the pair as a normalised double-word (TwoSum: exact for any
//                 two binary32 numbers).
__device__ __forceinline__ df64 mul_nn(df64 x, df64 y) {
    const float ph = __fmul_rn(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.hi, -ph);
    return df64(ph, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e)));
}
__device__ __forceinline__ df64 add_nn(df64 x, df64 y) {
    const df64 s = two_sum(x.hi, y.hi);
    return df64(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df64 sub_nn(df64 x, df64 y) { return add_nn(x, -y); }
// x times a binary32 y, unnormalised (DWTimesFP without its final FastTwoSum).
__device__ __forceinline__ df64 mul_nn(df64 x, float y) {
    const float ph = __fmul_rn(x.hi, y);
    return df64(ph, __fmaf_rn(x.lo, y, __fmaf_rn(x.hi, y, -ph)));
}
__device__ __forceinline__ df64 renorm(df64 x) { return two_sum(x.hi, x.lo); }

// 1 / x: the binary32 reciprocal of the leading word refined by one Newton
// step r' = r + r (1 - x r) evaluated in double-word arithmetic.
__device__ __forceinline__ df64 recip(df64 x) {
    const df64 r(__frcp_rn(x.hi), 0.0f);
    const df64 e = df64(1.0) - x * r;
    return r + r * e;
}

}  // namespace fd
