// Double-single arithmetic shared by the kernels that emulate wide
// precision on the FP32 pipes (the mixed path's diagonal blocks, scaling and
// Gram blocks; the a-posteriori error estimate).
#pragma once

#include <stdint.h>

namespace ccov {

// Double-single arithmetic: a value is an unevaluated sum hi + lo of two
// floats (about 44 significant bits; Dekker 1971, with the products split
// by FMA).  GB300 issues FP32 about eighty times faster than FP64 per SM,
// and the digits that the tensor-core products keep of L and L^-1 hold 39
// bits, so the one-CTA factorisation of a diagonal block runs in this form.
// Explicit _rn intrinsics keep the compiler from contracting the
// error-free transformations.
struct dsf {
    float h, l;
};

// acc + a * b
__device__ __forceinline__ dsf ds_fma(dsf acc, dsf a, dsf b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float s = __fadd_rn(acc.h, p);
    const float v = __fsub_rn(s, acc.h);
    float t = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, v)), __fsub_rn(p, v));
    t = __fadd_rn(t, __fadd_rn(acc.l, e));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ dsf ds_neg(dsf a) { return {-a.h, -a.l}; }

// a + b (two-sum of the high parts, low parts added, then renormalised)
__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
    const float s = __fadd_rn(a.h, b.h);
    const float v = __fsub_rn(s, a.h);
    float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
    t = __fadd_rn(t, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

// Q60 fixed point <-> double-single, with integer conversions only: v =
// f + r exactly with f = v rounded to a float (an integer value) and r the
// remainder (|r| <= 2^39); the power-of-two scalings are exact in float.
__device__ __forceinline__ dsf ds_from_fixed(long long v, float scale) {
    const float f = __ll2float_rn(v);
    const long long r = v - __float2ll_rz(f);
    return {__fmul_rn(f, scale), __fmul_rn(__ll2float_rn(r), scale)};
}

__device__ __forceinline__ dsf ds_mul(dsf a, dsf b) { return ds_fma({0.f, 0.f}, a, b); }

// A double as an unevaluated sum of two floats without FP64 arithmetic:
// the high float keeps the top 24 significand bits (truncated), the low one
// the other 29 bits (rounded to 24), so hi + lo equals z to 2^-48 relative.
// Below 2^-74 only the high float is kept and below 2^-126 the value becomes
// 0: against entries of Z_s of order 1 such terms are far below the 39-bit
// digits taken from it.
__device__ __forceinline__ dsf ds_from_double(double z) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(z);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int E = (int)((b >> 52) & 0x7FF) - 1023;
    if (E < -126) return {0.f, 0.f};
    if (E > 127) return {__uint_as_float(sign | 0x7F800000u), 0.f};   // beyond float range (or not finite)
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;                // 52 fraction bits
    const float hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29));
    const int es = E - 52 + 127;                                         // exponent field of 2^(E - 52)
    float lo = 0.f;
    if (es >= 1) lo = __fmul_rn(__uint2float_rn((unsigned)(m & 0x1FFFFFFFu)), __uint_as_float((unsigned)es << 23));
    return {hi, sign ? -lo : lo};
}

}  // namespace ccov
