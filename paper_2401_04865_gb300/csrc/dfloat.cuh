// dfloat.cuh -- double-float arithmetic on the FP32 pipes.
//
// A value is carried as an unevaluated sum hi + lo of two floats (about 48
// significant bits).  The error-free transformations are Knuth's two-sum,
// Dekker's fast two-sum (|a| >= |b|) and the two-product with a fused
// multiply-add; round-to-nearest intrinsics keep the compiler from contracting
// or reassociating them.  GB300 runs FP64 at a small fraction of its FP32 rate,
// so kernels whose FP64 work is arithmetic rather than memory traffic use these
// instead (the FP64 mesh transforms, the direct intra-body pair sums).
#pragma once

#include <cuda_runtime.h>

namespace ibp {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// Sum with one two-sum on the high parts: its error is bounded relative to
// |a| + |b| (not to |a + b|), which is what sums of same-signed or normwise-
// bounded terms need.
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_half(df a) { return {a.hi * 0.5f, a.lo * 0.5f}; }   // exact

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// b a for a float a: the exact product of a and b.hi plus a b.lo.
__device__ __forceinline__ df df_mul_f(df b, float a) {
    const float p = __fmul_rn(a, b.hi);
    float e = __fmaf_rn(a, b.hi, -p);
    e = __fmaf_rn(a, b.lo, e);
    return fast_two_sum(p, e);
}

// Sum over the warp (every lane receives it).
__device__ __forceinline__ df df_warp_sum(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const df w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    return v;
}

__device__ __forceinline__ df df_sqr(df a) {
    const float p = __fmul_rn(a.hi, a.hi);
    float e = __fmaf_rn(a.hi, a.hi, -p);
    e = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, e);
    return fast_two_sum(p, e);
}

// One Newton step from the correctly rounded FP32 root: s + (a - s^2) / (2 s).
__device__ __forceinline__ df df_sqrt(df a) {
    if (a.hi <= 0.0f) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s, s);
    const float e = __fmaf_rn(s, s, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
    return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

// a / b with one correction of the FP32 quotient.
__device__ __forceinline__ df df_div(df a, df b) {
    const float q = __fdiv_rn(a.hi, b.hi);
    const df qb = df_mul({q, 0.0f}, b);
    const df r = df_sub(a, qb);
    return fast_two_sum(q, __fdiv_rn(r.hi, b.hi));
}

__device__ __forceinline__ df df_from_double(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// Conversions with integer operations on the bits instead of FP64 conversions
// (GB300 issues those at its FP64 rate).
//
// df_split: hi = v with its significand cut to 24 bits, lo = the remaining 29
// significand bits rounded to FP32, so hi + lo = v to a relative 2^-47.  Zero
// gives (0, 0); exponents outside [-74, 127] (FP32 could not hold lo or hi) take
// df_from_double.
__device__ __forceinline__ df df_split(double v) {
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    if (((hw & 0x7FFFFFFFu) | lw) == 0u) return {0.0f, 0.0f};
    const int e = (int)((hw >> 20) & 0x7FFu) - 1023;
    if (e < -74 || e > 127) return df_from_double(v);
    const unsigned sign = hw & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);   // 2^(e - 52)
    const float lo = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), scale);
    return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

// The double with the value of f (exact): sign, exponent and significand moved
// into place; subnormal and non-finite f take the FP64 conversion.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    const unsigned ef = (u >> 23) & 0xFFu;
    if (ef == 0u || ef == 0xFFu) return (double)f;
    const unsigned hw = (u & 0x80000000u) | ((ef - 127u + 1023u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hw, (int)((u & 0x7u) << 29));
}

// hi + lo in FP64 with one FP64 addition
__device__ __forceinline__ double df_join(df a) { return widen(a.hi) + widen(a.lo); }

}  // namespace ibp
