// ffloat.cuh -- float-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On this GPU FP64 instructions issue at 1/57 of
// the FP32 rate with a 68-cycle latency, so reductions and scalar bookkeeping
// run in float-float and touch FP64 only once per reduction.  The error-free
// transformations are the classical ones (Knuth's two-sum, Dekker's
// fast-two-sum, the FMA-based two-product); the _rn intrinsics keep the
// compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

namespace cmg {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) {
    ff r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

__device__ __forceinline__ ff ff_zero() { return ff_make(0.f, 0.f); }

// Knuth two-sum: s + e == a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff_make(s, e);
}

// Dekker fast-two-sum (requires |a| >= |b| or a == 0).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff_make(s, e);
}

// p + e == a * b exactly (FMA-based).
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return ff_make(p, e);
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = two_sum(a.hi, b);
    const float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}

// Sum without the final renormalisation (hi + lo is still exact up to the
// rounding of the lo additions); renormalise with ff_norm when done.
__device__ __forceinline__ ff ff_add_lazy(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return ff_make(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_norm(ff a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const ff p = two_prod(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    const ff p = two_prod(a.hi, b);
    const float e = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

// a < b for normalised values.
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// Split a double into float-float with integer operations only (no FP64
// instruction): hi takes the leading 24 significant bits (truncated), lo the
// next bits rounded to a float.  Values outside the float exponent range, and
// lo parts below it, are dropped (returned as 0), which is far below the
// resolution the callers need.
__device__ __forceinline__ ff ff_from_double(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int E = (int)((b >> 52) & 0x7FFull);
    const int fe = E - 1023 + 127;
    if (fe <= 0 || fe >= 255) return ff_zero();
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    const float hi = __int_as_float((int)(sign | ((unsigned int)fe << 23) | (unsigned int)(mant >> 29)));
    // remainder: low 29 mantissa bits, worth rem * 2^(E - 1075)
    const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFull);
    const int se = E - 1075 + 127;   // float exponent of 2^(E - 1075)
    float lo = 0.f;
    if (se >= 1 && rem != 0u) {
        lo = __fmul_rn(__uint2float_rn(rem), __int_as_float(se << 23));
        if (sign) lo = -lo;
    }
    return fast_two_sum(hi, lo);
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff shfl_xor_ff(ff a, int o) {
    return ff_make(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
}

// Warp sum (xor tree, fixed order); every lane receives the sum.
__device__ __forceinline__ ff warp_sum_ff(ff a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = ff_add(a, shfl_xor_ff(a, o));
    return a;
}

}  // namespace cmg
