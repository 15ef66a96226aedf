// df64.cuh - double-float arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2 (48-bit significand, FP32 exponent
// range).  Built from the error-free transformations
//   two-sum      (Knuth, TAOCP vol. 2, 4.2.2): a + b = s + e exactly,
//   fast-two-sum (Dekker 1971), valid for |a| >= |b|,
//   two-product  (Dekker 1971; here with a fused multiply-add): a * b = p + e exactly,
// and Newton's iteration for the reciprocal.  GB300 issues FP32 at 58x its
// FP64 rate, so these sequences of FP32 operations are much cheaper than FP64.
// The _rn intrinsics keep the compiler from contracting or reassociating the
// error terms.
#pragma once

#include <cuda_runtime.h>

namespace gr {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// a + b with both low parts folded in after the exact high-part sum
// (absolute error about 2^-44 (|a| + |b|)): for terms of unequal size
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}

// a + b with exact sums of the high and of the low parts (absolute error
// about 2^-48 (|a| + |b|)): for sums that cancel, such as a stencil
__device__ __forceinline__ df df_add_acc(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b)
{
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mulf(df a, float b)
{
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// 1/a: FP32 estimate refined by one Newton step r + r (1 - a r) in double-float
__device__ __forceinline__ df df_recip(df a)
{
    const float r = 1.0f / a.hi;
    const df ar = df_mulf(a, r);
    const df e = df_add({1.0f, 0.0f}, df_neg(ar));
    const df c = two_prod(e.hi, r);
    return fast_two_sum(r, __fadd_rn(c.hi, __fmaf_rn(e.lo, r, c.lo)));
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// host-side split of a double constant into a double-float
inline df df_from_double_host(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

}  // namespace gr
