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
// (absolute error about 2^-47 (|a| + |b|), not relative to a + b)
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

// The FP64 versions of the split and the join, for the rare operands outside
// the integer paths' range.  Not inlined: as inline code the compiler may
// predicate them into the common path, where their FP64 conversions would
// occupy GB300's narrow FP64 pipe on every element.
static __device__ __noinline__ df split_double_fp64(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

static __device__ __noinline__ double join_double_fp64(df v) { return (double)v.hi + (double)v.lo; }

// Split a double into hi + lo FP32 with integer operations only (GB300's
// FP64 and conversion pipes are slow): hi keeps the sign, the exponent and the
// top 23 stored mantissa bits; lo is the remaining 29 bits converted to FP32
// (rounded to 24 bits, so hi + lo carries at least 48 significant bits) and
// scaled by 2^(e - 52).  The pair is renormalised by fast-two-sum.  Values
// whose exponent leaves FP32's normal range for lo (|x| < 2^-74) or hi
// (|x| >= 2^128) take the FP64 conversion instead; zeros keep their sign.
__device__ __forceinline__ df split_double(double x)
{
    // on the two 32-bit halves of x: hi32 = sign | exponent (11) | mantissa bits 51..32
    const unsigned hi32 = (unsigned)__double2hiint(x), lo32 = (unsigned)__double2loint(x);
    if (((hi32 << 1) | lo32) == 0u) return {__uint_as_float(hi32), 0.0f};  // +-0
    const int ex = (int)((hi32 >> 20) & 0x7ffu) - 1023;
    if ((unsigned)(ex + 74) > 201u) return split_double_fp64(x);  // ex < -74 or ex > 127
    const unsigned sign = hi32 & 0x80000000u;
    // top 23 stored mantissa bits: 20 from hi32, 3 from lo32
    const unsigned hib = sign | ((unsigned)(ex + 127) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
    const unsigned rem = lo32 & 0x1fffffffu;
    const float scale = __int_as_float((ex - 52 + 127) << 23);  // 2^(ex - 52), normal since ex >= -74
    const float lo = __uint_as_float(__float_as_uint((float)rem * scale) | sign);
    return fast_two_sum(__uint_as_float(hib), lo);
}

// hi + lo rounded to the nearest double (ties to even), with 32-bit integer
// operations only: lo, which lies below one unit in the last place of hi, is
// rounded to a whole number of units in the last place of double(hi) (at
// most 2^29 of them) and added to or subtracted from double(hi)'s bit
// pattern; the sum cannot leave hi's binade except upwards onto the next
// power of two, which the bit pattern carries correctly.  Needs |lo| < ulp(hi)
// (a renormalised pair) and a normal, finite hi; a power-of-two hi with lo
// of the other sign (the sum would drop a binade) and anything else take the
// FP64 sum.
__device__ __forceinline__ double join_double(df v)
{
    const unsigned bh = __float_as_uint(v.hi), bl = __float_as_uint(v.lo);
    const int e1 = (int)((bh >> 23) & 0xffu), e2 = (int)((bl >> 23) & 0xffu);
    const unsigned mh = bh & 0x7fffffu;
    const int d = e1 - (e2 ? e2 : 1);  // lo < 2^(24 - d) ulp(hi)
    const bool opp = ((bh ^ bl) >> 31) != 0u && (bl << 1) != 0u;
    if (e1 == 0 || e1 == 255 || e2 == 255 || d < 24 || (opp && mh == 0u)) return join_double_fp64(v);
    // double(hi): exponent e1 - 127 + 1023, stored mantissa mh << 29
    const unsigned long long P = ((unsigned long long)((bh & 0x80000000u) | ((unsigned)(e1 + 896) << 20) | (mh >> 3))
                                  << 32) |
                                 (unsigned long long)(mh << 29);
    // lo = m2 2^(29 - d) units of ulp(double(hi))
    const unsigned m2 = (bl & 0x7fffffu) | (e2 ? 0x800000u : 0u);
    const int sh = d - 29;
    unsigned r;
    if (sh <= 0) {
        r = m2 << (-sh);
    } else if (sh >= 25) {
        r = 0u;
    } else {
        const unsigned fm = m2 >> sh, rem = m2 & ((1u << sh) - 1u), half = 1u << (sh - 1);
        r = fm + ((rem > half || (rem == half && (fm & 1u))) ? 1u : 0u);
    }
    return __longlong_as_double((long long)(opp ? P - r : P + r));
}

// host-side split of a double constant into a double-float
inline df df_from_double_host(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

}  // namespace gr
