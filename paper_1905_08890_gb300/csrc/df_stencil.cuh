// df_stencil.cuh - the finest-level operator in double-float arithmetic,
// shared by the base residual kernels and the nested patches' relaxation.
#pragma once

#include "df64.cuh"
#include "gr_internal.cuh"

namespace gr {

// h^2 (L(u) - f) at one cell from the compensated sum of the seven stencil
// terms and -h^2 f (Sum2 of Ogita, Rump and Oishi 2005: the high parts
// through a two-sum chain, the chain's errors and all low parts added in
// FP32, which suffices since they are 2^-24 smaller).  The right-hand side and
// the coefficients arrive premultiplied by h^2 (f' = h^2 f; KHELM a' = h^2 m;
// KPSI a' = 2 pi h^2 s0, b' = h^2 AA / 8, cpr = 2 pi rho h^2), so no
// double-float scaling by 1/h^2 is needed; nh/nl are the six neighbours'
// high and low parts.  KPSI also returns h^2 times the Newton coefficient and
// 1/(6 + h^2 m).
template <int KIND>
__device__ __forceinline__ df df_cell(const float *nh, const float *nl, df u, df f, df a, df b, df cpr, float c5,
                                      float *mj_out, float *inv_out)
{
    const df p6 = two_prod(u.hi, -6.0f);
    float s = p6.hi, sig = __fmaf_rn(u.lo, -6.0f, p6.lo);
    {
        const df q = two_sum(s, -f.hi);
        s = q.hi;
        sig = __fadd_rn(sig, __fsub_rn(q.lo, f.lo));
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const df q = two_sum(s, nh[k]);
        s = q.hi;
        sig = __fadd_rn(sig, __fadd_rn(q.lo, nl[k]));
    }
    df e = fast_two_sum(s, sig);
    if (KIND == KHELM) {
        e = df_sub(e, df_mul(a, u));
    } else if (KIND == KPSI) {
        const df v = df_add({1.0f, 0.0f}, u);
        const df iv = df_recip(v);
        const df iv2 = df_mul(iv, iv), iv4 = df_mul(iv2, iv2);
        const df v2 = df_mul(v, v), v4 = df_mul(v2, v2);
        e = df_add(e, df_mul(a, iv));
        e = df_add(e, df_mul(b, df_mul(df_mul(iv4, iv2), iv)));
        e = df_sub(e, df_mul(df_mul(v4, v), cpr));
        const float mjh2 = a.hi * iv2.hi + 7.0f * b.hi * (iv4.hi * iv4.hi) + c5 * v4.hi;
        *mj_out = mjh2;
        *inv_out = 1.0f / (6.0f + mjh2);
    }
    return e;
}


// (hi, lo) + e, renormalised
__device__ __forceinline__ df df_plus_f(float hi, float lo, float e)
{
    df s = two_sum(hi, e);
    s.lo = __fadd_rn(s.lo, lo);
    return fast_two_sum(s.hi, s.lo);
}

}  // namespace gr
