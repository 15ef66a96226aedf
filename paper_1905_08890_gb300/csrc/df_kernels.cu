// df_kernels.cu - finest-level residual and update of the mixed solve in
// double-float arithmetic (df64.cuh).
//
// The defect-correction loop needs the fine residual eps = L(u) - f to well
// below the FP32 rounding of the Laplacian, whose terms are ~|u|/h^2 while
// the result is ~f.  With u, f and the coefficients stored as hi/lo FP32
// pairs (split layout, two float arrays each), the residual is formed with
// FP32 instructions only and carries about 48 significant bits, enough for a
// relative residual far below 1e-8 at 512^3; the FP32 correction e is then
// added back exactly as a double-float.
#include "df64.cuh"
#include "gr_internal.cuh"

namespace gr {
namespace {

inline int grid_for(int64_t work)
{
    int64_t b = (work + kBlock - 1) / kBlock;
    const int64_t cap = 152 * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

inline int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Split a double into hi + lo FP32 with integer operations only (GB300's
// FP64 and conversion pipes are slow): hi keeps the sign, the exponent and the
// top 23 stored mantissa bits; lo is the remaining 29 bits converted to FP32
// (rounded to 24 bits, so hi + lo carries at least 48 significant bits) and
// scaled by 2^(e - 52).  The pair is renormalised by fast-two-sum.  Values
// whose exponent leaves FP32's normal range for lo (|x| < 2^-74) or hi
// (|x| >= 2^128) take the FP64 conversion instead.
__device__ __forceinline__ df split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023;
    if (ex < -74 || ex > 127) {
        const float h = (float)x;
        return {h, (float)(x - (double)h)};
    }
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned hib = sign | ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    const unsigned rem = (unsigned)(b & 0x1fffffffu);
    const float scale = __int_as_float((ex - 52 + 127) << 23);  // 2^(ex - 52), normal since ex >= -74
    const float mag = (float)rem * scale;
    const float lo = sign ? -mag : mag;
    return fast_two_sum(__uint_as_float(hib), lo);
}

__global__ void k_df_split(int64_t cnt, const double *__restrict__ a, float *__restrict__ hi, float *__restrict__ lo)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = a[t];
        const df d = x == 0.0 ? df{0.0f, 0.0f} : split_double(x);
        hi[t] = d.hi;
        lo[t] = d.lo;
    }
}

__global__ void k_df_join(int64_t cnt, const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ a)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        a[t] = (double)hi[t] + (double)lo[t];
}

__device__ __forceinline__ void block_sum1(double a, double *out)
{
    __shared__ double sa[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sa[w] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kBlock / 32; q++) t += sa[q];
        out[2 * blockIdx.x] = t;
        out[2 * blockIdx.x + 1] = 0.0;
    }
}

// L(u) - f at one cell from the compensated neighbour sum (Sum2 of Ogita,
// Rump and Oishi 2005: the high parts through a two-sum chain, the chain's
// errors and all low parts added in FP32, which suffices since they are
// 2^-24 smaller).  nh/nl: the six neighbours' high and low parts.
template <int KIND>
__device__ __forceinline__ df df_cell(const float *nh, const float *nl, df u, df f, df a, df b, df ih2, df two_pi,
                                      df two_pi_rho, float rho10pi, float h2, float *mj_out, float *inv_out)
{
    const df p6 = two_prod(u.hi, -6.0f);
    float s = p6.hi, sig = __fmaf_rn(u.lo, -6.0f, p6.lo);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const df q = two_sum(s, nh[k]);
        s = q.hi;
        sig = __fadd_rn(sig, __fadd_rn(q.lo, nl[k]));
    }
    df e = df_mul(fast_two_sum(s, sig), ih2);
    if (KIND == KHELM) {
        e = df_sub(e, df_mul(a, u));
    } else if (KIND == KPSI) {
        const df v = df_add({1.0f, 0.0f}, u);
        const df iv = df_recip(v);
        const df iv2 = df_mul(iv, iv), iv4 = df_mul(iv2, iv2);
        const df v2 = df_mul(v, v), v4 = df_mul(v2, v2);
        e = df_add(e, df_mul(df_mul(a, iv), two_pi));
        e = df_add(e, df_mulf(df_mul(b, df_mul(df_mul(iv4, iv2), iv)), 0.125f));
        e = df_sub(e, df_mul(df_mul(v4, v), two_pi_rho));
        const float mj = two_pi.hi * a.hi * iv2.hi + 0.875f * b.hi * (iv4.hi * iv4.hi) + rho10pi * v4.hi;
        *mj_out = mj;
        *inv_out = 1.0f / (6.0f + h2 * mj);
    }
    return df_sub(e, f);
}

// eps = L(u) - f on the finest level; writes r32 = -eps and, for the psi
// kind, the Newton coefficient m32 = -dN/du with its FP32 inverse diagonal.
// One thread per row position (i, j, q) handles the red and the black cell
// there: each needs the other colour at the same q in rows (i +- 1, j),
// (i, j +- 1) and at q, q +- 1 in its own row, so every array element is
// read once as a cell and, close in time, as its neighbours' neighbour.
// Block partials: sum of (eps / ref)^2.
template <int KIND>
__global__ void __launch_bounds__(kBlock)
    k_df_resid(int lgn, const float *__restrict__ uh, const float *__restrict__ ul, const float *__restrict__ fh,
               const float *__restrict__ fl, const float *__restrict__ ah, const float *__restrict__ al,
               const float *__restrict__ bh, const float *__restrict__ bl, df ih2, df two_pi, df two_pi_rho,
               float rho10pi, float h2, float inv_ref, float *__restrict__ r32, float *__restrict__ m32,
               float *__restrict__ inv32, double *__restrict__ partials)
{
    // Two neighbouring half-indices q0, q0 + 1 of one row per thread (float2
    // loads), both colours: four cells.  32-bit offsets: grids up to 1024^3.
    const int lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int half = 1 << (3 * lgn - 1);
    float acc = 0.0f;
    for (int tp = blockIdx.x * blockDim.x + threadIdx.x; tp < (half >> 1); tp += gridDim.x * blockDim.x) {
        const int t = tp << 1;  // even: q0 = t & mh
        const int q = t & mh;
        const int j = (t >> lgh) & mn;
        const int i = t >> (lgh + lgn);
        const int r0 = t - q;
        const int ri = j << lgh;
        const int rip = (((i + 1) & mn) << (lgn + lgh)) + ri + q;
        const int rim = (((i - 1) & mn) << (lgn + lgh)) + ri + q;
        const int rj = i << (lgn + lgh);
        const int rjp = rj + (((j + 1) & mn) << lgh) + q;
        const int rjm = rj + (((j - 1) & mn) << lgh) + q;
        const int pr = (i + j) & 1;  // k parity of the red cells in this row
        // the own-row neighbour outside the pair: q0 + 2 (shift +1) or q0 - 1 (shift -1)
        const int xp = r0 + ((q + 2) & mh), xm = r0 + ((q - 1) & mh);
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const int own = (c ? half : 0) + t;
            const int oth = c ? 0 : half;
            const int up = c ? !pr : pr;  // this colour's shift is +1 when its k parity is 1
            float2 nh[5], nl[5];
            const int rows[5] = {rip, rim, rjp, rjm, t};
#pragma unroll
            for (int k = 0; k < 5; k++) {
                nh[k] = *reinterpret_cast<const float2 *>(uh + oth + rows[k]);
                nl[k] = *reinterpret_cast<const float2 *>(ul + oth + rows[k]);
            }
            const int xi = oth + (up ? xp : xm);
            const float xh = uh[xi], xl = ul[xi];
            const float2 u2h = *reinterpret_cast<const float2 *>(uh + own);
            const float2 u2l = *reinterpret_cast<const float2 *>(ul + own);
            const float2 f2h = *reinterpret_cast<const float2 *>(fh + own);
            const float2 f2l = *reinterpret_cast<const float2 *>(fl + own);
            float2 a2h = {0.0f, 0.0f}, a2l = {0.0f, 0.0f}, b2h = {0.0f, 0.0f}, b2l = {0.0f, 0.0f};
            if (KIND != KPOISSON) {
                a2h = *reinterpret_cast<const float2 *>(ah + own);
                a2l = *reinterpret_cast<const float2 *>(al + own);
            }
            if (KIND == KPSI) {
                b2h = *reinterpret_cast<const float2 *>(bh + own);
                b2l = *reinterpret_cast<const float2 *>(bl + own);
            }
            float mj[2] = {0.0f, 0.0f}, iv[2] = {0.0f, 0.0f};
            float rr[2];
#pragma unroll
            for (int e = 0; e < 2; e++) {
                float h6[6], l6[6];
#pragma unroll
                for (int k = 0; k < 5; k++) {
                    h6[k] = e ? nh[k].y : nh[k].x;
                    l6[k] = e ? nl[k].y : nl[k].x;
                }
                // shifted neighbour of cell q0 + e in the other colour's own row
                if (up) {
                    h6[5] = e ? xh : nh[4].y;
                    l6[5] = e ? xl : nl[4].y;
                } else {
                    h6[5] = e ? nh[4].x : xh;
                    l6[5] = e ? nl[4].x : xl;
                }
                const df u = {e ? u2h.y : u2h.x, e ? u2l.y : u2l.x};
                const df f = {e ? f2h.y : f2h.x, e ? f2l.y : f2l.x};
                const df a = {e ? a2h.y : a2h.x, e ? a2l.y : a2l.x};
                const df b = {e ? b2h.y : b2h.x, e ? b2l.y : b2l.x};
                const df r = df_cell<KIND>(h6, l6, u, f, a, b, ih2, two_pi, two_pi_rho, rho10pi, h2, &mj[e], &iv[e]);
                rr[e] = -(r.hi + r.lo);
                const float z = r.hi * inv_ref;
                acc = __fmaf_rn(z, z, acc);
            }
            *reinterpret_cast<float2 *>(r32 + own) = make_float2(rr[0], rr[1]);
            if (KIND == KPSI) {
                *reinterpret_cast<float2 *>(m32 + own) = make_float2(mj[0], mj[1]);
                *reinterpret_cast<float2 *>(inv32 + own) = make_float2(iv[0], iv[1]);
            }
        }
    }
    block_sum1((double)acc, partials);
}

// u (double-float) += e
__global__ void k_df_update(int64_t cnt, float *__restrict__ uh, float *__restrict__ ul, const float *__restrict__ e)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        df s = two_sum(uh[t], e[t]);
        s.lo = __fadd_rn(s.lo, ul[t]);
        s = fast_two_sum(s.hi, s.lo);
        uh[t] = s.hi;
        ul[t] = s.lo;
    }
}

}  // namespace

void df_split(int64_t cnt, const double *a, float *hi, float *lo, cudaStream_t st)
{
    GR_LAUNCH(k_df_split, grid_for(cnt), kBlock, st, cnt, a, hi, lo);
}

void df_join(int64_t cnt, const float *hi, const float *lo, double *a, cudaStream_t st)
{
    GR_LAUNCH(k_df_join, grid_for(cnt), kBlock, st, cnt, hi, lo, a);
}

int df_resid(int kind, int n, const float *uh, const float *ul, const float *fh, const float *fl, const float *ah,
             const float *al, const float *bh, const float *bl, double ih2, double rho, double h2, double ref,
             float *r32, float *m32, float *inv32, double *partials, cudaStream_t st)
{
    const int lgn = log2i(n);
    int g = grid_for((int64_t)n * n * n / 4);
    if (g > kMaxRedBlocks) g = kMaxRedBlocks;
    const df dih2 = df_from_double_host(ih2), d2pi = df_from_double_host(2.0 * kPi),
             d2pr = df_from_double_host(2.0 * kPi * rho);
    const float r10 = (float)(10.0 * kPi * rho), fh2 = (float)h2, iref = (float)(1.0 / ref);
    if (kind == KPOISSON)
        GR_LAUNCH(k_df_resid<KPOISSON>, g, kBlock, st, lgn, uh, ul, fh, fl, ah, al, bh, bl, dih2, d2pi, d2pr, r10,
                  fh2, iref, r32, m32, inv32, partials);
    else if (kind == KHELM)
        GR_LAUNCH(k_df_resid<KHELM>, g, kBlock, st, lgn, uh, ul, fh, fl, ah, al, bh, bl, dih2, d2pi, d2pr, r10, fh2,
                  iref, r32, m32, inv32, partials);
    else
        GR_LAUNCH(k_df_resid<KPSI>, g, kBlock, st, lgn, uh, ul, fh, fl, ah, al, bh, bl, dih2, d2pi, d2pr, r10, fh2,
                  iref, r32, m32, inv32, partials);
    return g;
}

void df_update(int n, float *uh, float *ul, const float *e, cudaStream_t st)
{
    const int64_t cnt = (int64_t)n * n * n;
    GR_LAUNCH(k_df_update, grid_for(cnt), kBlock, st, cnt, uh, ul, e);
}

}  // namespace gr
