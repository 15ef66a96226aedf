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

__global__ void k_df_split(int64_t cnt, const double *__restrict__ a, float *__restrict__ hi, float *__restrict__ lo)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = a[t];
        const float h = (float)x;
        hi[t] = h;
        lo[t] = (float)(x - (double)h);
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

// eps = L(u) - f on every cell of the finest level; writes r32 = -eps and,
// for the psi kind, the Newton coefficient m32 = -dN/du and 1/(6 + h^2 m32).
// Block partials: sum of (eps / ref)^2.
template <int KIND>
__global__ void __launch_bounds__(kBlock)
    k_df_resid(int lgn, const float *__restrict__ uh, const float *__restrict__ ul, const float *__restrict__ fh,
               const float *__restrict__ fl, const float *__restrict__ ah, const float *__restrict__ al,
               const float *__restrict__ bh, const float *__restrict__ bl, df ih2, df two_pi, df two_pi_rho,
               float rho10pi, float h2, float inv_ref, float *__restrict__ r32, float *__restrict__ m32,
               float *__restrict__ inv32, double *__restrict__ partials)
{
    const int lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int64_t half = (int64_t)1 << (3 * lgn - 1);
    const int64_t cnt = 2 * half;
    float acc = 0.0f;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int color = (int)(t >> (3 * lgn - 1));
        const int64_t tt = t - (color ? half : 0);
        const int64_t o = color ? 0 : half;  // start of the other colour
        const int q = (int)(tt & mh);
        const int j = (int)((tt >> lgh) & mn);
        const int i = (int)(tt >> (lgh + lgn));
        const int p = (i + j + color) & 1;
        const int64_t r0 = o + tt - q;
        const int64_t ri = (int64_t)j << lgh;
        const int64_t rip = o + ((int64_t)((i + 1) & mn) << (lgn + lgh)) + ri;
        const int64_t rim = o + ((int64_t)((i - 1) & mn) << (lgn + lgh)) + ri;
        const int64_t rj = o + ((int64_t)i << (lgn + lgh));
        const int64_t rjp = rj + ((int64_t)((j + 1) & mn) << lgh);
        const int64_t rjm = rj + ((int64_t)((j - 1) & mn) << lgh);
        const int qs = (q + (p ? 1 : -1)) & mh;
        // sum of the six neighbours minus 6 u by compensated summation
        // (Ogita, Rump and Oishi 2005, Sum2): the high parts go through a
        // two-sum chain, the chain's errors and all low parts are added in
        // FP32, which is exact enough since they are 2^-24 smaller
        const int64_t nbi[6] = {rip + q, rim + q, rjp + q, rjm + q, r0 + q, r0 + qs};
        const df u = {uh[t], ul[t]};
        const df p6 = two_prod(u.hi, -6.0f);
        float s = p6.hi, sig = __fmaf_rn(u.lo, -6.0f, p6.lo);
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const df a = two_sum(s, uh[nbi[k]]);
            s = a.hi;
            sig = __fadd_rn(sig, __fadd_rn(a.lo, ul[nbi[k]]));
        }
        df e = df_mul(fast_two_sum(s, sig), ih2);
        if (KIND == KHELM) {
            e = df_sub(e, df_mul(df{ah[t], al[t]}, u));
        } else if (KIND == KPSI) {
            const df s0 = {ah[t], al[t]}, aa = {bh[t], bl[t]};
            const df v = df_add({1.0f, 0.0f}, u);
            const df iv = df_recip(v);
            const df iv2 = df_mul(iv, iv), iv4 = df_mul(iv2, iv2);
            const df v2 = df_mul(v, v), v4 = df_mul(v2, v2);
            e = df_add(e, df_mul(df_mul(s0, iv), two_pi));
            e = df_add(e, df_mulf(df_mul(aa, df_mul(df_mul(iv4, iv2), iv)), 0.125f));
            e = df_sub(e, df_mul(df_mul(v4, v), two_pi_rho));
            const float mj = two_pi.hi * s0.hi * iv2.hi + 0.875f * aa.hi * (iv4.hi * iv4.hi) + rho10pi * v4.hi;
            m32[t] = mj;
            inv32[t] = 1.0f / (6.0f + h2 * mj);
        }
        e = df_sub(e, df{fh[t], fl[t]});
        r32[t] = -(e.hi + e.lo);
        const float z = e.hi * inv_ref;
        acc = __fmaf_rn(z, z, acc);
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
    int g = grid_for((int64_t)n * n * n);
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
