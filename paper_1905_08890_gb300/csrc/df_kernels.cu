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
#include "df_stencil.cuh"

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

// W consecutive floats (W = 2 or 4) as one vector access
template <int W>
__device__ __forceinline__ void ldv(const float *p, float (&v)[W])
{
    if (W == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x, v[1] = t.y;
    }
}

template <int W>
__device__ __forceinline__ void stv(float *p, const float (&v)[W])
{
    if (W == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

// blocks per SM the residual kernel is compiled for (registers per thread)
template <int KIND, int W>
constexpr int resid_min_blocks()
{
    return W == 4 ? (KIND == KPSI ? 2 : 3) : (KIND == KPOISSON ? 5 : (KIND == KHELM ? 4 : 3));
}

// eps = L(u) - f on the finest level; writes r32 = -eps and, for the psi
// kind, the Newton coefficient m32 = -dN/du with its FP32 inverse diagonal.
// One thread per chunk of W consecutive half-indices q0 .. q0 + W - 1 of a row
// (i, j) handles the red and the black cells there (2W cells): each needs the
// other colour at the same half-indices in rows (i +- 1, j), (i, j +- 1) and
// at q, q +- 1 in its own row, which are W-wide vector loads plus one scalar
// for the own-row neighbour outside the chunk.  W = 4 (n >= 8) gives each
// thread enough independent loads to keep HBM busy; W = 2 serves n = 4.
// f, a, b: the h^2-premultiplied pairs of df_cell.  32-bit offsets: grids up
// to 1024^3.  Also the first red relaxation of the FP32 correction cycle,
// which starts from e = 0: e_red = -h^2 r / 6 (Poisson) or -h^2 r / (6 + h^2 m).
// SHIFT (Poisson with nested patches): every cell's right-hand side is
// f + fshift[0] (the solvability constant), i.e. h^2 f + fshift[0] * fsh_scale.
template <int KIND, int W, bool SHIFT = false>
__global__ void __launch_bounds__(kBlock, (resid_min_blocks<KIND, W>()))
    k_df_resid(int lgn, const float *__restrict__ uh, const float *__restrict__ ul, const float *__restrict__ fh,
               const float *__restrict__ fl, const float *__restrict__ ah, const float *__restrict__ al,
               const float *__restrict__ bh, const float *__restrict__ bl, df cpr, float c5, float ih2,
               float ih2_ref, float *__restrict__ r32, float *__restrict__ m32, float *__restrict__ inv32,
               const float *__restrict__ inv_in, float *__restrict__ e32, double *__restrict__ partials, int rev,
               const double *__restrict__ fshift, double fsh_scale)
{
    pdl_begin();
    const int lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int half = 1 << (3 * lgn - 1);
    float acc = 0.0f;
    df fs = {0.0f, 0.0f};
    if (SHIFT) fs = split_double(fshift[0] * fsh_scale);
    for (int tp = blockIdx.x * blockDim.x + threadIdx.x; tp < half / W; tp += gridDim.x * blockDim.x) {
        const int t = (rev ? half / W - 1 - tp : tp) * W;  // q0 = t & mh, a multiple of W
        const int q = t & mh;
        const int j = (t >> lgh) & mn;
        const int i = t >> (lgh + lgn);
        const int r0 = t - q;
        const int ri = j << lgh;
        const int rj = i << (lgn + lgh);
        const int rows[5] = {(((i + 1) & mn) << (lgn + lgh)) + ri + q, (((i - 1) & mn) << (lgn + lgh)) + ri + q,
                             rj + (((j + 1) & mn) << lgh) + q, rj + (((j - 1) & mn) << lgh) + q, t};
        const int pr = (i + j) & 1;  // k parity of the red cells in this row
        // the own-row neighbour outside the chunk: q0 + W (shift +1) or q0 - 1 (shift -1)
        const int xp = r0 + ((q + W) & mh), xm = r0 + ((q - 1) & mh);
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const int own = (c ? half : 0) + t;
            const int oth = c ? 0 : half;
            const int up = c ? !pr : pr;  // this colour's shift is +1 when its k parity is 1
            float nh[5][W], nl[5][W];
#pragma unroll
            for (int k = 0; k < 5; k++) {
                ldv<W>(uh + oth + rows[k], nh[k]);
                ldv<W>(ul + oth + rows[k], nl[k]);
            }
            const int xi = oth + (up ? xp : xm);
            const float xh = uh[xi], xl = ul[xi];
            float u_h[W], u_l[W], f_h[W], f_l[W], a_h[W] = {}, a_l[W] = {}, b_h[W] = {}, b_l[W] = {};
            ldv<W>(uh + own, u_h);
            ldv<W>(ul + own, u_l);
            ldv<W>(fh + own, f_h);
            ldv<W>(fl + own, f_l);
            if (KIND != KPOISSON) {
                ldv<W>(ah + own, a_h);
                ldv<W>(al + own, a_l);
            }
            if (KIND == KPSI) {
                ldv<W>(bh + own, b_h);
                ldv<W>(bl + own, b_l);
            }
            float mj[W] = {}, iv[W] = {}, rr[W], sh[W];
#pragma unroll
            for (int e = 0; e < W; e++) {
                float h6[6], l6[6];
#pragma unroll
                for (int k = 0; k < 5; k++) {
                    h6[k] = nh[k][e];
                    l6[k] = nl[k][e];
                }
                // shifted neighbour of cell q0 + e in the other colour's own row
                if (up) {
                    h6[5] = e == W - 1 ? xh : nh[4][e + 1 < W ? e + 1 : 0];
                    l6[5] = e == W - 1 ? xl : nl[4][e + 1 < W ? e + 1 : 0];
                } else {
                    h6[5] = e == 0 ? xh : nh[4][e > 0 ? e - 1 : 0];
                    l6[5] = e == 0 ? xl : nl[4][e > 0 ? e - 1 : 0];
                }
                const df fe = SHIFT ? df_add({f_h[e], f_l[e]}, fs) : df{f_h[e], f_l[e]};
                const df r = df_cell<KIND>(h6, l6, {u_h[e], u_l[e]}, fe, {a_h[e], a_l[e]}, {b_h[e], b_l[e]}, cpr,
                                           c5, &mj[e], &iv[e]);  // h^2 eps
                sh[e] = r.hi + r.lo;
                rr[e] = -sh[e] * ih2;
                const float z = r.hi * ih2_ref;
                acc = __fmaf_rn(z, z, acc);
            }
            stv<W>(r32 + own, rr);
            if (KIND == KPSI) {
#pragma unroll
                for (int e = 0; e < W; e++) mj[e] *= ih2;
                stv<W>(m32 + own, mj);
                stv<W>(inv32 + own, iv);
            }
            if (c == 0 && e32) {
                float g[W];
                if (KIND == KHELM) {
                    ldv<W>(inv_in + own, g);
                } else {
#pragma unroll
                    for (int e = 0; e < W; e++) g[e] = KIND == KPOISSON ? 1.0f / 6.0f : iv[e];
                }
#pragma unroll
                for (int e = 0; e < W; e++) g[e] *= sh[e];
                stv<W>(e32 + own, g);
            }
        }
    }
    block_sum2f(acc, 0.0f, partials);
}


// u (double-float) += e
__global__ void k_df_update(int64_t cnt, float *__restrict__ uh, float *__restrict__ ul, const float *__restrict__ e)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const df s = df_plus_f(uh[t], ul[t], e[t]);
        uh[t] = s.hi;
        ul[t] = s.lo;
    }
}

// The last (black) relaxation pass of the FP32 correction cycle fused with the
// update u += e of both colours: the black corrections are formed as in a
// colour pass and added to u straight away, the red ones (this pass's
// neighbours, read anyway) likewise, so e's black half is never written.
// Four consecutive half-indices per thread (float4), n >= 8; inv: KHELM's
// 1/(6 + h^2 m).
template <int KIND>
__global__ void __launch_bounds__(kBlock)
    k_df_black_update(int lgn, const float *__restrict__ e, const float *__restrict__ r, const float *__restrict__ inv,
                      float h2, float *__restrict__ uh, float *__restrict__ ul, int rev)
{
    pdl_begin();
    const int lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int half = 1 << (3 * lgn - 1);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < (half >> 2); v += gridDim.x * blockDim.x) {
        const int t = (rev ? (half >> 2) - 1 - v : v) << 2;
        const int q = t & mh;
        const int j = (t >> lgh) & mn;
        const int i = t >> (lgh + lgn);
        const int p = (i + j + 1) & 1;  // black cells' k parity offset in this row
        const int r0 = t - q;
        const int ri = j << lgh;
        const int rip = (((i + 1) & mn) << (lgn + lgh)) + ri;
        const int rim = (((i - 1) & mn) << (lgn + lgh)) + ri;
        const int rj = i << (lgn + lgh);
        const int rjp = rj + (((j + 1) & mn) << lgh);
        const int rjm = rj + (((j - 1) & mn) << lgh);
        const float4 A = *reinterpret_cast<const float4 *>(e + rip + q);
        const float4 B = *reinterpret_cast<const float4 *>(e + rim + q);
        const float4 C = *reinterpret_cast<const float4 *>(e + rjp + q);
        const float4 D = *reinterpret_cast<const float4 *>(e + rjm + q);
        const float4 E = *reinterpret_cast<const float4 *>(e + r0 + q);
        const float4 F = *reinterpret_cast<const float4 *>(r + half + t);
        const float x = e[r0 + ((q + (p ? 4 : -1)) & mh)];
        const float4 Sh = p ? make_float4(E.y, E.z, E.w, x) : make_float4(x, E.x, E.y, E.z);
        float4 G = make_float4(1.0f / 6.0f, 1.0f / 6.0f, 1.0f / 6.0f, 1.0f / 6.0f);
        if (KIND == KHELM) G = *reinterpret_cast<const float4 *>(inv + half + t);
        float blk[4];
        blk[0] = (A.x + B.x + C.x + D.x + E.x + Sh.x - h2 * F.x) * G.x;
        blk[1] = (A.y + B.y + C.y + D.y + E.y + Sh.y - h2 * F.y) * G.y;
        blk[2] = (A.z + B.z + C.z + D.z + E.z + Sh.z - h2 * F.z) * G.z;
        blk[3] = (A.w + B.w + C.w + D.w + E.w + Sh.w - h2 * F.w) * G.w;
        const float red[4] = {E.x, E.y, E.z, E.w};
#pragma unroll
        for (int c = 0; c < 2; c++) {
            float4 *H = reinterpret_cast<float4 *>(uh + (c ? half : 0) + t);
            float4 *L = reinterpret_cast<float4 *>(ul + (c ? half : 0) + t);
            const float4 h4 = *H, l4 = *L;
            const float *d = c ? blk : red;
            const df s0 = df_plus_f(h4.x, l4.x, d[0]), s1 = df_plus_f(h4.y, l4.y, d[1]),
                     s2 = df_plus_f(h4.z, l4.z, d[2]), s3 = df_plus_f(h4.w, l4.w, d[3]);
            *H = make_float4(s0.hi, s1.hi, s2.hi, s3.hi);
            *L = make_float4(s0.lo, s1.lo, s2.lo, s3.lo);
        }
    }
}

}  // namespace

int df_resid(int kind, int n, const float *uh, const float *ul, const float *fh, const float *fl, const float *ah,
             const float *al, const float *bh, const float *bl, double h2, double rho, double ref, float *r32,
             float *m32, float *inv32, const float *inv_in, float *e32, double *partials, cudaStream_t st, int rev,
             const double *fshift)
{
    const int lgn = log2i(n);
    const int w = n >= 8 ? 4 : 2;
    const int64_t threads = (int64_t)n * n * n / (2 * w);
    const df cpr = df_from_double_host(2.0 * kPi * rho * h2);
    const float c5 = (float)(10.0 * kPi * rho * h2), ih2 = (float)(1.0 / h2), ih2_ref = (float)(1.0 / (h2 * ref));
    int g = 0;
#define GR_DF_RESID(K, W, S)                                                                                     \
    do {                                                                                                         \
        g = wave_grid(k_df_resid<K, W, S>, threads);                                                             \
        GR_LAUNCH((k_df_resid<K, W, S>), g, kBlock, st, lgn, uh, ul, fh, fl, ah, al, bh, bl, cpr, c5, ih2,       \
                  ih2_ref, r32, m32, inv32, inv_in, e32, partials, rev, fshift, h2);                             \
    } while (0)
    if (kind == KPOISSON && fshift) {
        if (w == 4) GR_DF_RESID(KPOISSON, 4, true);
        else GR_DF_RESID(KPOISSON, 2, true);
    } else if (kind == KPOISSON) {
        if (w == 4) GR_DF_RESID(KPOISSON, 4, false);
        else GR_DF_RESID(KPOISSON, 2, false);
    } else if (kind == KHELM) {
        if (w == 4) GR_DF_RESID(KHELM, 4, false);
        else GR_DF_RESID(KHELM, 2, false);
    } else {
        if (w == 4) GR_DF_RESID(KPSI, 4, false);
        else GR_DF_RESID(KPSI, 2, false);
    }
#undef GR_DF_RESID
    return g;
}

void df_black_update(int kind, int n, const float *e, const float *r, const float *inv, double h2, float *uh,
                     float *ul, cudaStream_t st, int rev)
{
    const int lgn = log2i(n);
    const int64_t threads = (int64_t)n * n * n / 8;
    if (kind == KPOISSON)
        GR_LAUNCH(k_df_black_update<KPOISSON>, wave_grid(k_df_black_update<KPOISSON>, threads), kBlock, st, lgn, e, r,
                  inv, (float)h2, uh, ul, rev);
    else
        GR_LAUNCH(k_df_black_update<KHELM>, wave_grid(k_df_black_update<KHELM>, threads), kBlock, st, lgn, e, r, inv,
                  (float)h2, uh, ul, rev);
}

void df_update(int n, float *uh, float *ul, const float *e, cudaStream_t st)
{
    const int64_t cnt = (int64_t)n * n * n;
    GR_LAUNCH(k_df_update, grid_for(cnt), kBlock, st, cnt, uh, ul, e);
}

}  // namespace gr
