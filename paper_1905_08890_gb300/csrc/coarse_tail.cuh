// coarse_tail.cuh - levels 16^3 .. 2^3 of the FP32 correction V-cycle inside
// one thread block (shared-memory level arrays), used by the single-block
// coarse tail and by the cluster kernel of the coarse levels.  The block
// performs the operations of the per-level kernels in their order: red then
// black passes with k_sweep4's addressing and order of additions, residual
// and 8-child restriction, the FP64 2^3 solve, trilinear prolongation.
#pragma once

#include "gr_internal.cuh"

namespace gr {
namespace {

constexpr int kTailN = 16;
constexpr int kTailThreads = 1024;

struct TailLevel {
    float *e, *r, *m, *inv;
    int lg;
    float h2, ih2;
};

__device__ __forceinline__ int tail_sidx(int lg, int i, int j, int k)
{
    return ((i + j + k) & 1) * (1 << (3 * lg - 1)) + ((((i << lg) + j) << (lg - 1)) + (k >> 1));
}

// W consecutive floats (W = 4 or 2, aligned to W) as one vector access
template <int W>
__device__ __forceinline__ void tail_ldv(const float *p, float (&v)[W])
{
    if (W == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x, v[1] = t.y;
    }
}

// one colour pass on a level of the tail, W consecutive half-indices of a row
// per thread (W = 4 from 8^3, 2 on 4^3), with the addressing and the order of
// additions of the full-grid colour pass (k_sweep4); each row's W values are
// one vector access (scalar accesses W floats apart put W threads of a warp
// on each shared-memory bank)
template <int KIND, int W>
__device__ void tail_sweep_w(const TailLevel &L, int color)
{
    const int lgn = L.lg, lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int half = 1 << (3 * lgn - 1), off = color ? half : 0;
    float *own = L.e + off;
    const float *oth = L.e + (half - off);
    for (int v = threadIdx.x; v < half / W; v += blockDim.x) {
        const int t = v * W;
        const int q = t & mh, j = (t >> lgh) & mn, i = t >> (lgh + lgn);
        const int p = (i + j + color) & 1;
        const int r0 = t - q, ri = j << lgh;
        const int rip = (((i + 1) & mn) << (lgn + lgh)) + ri, rim = (((i - 1) & mn) << (lgn + lgh)) + ri;
        const int rj = i << (lgn + lgh);
        const int rjp = rj + (((j + 1) & mn) << lgh), rjm = rj + (((j - 1) & mn) << lgh);
        const float x = oth[r0 + ((q + (p ? W : -1)) & mh)];
        float A[W], B[W], C[W], D[W], E[W], F[W], G[W];
        tail_ldv<W>(oth + rip + q, A);
        tail_ldv<W>(oth + rim + q, B);
        tail_ldv<W>(oth + rjp + q, C);
        tail_ldv<W>(oth + rjm + q, D);
        tail_ldv<W>(oth + r0 + q, E);
        tail_ldv<W>(L.r + off + t, F);
        if (KIND != KPOISSON) tail_ldv<W>(L.inv + off + t, G);
        float out[W];
#pragma unroll
        for (int e = 0; e < W; e++) {
            const float sh = p ? (e + 1 < W ? E[e + 1 < W ? e + 1 : 0] : x) : (e > 0 ? E[e > 0 ? e - 1 : 0] : x);
            const float nb = A[e] + B[e] + C[e] + D[e] + E[e] + sh;
            out[e] = __fmaf_rn(-L.h2, F[e], nb) * (KIND == KPOISSON ? 1.0f / 6.0f : G[e]);
        }
        if (W == 4) *reinterpret_cast<float4 *>(own + t) = make_float4(out[0], out[1], out[2], out[3]);
        else *reinterpret_cast<float2 *>(own + t) = make_float2(out[0], out[1 % W]);
    }
    __syncthreads();
}

template <int KIND>
__device__ void tail_sweep(const TailLevel &L, int color)
{
    if (L.lg >= 3) tail_sweep_w<KIND, 4>(L, color);
    else tail_sweep_w<KIND, 2>(L, color);
}

// residual L(e) - r of every cell of level A into A's scratch row array res
// (split layout), then the 8-child averages, negated, as the next level's
// right-hand side (its correction starts at zero)
template <int KIND>
__device__ void tail_down(const TailLevel &A, const TailLevel &C, float *res)
{
    const int lgn = A.lg, lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int half = 1 << (3 * lgn - 1);
    for (int tt = threadIdx.x; tt < 2 * half; tt += blockDim.x) {
        const int color = tt >= half, t = tt - (color ? half : 0);
        const int off = color ? half : 0;
        const float *oth = A.e + (half - off);
        const int q = t & mh, j = (t >> lgh) & mn, i = t >> (lgh + lgn);
        const int p = (i + j + color) & 1;
        const int r0 = t - q, ri = j << lgh;
        const int rip = (((i + 1) & mn) << (lgn + lgh)) + ri, rim = (((i - 1) & mn) << (lgn + lgh)) + ri;
        const int rj = i << (lgn + lgh);
        const int rjp = rj + (((j + 1) & mn) << lgh), rjm = rj + (((j - 1) & mn) << lgh);
        const float nb = oth[rip + q] + oth[rim + q] + oth[rjp + q] + oth[rjm + q] + oth[r0 + q] +
                         oth[r0 + ((q + (p ? 1 : -1)) & mh)];
        const int id = off + t;
        const float u = A.e[id];
        float lap = (nb - 6.0f * u) * A.ih2;
        if (KIND == KHELM) lap -= A.m[id] * u;
        res[id] = lap - A.r[id];
    }
    __syncthreads();
    const int lc = C.lg, mc = (1 << lc) - 1;
    for (int t = threadIdx.x; t < (1 << (3 * lc)); t += blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        float s = 0.0f;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int c = 0; c < 2; c++) s += res[tail_sidx(A.lg, 2 * I + a, 2 * J + b, 2 * K + c)];
        const int cid = tail_sidx(lc, I, J, K);
        C.r[cid] = -(0.125f * s);
        C.e[cid] = 0.0f;
    }
    __syncthreads();
}

// trilinear prolongation of the coarser level's correction added to level A;
// black_only: a red pass follows, which does not read the red values, so only
// the black cells take the correction (as prolong_add_black)
__device__ void tail_up(const TailLevel &A, const TailLevel &C, bool black_only)
{
    const int lc = C.lg, mc = (1 << lc) - 1, lf = A.lg, nf1 = (1 << lf) - 1, lgh = lf - 1, mh = (1 << lgh) - 1;
    const int half = 1 << (3 * lf - 1);
    const int ncell = black_only ? half : 2 * half;
    for (int tt = threadIdx.x; tt < ncell; tt += blockDim.x) {
        // split index: colour 1 (black) first when black_only, else both colours
        const int color = black_only ? 1 : (tt >= half), t = tt - ((!black_only && color) ? half : 0);
        const int q = t & mh, j = (t >> lgh) & nf1, i = t >> (lgh + lf);
        const int k = 2 * q + ((i + j + color) & 1);
        int Ia[2], Jb[2], Kc[2];
        Ia[0] = i >> 1;
        Ia[1] = (i & 1) ? ((Ia[0] + 1) & mc) : ((Ia[0] - 1) & mc);
        Jb[0] = j >> 1;
        Jb[1] = (j & 1) ? ((Jb[0] + 1) & mc) : ((Jb[0] - 1) & mc);
        Kc[0] = k >> 1;
        Kc[1] = (k & 1) ? ((Kc[0] + 1) & mc) : ((Kc[0] - 1) & mc);
        const float w[2] = {0.75f, 0.25f};
        float z[2][2];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                z[a][b] = w[0] * C.e[tail_sidx(lc, Ia[a], Jb[b], Kc[0])] + w[1] * C.e[tail_sidx(lc, Ia[a], Jb[b], Kc[1])];
        const float y0 = w[0] * z[0][0] + w[1] * z[0][1], y1 = w[0] * z[1][0] + w[1] * z[1][1];
        A.e[(color ? half : 0) + t] += w[0] * y0 + w[1] * y1;
    }
    __syncthreads();
}

// Exact solve of a linear 2^3 level.  On 2^3 every neighbour of a cell along
// an axis is the same cell of the other colour, counted twice, so the level
// reads (6 + h^2 m_x) e_x - 2 sum_{y ~ x} e_y = -h^2 r_x, where y ~ x are the
// three cells that differ from x in one coordinate (x = 4i + 2j + k).
// KPOISSON (m = 0): the 8-point Walsh-Hadamard basis (-1)^(s.x)
// diagonalises the operator, eigenvalue 4|s| (|s| the number of bits set in
// s), so e = W diag(1 / (4|s|)) W (-h^2 r) / 8 with the s = 0 component, the
// mean, set to zero: the mean-free solution.  KHELM (m >= 0, not all zero):
// Gauss-Jordan elimination, one row per lane (symmetric and diagonally
// dominant, no pivoting); m = 0 on all eight cells takes the Poisson solve.  The red-black sweeps this replaces converge to the same
// solution (the 2^3 level is solved, Sec. 4.3.1).  Called by a whole warp;
// lane x < 8 passes r_x and m_x of cell x and receives e_x (lanes 8..31
// repeat lanes 0..7).
// the KPOISSON solve (whole warp, lanes in groups of eight)
__device__ __forceinline__ double coarsest_wht(double rx, double h2)
{
    const unsigned full = 0xffffffffu;
    const int x = threadIdx.x & 7;
    double v = -h2 * rx;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const double w = __shfl_xor_sync(full, v, 1 << b);
        v = ((x >> b) & 1) ? w - v : v + w;
    }
    const int s = __popc(x);
    v = s ? v / (4.0 * s) : 0.0;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const double w = __shfl_xor_sync(full, v, 1 << b);
        v = ((x >> b) & 1) ? w - v : v + w;
    }
    return 0.125 * v;
}

template <int KIND>
__device__ __forceinline__ double coarsest_exact(double rx, double mx, double h2)
{
    const unsigned full = 0xffffffffu;
    const int x = threadIdx.x & 7;
    if (KIND == KPOISSON) return coarsest_wht(rx, h2);
    // m = 0 on every cell would leave the Laplacian, singular on the constant
    // mode: then its mean-free solution.  No caller reaches it: the contexts
    // require rho_hat > 0, which puts K^2 = 24 pi rho_hat into the lapse's m
    // and 10 pi rho_hat psi^4 into the psi equation's Newton coefficient.
    // (The sum is the same in every group of eight lanes.)
    double ms = mx;
#pragma unroll
    for (int b = 0; b < 3; b++) ms += __shfl_xor_sync(full, ms, 1 << b);
    if (!(ms > 0.0)) return coarsest_wht(rx, h2);
    double a[8];
#pragma unroll
    for (int y = 0; y < 8; y++) a[y] = y == x ? 6.0 + h2 * mx : (__popc(x ^ y) == 1 ? -2.0 : 0.0);
    double b = -h2 * rx;
#pragma unroll
    for (int p = 0; p < 8; p++) {
        const int src = (threadIdx.x & ~7) + p;  // row p of this lane's group of eight
        const double piv = __shfl_sync(full, a[p], src);
        const double bp = __shfl_sync(full, b, src);
        double row[8];
#pragma unroll
        for (int k = p + 1; k < 8; k++) row[k] = __shfl_sync(full, a[k], src);
        if (x != p) {
            const double f = a[p] / piv;
#pragma unroll
            for (int k = p + 1; k < 8; k++) a[k] = fma(-f, row[k], a[k]);
            b = fma(-f, bp, b);
        }
    }
    double d = a[0];
#pragma unroll
    for (int y = 1; y < 8; y++) d = y == x ? a[y] : d;
    return b / d;
}

// FP64 solve of the 2^3 level (as k_coarsest), by the first warp: the
// right-hand side's mean removed (KPOISSON), then the exact solve
template <int KIND>
__device__ void tail_coarsest(const TailLevel &Z)
{
    __shared__ double sf[8];
    const int t = threadIdx.x;
    if (t < 32) {
        if (t < 8) sf[t] = Z.r[t];
        __syncwarp();
        if (KIND == KPOISSON && t == 0) {
            double m = 0.0;
            for (int q = 0; q < 8; q++) m += sf[q];
            m *= 0.125;
            for (int q = 0; q < 8; q++) sf[q] -= m;
        }
        __syncwarp();
        // lane x holds cell x = 4i + 2j + k, split index 4 ((i + j + k) & 1) + 2i + j
        const int x = t & 7, i = x >> 2, j = (x >> 1) & 1, k = x & 1;
        const int id = 4 * ((i + j + k) & 1) + 2 * i + j;
        const double e = coarsest_exact<KIND>(sf[id], KIND == KPOISSON ? 0.0 : (double)Z.m[id], (double)Z.h2);
        if (t < 8) Z.e[id] = (float)e;
    }
    __syncthreads();
}

// one correction V-cycle over the tail levels L[3] (16^3, e and r given) ..
// L[0] (2^3): nu1 red-black sweeps, residual-restriction, the 2^3 solve,
// prolongation and nu2 sweeps; res: scratch of 16^3 floats
template <int KIND>
__device__ __forceinline__ void tail_cycle(TailLevel (&L)[4], float *res, int nu1, int nu2)
{
#pragma unroll
    for (int l = 3; l >= 1; l--) {
        for (int s = 0; s < nu1; s++) {
            tail_sweep<KIND>(L[l], 0);
            tail_sweep<KIND>(L[l], 1);
        }
        tail_down<KIND>(L[l], L[l - 1], res);
    }
    tail_coarsest<KIND>(L[0]);
#pragma unroll
    for (int l = 1; l <= 3; l++) {
        tail_up(L[l], L[l - 1], nu2 > 0);
        for (int s = 0; s < nu2; s++) {
            tail_sweep<KIND>(L[l], 0);
            tail_sweep<KIND>(L[l], 1);
        }
    }
}

}  // namespace
}  // namespace gr
