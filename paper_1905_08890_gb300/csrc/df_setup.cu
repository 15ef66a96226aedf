// df_setup.cu - set-up and write-back of the double-float mixed solve.
//
// In the double-float mode the finest level is never held in FP64.  These
// kernels read the natural [n][n][n] FP64 sources and fields and write the
// unknown, the right-hand side and the coefficients of one equation as hi/lo
// FP32 pairs in the red-black split layout; the arithmetic of the sources
// (mean removal, the central differences of Sec. 4.3.1, the powers of psi) is
// double-float, fed by the integer split of df64.cuh.  FP64 appears once per
// thread (the block sums), never per cell: GB300 issues FP64 at 1/58 of its
// FP32 rate, and per-cell FP64 arithmetic would make these memory-sized
// passes compute bound.  The write-back joins each pair into a double with
// integer operations (join_double).
//
// Threads of the split-layout kernels own a pair of cells k0 = 2q, k0 + 1 of
// row (i, j): one is red, one black, so both colours' arrays are written
// coalesced at the same split offset t, and the natural arrays are read in
// whole rows.
#include "df64.cuh"
#include "gr_internal.cuh"

namespace gr {
namespace {

inline int grid_for(int64_t work)
{
    int64_t b = (work + kBlock - 1) / kBlock;
    const int64_t cap = kMaxRedBlocks;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

inline int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// natural index; 32-bit since n <= 1024
__device__ __forceinline__ int nat(int lgn, int i, int j, int k) { return (((i << lgn) + j) << lgn) + k; }

__device__ __forceinline__ df ld(const double *__restrict__ a, int64_t id) { return split_double(a[id]); }

__device__ __forceinline__ df ldp(const float *__restrict__ h, const float *__restrict__ l, int64_t id)
{
    return {h[id], l[id]};
}

__device__ __forceinline__ void stp(float *__restrict__ h, float *__restrict__ l, int64_t id, df v)
{
    h[id] = v.hi;
    l[id] = v.lo;
}

// Threads of the split-layout kernels own kChunk consecutive half-indices
// t .. t + kChunk - 1 of a row (i, j), that is the 2 kChunk cells
// k = k0 .. k0 + 2 kChunk - 1 with k0 = 2 (t mod n/2); cell k0 + e has colour
// c0 ^ (e & 1) and split index (c0 ^ (e & 1)) n^3/2 + t + e/2.  Several cells
// per thread keep more independent loads in flight.
constexpr int kChunk = 2;

struct PairPos {
    int i, j, k0, c0;
    int64_t t, half;
};

__device__ __forceinline__ PairPos pair_pos(int lgn, int64_t t)
{
    const int lgh = lgn - 1, mn = (1 << lgn) - 1;
    PairPos p;
    p.t = t;
    p.half = (int64_t)1 << (3 * lgn - 1);
    p.k0 = 2 * (int)(t & ((1 << lgh) - 1));
    p.j = (int)((t >> lgh) & mn);
    p.i = (int)(t >> (lgh + lgn));
    p.c0 = (p.i + p.j) & 1;
    return p;
}

// The four cells k0 .. k0 + 3 of a thread (kChunk = 2): natural-layout
// values by two 16-byte loads, split-layout pairs by 8-byte loads and stores
// (cells 0 and 2 have colour c0 and split indices t, t + 1; cells 1 and 3 the
// other colour).
static_assert(kChunk == 2, "the vector accesses below assume four cells per thread");

__device__ __forceinline__ void ld4(const double *__restrict__ a, int id0, df v[4])
{
    const double2 x = *reinterpret_cast<const double2 *>(a + id0), y = *reinterpret_cast<const double2 *>(a + id0 + 2);
    v[0] = split_double(x.x), v[1] = split_double(x.y), v[2] = split_double(y.x), v[3] = split_double(y.y);
}

__device__ __forceinline__ void st4(double *__restrict__ a, int id0, const double v[4])
{
    *reinterpret_cast<double2 *>(a + id0) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(a + id0 + 2) = make_double2(v[2], v[3]);
}

__device__ __forceinline__ void stp4(float *__restrict__ h, float *__restrict__ l, const PairPos &p, const df v[4])
{
    const int64_t a = (p.c0 ? p.half : 0) + p.t, b = (p.c0 ? 0 : p.half) + p.t;
    *reinterpret_cast<float2 *>(h + a) = make_float2(v[0].hi, v[2].hi);
    *reinterpret_cast<float2 *>(l + a) = make_float2(v[0].lo, v[2].lo);
    *reinterpret_cast<float2 *>(h + b) = make_float2(v[1].hi, v[3].hi);
    *reinterpret_cast<float2 *>(l + b) = make_float2(v[1].lo, v[3].lo);
}

__device__ __forceinline__ void stf4(float *__restrict__ h, const PairPos &p, const float v[4])
{
    const int64_t a = (p.c0 ? p.half : 0) + p.t, b = (p.c0 ? 0 : p.half) + p.t;
    *reinterpret_cast<float2 *>(h + a) = make_float2(v[0], v[2]);
    *reinterpret_cast<float2 *>(h + b) = make_float2(v[1], v[3]);
}

__device__ __forceinline__ void ldp4(const float *__restrict__ h, const float *__restrict__ l, const PairPos &p, df v[4])
{
    const int64_t a = (p.c0 ? p.half : 0) + p.t, b = (p.c0 ? 0 : p.half) + p.t;
    const float2 ha = *reinterpret_cast<const float2 *>(h + a), la = *reinterpret_cast<const float2 *>(l + a);
    const float2 hb = *reinterpret_cast<const float2 *>(h + b), lb = *reinterpret_cast<const float2 *>(l + b);
    v[0] = {ha.x, la.x}, v[1] = {hb.x, lb.x}, v[2] = {ha.y, la.y}, v[3] = {hb.y, lb.y};
}

// running sum of df values (high parts through two-sum, errors and low parts
// in FP32) and sum of squares of the high parts
struct Acc {
    df s = {0.0f, 0.0f};
    float q = 0.0f;
    __device__ __forceinline__ void add(df x)
    {
        const df t = two_sum(s.hi, x.hi);
        s.hi = t.hi;
        s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, x.lo));
        q = __fmaf_rn(x.hi, x.hi, q);
    }
    // block partials: the warp sums in double-float (FP32) arithmetic, the
    // eight warp totals in FP64
    __device__ __forceinline__ void flush(double *partials) const
    {
        __shared__ double sa[kBlock / 32], sb[kBlock / 32];
        df a = s;
        float b = q;
        for (int o = 16; o > 0; o >>= 1) {
            const df t = {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
            a = df_add(a, t);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            sa[w] = (double)a.hi + (double)a.lo;
            sb[w] = (double)b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ta = 0.0, tb = 0.0;
            for (int k = 0; k < kBlock / 32; k++) {
                ta += sa[k];
                tb += sb[k];
            }
            partials[2 * blockIdx.x] = ta;
            partials[2 * blockIdx.x + 1] = tb;
        }
    }
};

__device__ __forceinline__ df df_scale2(df a, float p2) { return {a.hi * p2, a.lo * p2}; }  // exact for p2 = 2^k

// ---------------------------------------------------------------- sums
__global__ void __launch_bounds__(kBlock) k_dfs_sum(int64_t cnt, const double *__restrict__ a, double *partials)
{
    pdl_begin();
    Acc acc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        acc.add(ld(a, t));
    acc.flush(partials);
}

__global__ void __launch_bounds__(kBlock)
    k_dfs_pair_sum(int64_t cnt, const float *__restrict__ h, const float *__restrict__ l, double *partials)
{
    pdl_begin();
    Acc acc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        acc.add(ldp(h, l, t));
    acc.flush(partials);
}

// Row reads of four consecutive cells k0 .. k0 + 3 (k0 a multiple of 4) of
// the natural row starting at r, with the two periodic end values k0 - 1 and
// k0 + 4 for the six-value forms: pair arrays (h, l) by 16-byte loads, FP64
// arrays by two 16-byte loads and split.
__device__ __forceinline__ void hl_row4(const float *__restrict__ h, const float *__restrict__ l, int r, int k0, df o[4])
{
    const float4 a = *reinterpret_cast<const float4 *>(h + r + k0), b = *reinterpret_cast<const float4 *>(l + r + k0);
    o[0] = {a.x, b.x}, o[1] = {a.y, b.y}, o[2] = {a.z, b.z}, o[3] = {a.w, b.w};
}
__device__ __forceinline__ void hl_row6(const float *__restrict__ h, const float *__restrict__ l, int r, int k0, int m,
                                        df o[6])
{
    const int km = r + ((k0 - 1) & m), kp = r + ((k0 + 4) & m);
    o[0] = {h[km], l[km]};
    hl_row4(h, l, r, k0, o + 1);
    o[5] = {h[kp], l[kp]};
}
__device__ __forceinline__ void d_row6(const double *__restrict__ a, int r, int k0, int m, df o[6])
{
    o[0] = ld(a, r + ((k0 - 1) & m));
    ld4(a, r + k0, o + 1);
    o[5] = ld(a, r + ((k0 + 4) & m));
}

// ---------------------------------------------------------------- Poisson right-hand sides
// SRC_MEAN: f = scale (s - <s>), <s> = sum[0] inv_cnt           (V_i, Eq. MG-linear-1a)
// SRC_DIV:  f = scale sum_l (F_l(+l) - F_l(-l)), scale = -1/(8h) (U and b, Eqs. MG-linear-1, -2)
// SRC_SHIFT: f = scale sum_l (A^{cl} w)(+l) - (A^{cl} w)(-l), scale = 1/h  (B^c, Eq. MG-linear-2a)
// Each also loads the unknown from the field and accumulates sum f, sum f^2.
// Differences of neighbouring values use the plain double-float sum: its
// absolute error, about 2^-47 of the operands, is near 2^-37 of a central
// difference at 512^3.
enum Src : int { SRC_MEAN = 0, SRC_DIV = 1, SRC_SHIFT = 2 };

struct PoissonArgs {
    const double *s[3];  // SRC_MEAN: s[0]; SRC_DIV: F_x, F_y, F_z
    const double *sum;   // SRC_MEAN: device sum of s[0]
    double inv_cnt;
    const float *A;      // SRC_SHIFT: A^{ij} pairs, natural, component c at A + 2 c N (hi), A + (2c+1) N (lo)
    const float *wh, *wl;  // SRC_SHIFT: weight pairs, natural
    int comp;            // SRC_SHIFT: the component c of B^c
    df scale;
    const double *fld;  // the unknown (natural)
    float *uh, *ul, *fh, *fl;
};

template <int SRC>
__global__ void __launch_bounds__(kBlock, SRC == SRC_SHIFT ? 2 : 3) k_dfs_poisson(int lgn, PoissonArgs a, double *partials)
{
    pdl_begin();
    const int mn = (1 << lgn) - 1;
    const int64_t N = (int64_t)1 << (3 * lgn);
    df mu = {0.0f, 0.0f};
    if (SRC == SRC_MEAN) mu = split_double(a.sum[0] * a.inv_cnt);
    const df nmu = df_neg(mu);
    int tab[3] = {0, 0, 0};
    if (SRC == SRC_SHIFT) {
        // A^{c l} for l = x, y, z in the xx yy zz xy xz yz order
        const int rows[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
        for (int l = 0; l < 3; l++) tab[l] = rows[a.comp][l];
    }
    Acc acc;
    for (int64_t tc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tc < (N >> 1) / kChunk;
         tc += (int64_t)gridDim.x * blockDim.x) {
        const PairPos p = pair_pos(lgn, tc * kChunk);
        df fv[4], uv[4], sv[4];
        ld4(a.fld, nat(lgn, p.i, p.j, p.k0), uv);
        if (SRC == SRC_MEAN) ld4(a.s[0], nat(lgn, p.i, p.j, p.k0), sv);
        if (SRC == SRC_MEAN) {
#pragma unroll
            for (int e = 0; e < 2 * kChunk; e++) fv[e] = df_mul(df_add_acc(sv[e], nmu), a.scale);
        } else {
            // the +l and -l neighbours of the four cells: rows (i +- 1, j), (i, j +- 1), and the own row's
            // values k0 - 1 .. k0 + 4; per cell the sum over l = x, y, z of the differences, in that order
            const int rows[2][2] = {{nat(lgn, (p.i + 1) & mn, p.j, 0), nat(lgn, (p.i - 1) & mn, p.j, 0)},
                                    {nat(lgn, p.i, (p.j + 1) & mn, 0), nat(lgn, p.i, (p.j - 1) & mn, 0)}};
            const int own = nat(lgn, p.i, p.j, 0);
            df d[4];
#pragma unroll
            for (int l = 0; l < 3; l++) {
                df P[4], M[4];
                if (SRC == SRC_DIV) {
                    if (l < 2) {
                        ld4(a.s[l], rows[l][0] + p.k0, P);
                        ld4(a.s[l], rows[l][1] + p.k0, M);
                    } else {
                        df z[6];
                        d_row6(a.s[2], own, p.k0, mn, z);
#pragma unroll
                        for (int e = 0; e < 4; e++) P[e] = z[e + 2], M[e] = z[e];
                    }
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const df q = df_add(P[e], df_neg(M[e]));
                        d[e] = l == 0 ? q : df_add(d[e], q);
                    }
                } else {
                    const float *Ah = a.A + 2 * tab[l] * N, *Al = Ah + N;
                    df WP[4], WM[4];
                    if (l < 2) {
                        hl_row4(Ah, Al, rows[l][0], p.k0, P);
                        hl_row4(Ah, Al, rows[l][1], p.k0, M);
                        hl_row4(a.wh, a.wl, rows[l][0], p.k0, WP);
                        hl_row4(a.wh, a.wl, rows[l][1], p.k0, WM);
                    } else {
                        df za[6], zw[6];
                        hl_row6(Ah, Al, own, p.k0, mn, za);
                        hl_row6(a.wh, a.wl, own, p.k0, mn, zw);
#pragma unroll
                        for (int e = 0; e < 4; e++) P[e] = za[e + 2], M[e] = za[e], WP[e] = zw[e + 2], WM[e] = zw[e];
                    }
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const df fp = df_mul(P[e], WP[e]);
                        const df fm = df_mul(M[e], WM[e]);
                        d[e] = df_add(l == 0 ? df{0.0f, 0.0f} : d[e], df_add(fp, df_neg(fm)));
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++) fv[e] = df_mul(d[e], a.scale);
        }
#pragma unroll
        for (int e = 0; e < 2 * kChunk; e++) acc.add(fv[e]);
        stp4(a.fh, a.fl, p, fv);
        stp4(a.uh, a.ul, p, uv);
    }
    acc.flush(partials);
}

// ---------------------------------------------------------------- A_ij
// Natural-layout pairs of four fields (V_x, V_y, V_z, U): split once, since
// the A_ij stencil reads each value up to 19 times.
__global__ void __launch_bounds__(kBlock)
    k_dfs_split4(int64_t cnt, const double *__restrict__ a0, const double *__restrict__ a1,
                 const double *__restrict__ a2, const double *__restrict__ a3, float *__restrict__ p0,
                 float *__restrict__ p1, float *__restrict__ p2, float *__restrict__ p3)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        stp(p0, p0 + cnt, t, ld(a0, t));
        stp(p1, p1 + cnt, t, ld(a1, t));
        stp(p2, p2 + cnt, t, ld(a2, t));
        stp(p3, p3 + cnt, t, ld(a3, t));
    }
}

// A_ij of Eq. Aij-discrete-2 (xx yy zz xy xz yz) and AA = A_ij A^ij as
// natural-layout pairs, from the pairs of V_x, V_y, V_z, U (hi at P[f],
// lo at P[f] + n^3); D_a V_l central, U's second derivatives by the
// three-point and four-corner stencils (Eq. U-cross-deriv), differences by
// the plain double-float sum as in the Poisson right-hand sides.  Each thread
// makes four consecutive cells k0 .. k0 + 3 of a row: every neighbour row is
// read once as a pair of float4 (with the two wrapped end values where the
// k neighbours are needed), and the outputs are written as float4.  The
// double-float operations of each cell are those of a cell-by-cell
// evaluation, in the same order; the components are formed one after another
// (AA's sums of squares accumulate in the order xx, yy, zz and xy, xz, yz).

// values k0 .. k0 + 3 of the row starting at r of a pair array f (lo at f + N)
__device__ __forceinline__ void prow4(const float *__restrict__ f, int64_t N, int r, int k0, df o[4])
{
    const float4 h = *reinterpret_cast<const float4 *>(f + r + k0), l = *reinterpret_cast<const float4 *>(f + N + r + k0);
    o[0] = {h.x, l.x}, o[1] = {h.y, l.y}, o[2] = {h.z, l.z}, o[3] = {h.w, l.w};
}

// values k0 - 1 .. k0 + 4 (periodic) of the row starting at r
__device__ __forceinline__ void prow6(const float *__restrict__ f, int64_t N, int r, int k0, int m, df o[6])
{
    const int km = r + ((k0 - 1) & m), kp = r + ((k0 + 4) & m);
    o[0] = {f[km], f[N + km]};
    prow4(f, N, r, k0, o + 1);
    o[5] = {f[kp], f[N + kp]};
}

__device__ __forceinline__ void pst4(float *__restrict__ h, float *__restrict__ l, int t, const df v[4])
{
    *reinterpret_cast<float4 *>(h + t) = make_float4(v[0].hi, v[1].hi, v[2].hi, v[3].hi);
    *reinterpret_cast<float4 *>(l + t) = make_float4(v[0].lo, v[1].lo, v[2].lo, v[3].lo);
}

__global__ void __launch_bounds__(kBlock, 2)
    k_dfs_aij(int lgn, df inv2h, df ih2, const float *__restrict__ Pvx, const float *__restrict__ Pvy,
              const float *__restrict__ Pvz, const float *__restrict__ Pu, float *__restrict__ A,
              float *__restrict__ AAh, float *__restrict__ AAl)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * lgn);
    const int m = (1 << lgn) - 1;
    const float *V[3] = {Pvx, Pvy, Pvz};
    const df qih2 = df_scale2(ih2, 0.25f);
    auto diff = [&](df a, df b) { return df_add(a, df_neg(b)); };
    for (int tc = blockIdx.x * blockDim.x + threadIdx.x; tc < (int)(N >> 2); tc += gridDim.x * blockDim.x) {
        const int t = tc << 2;
        const int k0 = t & m, j = (t >> lgn) & m, i = t >> (2 * lgn);
        const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
        const int r = t - k0;                                   // row (i, j)
        const int rp[2] = {nat(lgn, ip, j, 0), nat(lgn, i, jp, 0)};  // rows (i + 1, j), (i, j + 1)
        const int rm[2] = {nat(lgn, im, j, 0), nat(lgn, i, jm, 0)};  // rows (i - 1, j), (i, j - 1)
        // D_ax V_l of the four cells: x and y from the neighbour rows, z along the own row
        auto dv = [&](int ax, int l, df d[4]) {
            if (ax < 2) {
                df a[4], b[4];
                prow4(V[l], N, rp[ax], k0, a);
                prow4(V[l], N, rm[ax], k0, b);
#pragma unroll
                for (int e = 0; e < 4; e++) d[e] = df_mul(diff(a[e], b[e]), inv2h);
            } else {
                df z[6];
                prow6(V[l], N, r, k0, m, z);
#pragma unroll
                for (int e = 0; e < 4; e++) d[e] = df_mul(diff(z[e + 2], z[e]), inv2h);
            }
        };
        df Dd[3][4], divV[4], dd[4], oo[4], u0m2[4], U6[6];
        dv(0, 0, Dd[0]);
        dv(1, 1, Dd[1]);
        dv(2, 2, Dd[2]);
        prow6(Pu, N, r, k0, m, U6);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            divV[e] = df_add(df_add(Dd[0][e], Dd[1][e]), Dd[2][e]);
            u0m2[e] = df_scale2(U6[e + 1], -2.0f);
        }
        // diagonal components
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            df up[4], um[4], Ad[4];
            if (ax < 2) {
                prow4(Pu, N, rp[ax], k0, up);
                prow4(Pu, N, rm[ax], k0, um);
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++) up[e] = U6[e + 2], um[e] = U6[e];
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const df Uaa = df_mul(df_add(df_add(up[e], um[e]), u0m2[e]), ih2);
                Ad[e] = df_add(df_add(df_scale2(Dd[ax][e], 2.0f), df_scale2(divV[e], -0.5f)), df_scale2(Uaa, 2.0f));
                const df sq = df_mul(Ad[e], Ad[e]);
                dd[e] = ax == 0 ? sq : df_add(dd[e], sq);
            }
            pst4(A + 2 * ax * N, A + (2 * ax + 1) * N, t, Ad);
        }
        // off-diagonal components xy, xz, yz: D_a V_b + D_b V_a + 2 U_ab
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int a = c < 2 ? 0 : 1, b = c == 0 ? 1 : 2;
            df Dab[4], Dba[4], Uab[4], Ao[4];
            dv(a, b, Dab);
            dv(b, a, Dba);
            if (c == 0) {  // corners (i +- 1, j +- 1) at k
                df pp[4], mm[4], mp[4], pm[4];
                prow4(Pu, N, nat(lgn, ip, jp, 0), k0, pp);
                prow4(Pu, N, nat(lgn, im, jm, 0), k0, mm);
                prow4(Pu, N, nat(lgn, im, jp, 0), k0, mp);
                prow4(Pu, N, nat(lgn, ip, jm, 0), k0, pm);
#pragma unroll
                for (int e = 0; e < 4; e++) Uab[e] = df_mul(diff(df_add(pp[e], mm[e]), df_add(mp[e], pm[e])), qih2);
            } else {  // corners (x_a +- 1, k +- 1): rows (i +- 1, j) (c = 1) or (i, j +- 1) (c = 2)
                df P6[6], M6[6];
                prow6(Pu, N, rp[c - 1], k0, m, P6);
                prow6(Pu, N, rm[c - 1], k0, m, M6);
#pragma unroll
                for (int e = 0; e < 4; e++)
                    Uab[e] = df_mul(diff(df_add(P6[e + 2], M6[e]), df_add(M6[e + 2], P6[e])), qih2);
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                Ao[e] = df_add(df_add(Dab[e], Dba[e]), df_scale2(Uab[e], 2.0f));
                const df sq = df_mul(Ao[e], Ao[e]);
                oo[e] = c == 0 ? sq : df_add(oo[e], sq);
            }
            pst4(A + 2 * (3 + c) * N, A + (2 * (3 + c) + 1) * N, t, Ao);
        }
        df aa[4];
#pragma unroll
        for (int e = 0; e < 4; e++) aa[e] = df_add(dd[e], df_scale2(oo[e], 2.0f));
        pst4(AAh, AAl, t, aa);
    }
}

// ---------------------------------------------------------------- psi, alpha psi
// psi (Eq. MG-nonlinear): unknown psi - 1, a' = 2 pi h^2 s0, b' = h^2 AA / 8,
// f = 0 (the premultiplied coefficients of the residual kernel); sums of s0^2
__global__ void __launch_bounds__(kBlock)
    k_dfs_psi(int lgn, df a_scale, df b_scale, const double *__restrict__ psi, const double *__restrict__ s0,
              const float *__restrict__ AAh, const float *__restrict__ AAl, float *__restrict__ uh,
              float *__restrict__ ul, float *__restrict__ ah, float *__restrict__ al, float *__restrict__ bh,
              float *__restrict__ bl, float *__restrict__ fh, float *__restrict__ fl, double *partials)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * lgn);
    const df m1 = {-1.0f, 0.0f};
    Acc acc;
    for (int64_t tc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tc < (N >> 1) / kChunk;
         tc += (int64_t)gridDim.x * blockDim.x) {
        const PairPos p = pair_pos(lgn, tc * kChunk);
        const int id0 = nat(lgn, p.i, p.j, p.k0);
        df sv[4], pv[4], uo[4], ao[4], bo[4];
        const df zo[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
        ld4(s0, id0, sv);
        ld4(psi, id0, pv);
        const float4 Ah = *reinterpret_cast<const float4 *>(AAh + id0), Al = *reinterpret_cast<const float4 *>(AAl + id0);
        const df av[4] = {{Ah.x, Al.x}, {Ah.y, Al.y}, {Ah.z, Al.z}, {Ah.w, Al.w}};
#pragma unroll
        for (int e = 0; e < 2 * kChunk; e++) {
            uo[e] = df_add_acc(pv[e], m1);
            ao[e] = df_mul(sv[e], a_scale);
            bo[e] = df_mul(av[e], b_scale);
            acc.add(sv[e]);
        }
        stp4(uh, ul, p, uo);
        stp4(ah, al, p, ao);
        stp4(bh, bl, p, bo);
        stp4(fh, fl, p, zo);
    }
    acc.flush(partials);
}

// lapse equation for phi = alpha psi (Eq. sol-scheme-CMC with s = psi^-4 sigma),
// unknown phi - 1:  lap(phi - 1) - m (phi - 1) = m - psi^5 Kdot, with
// m = 2 pi psi^-2 (s0 + 2 sigma psi^-4) + 7/8 AA psi^-8 + 5/12 K^2 psi^4.
// Writes u, a' = h^2 m and f' = h^2 (m - psi^5 Kdot) as pairs, m and
// 1/(6 + h^2 m) in FP32; sums of (psi^5 Kdot)^2.  k2c = 5/12 K^2.
__global__ void __launch_bounds__(kBlock)
    k_dfs_apsi(int lgn, float h2, df h2d, const double *__restrict__ psi, const double *__restrict__ apsi,
               const double *__restrict__ s0, const double *__restrict__ sig, const float *__restrict__ AAh,
               const float *__restrict__ AAl, df two_pi, df k2c, df kdot, float *__restrict__ uh,
               float *__restrict__ ul, float *__restrict__ ah, float *__restrict__ al, float *__restrict__ fh,
               float *__restrict__ fl, float *__restrict__ m32, float *__restrict__ inv32, double *partials)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * lgn);
    const df m1 = {-1.0f, 0.0f};
    Acc acc;
    for (int64_t tc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tc < (N >> 1) / kChunk;
         tc += (int64_t)gridDim.x * blockDim.x) {
        const PairPos p = pair_pos(lgn, tc * kChunk);
        const int id0 = nat(lgn, p.i, p.j, p.k0);
        df psv[4], apv[4], s0v[4], sgv[4], uo[4], ao[4], fo[4];
        float mo[4], io[4];
        ld4(psi, id0, psv);
        ld4(apsi, id0, apv);
        ld4(s0, id0, s0v);
        ld4(sig, id0, sgv);
        const float4 Ah = *reinterpret_cast<const float4 *>(AAh + id0), Al = *reinterpret_cast<const float4 *>(AAl + id0);
        const df av[4] = {{Ah.x, Al.x}, {Ah.y, Al.y}, {Ah.z, Al.z}, {Ah.w, Al.w}};
#pragma unroll
        for (int e = 0; e < 2 * kChunk; e++) {
            const df ps = psv[e];
            const df ip = df_recip(ps);
            const df ip2 = df_mul(ip, ip), ip4 = df_mul(ip2, ip2), ip8 = df_mul(ip4, ip4);
            const df p2 = df_mul(ps, ps), p4 = df_mul(p2, p2), p5 = df_mul(p4, ps);
            const df inner = df_add(s0v[e], df_mul(df_scale2(sgv[e], 2.0f), ip4));
            const df mm = df_add(df_add(df_mul(df_mul(two_pi, ip2), inner), df_mulf(df_mul(av[e], ip8), 0.875f)),
                                 df_mul(p4, k2c));
            const df src = df_mul(p5, kdot);
            uo[e] = df_add_acc(apv[e], m1);
            ao[e] = df_mul(mm, h2d);
            fo[e] = df_mul(df_add(mm, df_neg(src)), h2d);
            mo[e] = mm.hi;
            io[e] = 1.0f / (6.0f + h2 * mm.hi);
            acc.add(src);
        }
        stp4(uh, ul, p, uo);
        stp4(ah, al, p, ao);
        stp4(fh, fl, p, fo);
        stf4(m32, p, mo);
        stf4(inv32, p, io);
    }
    acc.flush(partials);
}

// shift weight alpha psi^-6 = (alpha psi) psi^-7, natural pairs
__global__ void __launch_bounds__(kBlock) k_dfs_weight(int64_t cnt, const double *__restrict__ psi,
                                                       const double *__restrict__ apsi, float *__restrict__ wh,
                                                       float *__restrict__ wl)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const df ip = df_recip(ld(psi, t));
        const df ip2 = df_mul(ip, ip), ip4 = df_mul(ip2, ip2);
        stp(wh, wl, t, df_mul(ld(apsi, t), df_mul(df_mul(ip4, ip2), ip)));
    }
}

// ---------------------------------------------------------------- write-back
// nat = join(u - <u>) (+ 1 for the deviation unknowns), <u> = sum[0] inv_cnt
// DEV as a template parameter: a runtime flag would leave a predicated FP64
// add on every element, which still occupies the narrow FP64 pipe
template <int DEV>
__global__ void __launch_bounds__(kBlock)
    k_dfs_store(int lgn, const float *__restrict__ uh, const float *__restrict__ ul, const double *__restrict__ sum,
                double inv_cnt, double *__restrict__ out)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * lgn);
    const df nmu = sum ? df_neg(split_double(sum[0] * inv_cnt)) : df{0.0f, 0.0f};
    for (int64_t tc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tc < (N >> 1) / kChunk;
         tc += (int64_t)gridDim.x * blockDim.x) {
        const PairPos p = pair_pos(lgn, tc * kChunk);
        df v[4];
        double d[4];
        ldp4(uh, ul, p, v);
#pragma unroll
        for (int e = 0; e < 2 * kChunk; e++) {
            if (sum) v[e] = df_add_acc(v[e], nmu);
            d[e] = join_double(v[e]);
            if (DEV) d[e] += 1.0;
        }
        st4(out, nat(lgn, p.i, p.j, p.k0), d);
    }
}

}  // namespace

// ================================================================ launchers
int dfs_sum(int64_t cnt, const double *a, double *partials, cudaStream_t st)
{
    const int g = grid_for(cnt);
    GR_LAUNCH(k_dfs_sum, g, kBlock, st, cnt, a, partials);
    return g;
}

int dfs_pair_sum(int64_t cnt, const float *h, const float *l, double *partials, cudaStream_t st)
{
    const int g = grid_for(cnt);
    GR_LAUNCH(k_dfs_pair_sum, g, kBlock, st, cnt, h, l, partials);
    return g;
}

int dfs_mean_rhs(int n, const double *s, const double *sum, double scale, const double *fld, float *uh, float *ul,
                 float *fh, float *fl, double *partials, cudaStream_t st)
{
    const int lgn = log2i(n);
    PoissonArgs a = {};
    a.s[0] = s;
    a.sum = sum;
    a.inv_cnt = 1.0 / ((double)n * n * n);
    a.scale = df_from_double_host(scale);
    a.fld = fld;
    a.uh = uh;
    a.ul = ul;
    a.fh = fh;
    a.fl = fl;
    const int g = wave_grid(k_dfs_poisson<SRC_MEAN>, (int64_t)n * n * n / (2 * kChunk));
    GR_LAUNCH(k_dfs_poisson<SRC_MEAN>, g, kBlock, st, lgn, a, partials);
    return g;
}

int dfs_div_rhs(int n, double scale, const double *Fx, const double *Fy, const double *Fz, const double *fld,
                float *uh, float *ul, float *fh, float *fl, double *partials, cudaStream_t st)
{
    const int lgn = log2i(n);
    PoissonArgs a = {};
    a.s[0] = Fx;
    a.s[1] = Fy;
    a.s[2] = Fz;
    a.scale = df_from_double_host(scale);
    a.fld = fld;
    a.uh = uh;
    a.ul = ul;
    a.fh = fh;
    a.fl = fl;
    const int g = wave_grid(k_dfs_poisson<SRC_DIV>, (int64_t)n * n * n / (2 * kChunk));
    GR_LAUNCH(k_dfs_poisson<SRC_DIV>, g, kBlock, st, lgn, a, partials);
    return g;
}

int dfs_shift_rhs(int n, double scale, const float *A, const float *wh, const float *wl, int comp, const double *fld,
                  float *uh, float *ul, float *fh, float *fl, double *partials, cudaStream_t st)
{
    const int lgn = log2i(n);
    PoissonArgs a = {};
    a.A = A;
    a.wh = wh;
    a.wl = wl;
    a.comp = comp;
    a.scale = df_from_double_host(scale);
    a.fld = fld;
    a.uh = uh;
    a.ul = ul;
    a.fh = fh;
    a.fl = fl;
    const int g = wave_grid(k_dfs_poisson<SRC_SHIFT>, (int64_t)n * n * n / (2 * kChunk));
    GR_LAUNCH(k_dfs_poisson<SRC_SHIFT>, g, kBlock, st, lgn, a, partials);
    return g;
}

void dfs_aij(int n, double inv2h, double ih2, const double *Vx, const double *Vy, const double *Vz, const double *U,
             float *const scratch[4], float *A, float *AAh, float *AAl, cudaStream_t st)
{
    const int lgn = log2i(n);
    const int64_t N = (int64_t)n * n * n;
    GR_LAUNCH(k_dfs_split4, grid_for(N), kBlock, st, N, Vx, Vy, Vz, U, scratch[0], scratch[1], scratch[2],
              scratch[3]);
    GR_LAUNCH(k_dfs_aij, wave_grid(k_dfs_aij, N / 4), kBlock, st, lgn, df_from_double_host(inv2h), df_from_double_host(ih2),
              scratch[0], scratch[1], scratch[2], scratch[3], A, AAh, AAl);
}

int dfs_psi(int n, double h2, const double *psi, const double *s0, const float *AAh, const float *AAl, float *uh,
            float *ul, float *ah, float *al, float *bh, float *bl, float *fh, float *fl, double *partials,
            cudaStream_t st)
{
    const int lgn = log2i(n);
    const int g = wave_grid(k_dfs_psi, (int64_t)n * n * n / (2 * kChunk));
    GR_LAUNCH(k_dfs_psi, g, kBlock, st, lgn, df_from_double_host(2.0 * kPi * h2), df_from_double_host(0.125 * h2),
              psi, s0, AAh, AAl, uh, ul, ah, al, bh, bl, fh, fl, partials);
    return g;
}

int dfs_apsi(int n, double h2, const double *psi, const double *apsi, const double *s0, const double *sig,
             const float *AAh, const float *AAl, double K2, double Kdot, float *uh, float *ul, float *ah, float *al,
             float *fh, float *fl, float *m32, float *inv32, double *partials, cudaStream_t st)
{
    const int lgn = log2i(n);
    const int g = wave_grid(k_dfs_apsi, (int64_t)n * n * n / (2 * kChunk));
    GR_LAUNCH(k_dfs_apsi, g, kBlock, st, lgn, (float)h2, df_from_double_host(h2), psi, apsi, s0, sig, AAh, AAl,
              df_from_double_host(2.0 * kPi), df_from_double_host(5.0 / 12.0 * K2), df_from_double_host(Kdot), uh,
              ul, ah, al, fh, fl, m32, inv32, partials);
    return g;
}

void dfs_weight(int n, const double *psi, const double *apsi, float *wh, float *wl, cudaStream_t st)
{
    const int64_t cnt = (int64_t)n * n * n;
    GR_LAUNCH(k_dfs_weight, grid_for(cnt), kBlock, st, cnt, psi, apsi, wh, wl);
}

void dfs_store(int n, const float *uh, const float *ul, const double *sum, int dev, double *out, cudaStream_t st)
{
    const int lgn = log2i(n);
    const int64_t N = (int64_t)n * n * n;
    const int64_t threads = N / (2 * kChunk);
    if (dev)
        GR_LAUNCH(k_dfs_store<1>, wave_grid(k_dfs_store<1>, threads), kBlock, st, lgn, uh, ul, sum, 1.0 / (double)N,
                  out);
    else
        GR_LAUNCH(k_dfs_store<0>, wave_grid(k_dfs_store<0>, threads), kBlock, st, lgn, uh, ul, sum, 1.0 / (double)N,
                  out);
}

}  // namespace gr
