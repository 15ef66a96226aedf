// mg_kernels.cu - multigrid kernels on red-black split level arrays.
//
// Operators (Sec. 4.3): 7-point Laplacian (nb - 6u)/h^2 and
//   KPOISSON  L(u) = lap u
//   KHELM     L(u) = lap u - m u                          (alpha psi, Eq. sol-scheme-CMC)
//   KPSI      L(u) = lap u + 2 pi s0/psi + AA/(8 psi^7) - 2 pi rho psi^5,  psi = 1 + u
//                                                         (Eq. sol-scheme-H-constraint)
// Relaxation: red-black Gauss-Seidel, one Newton step per cell for KPSI (Sec. 4.3.2).
// Transfers: R = average of the 8 children, P = cell-centred trilinear (3/4, 1/4).
#include "gr_internal.cuh"
#include "coarse_tail.cuh"

namespace gr {
namespace {

inline int grid_for(int64_t work)
{
    int64_t b = (work + kBlock - 1) / kBlock;
    const int64_t cap = 152 * 16;  // grid-stride beyond 16 resident blocks per SM
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

inline int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// split-layout index of natural coordinates on a level of extent 2^lgn
__device__ __forceinline__ int64_t sidx(int lgn, int i, int j, int k)
{
    const int64_t half = (int64_t)1 << (3 * lgn - 1);
    return (int64_t)((i + j + k) & 1) * half + ((((int64_t)i << lgn) + j) << (lgn - 1)) + (k >> 1);
}

// 32-bit variant (grids up to 1024^3 have fewer than 2^31 cells)
__device__ __forceinline__ int sidx32(int lgn, int i, int j, int k)
{
    return (((i + j + k) & 1) << (3 * lgn - 1)) + ((((i << lgn) + j) << (lgn - 1)) + (k >> 1));
}

// natural coordinates of split index t
__device__ __forceinline__ void scoord(int lgn, int64_t t, int &i, int &j, int &k)
{
    const int n1 = (1 << lgn) - 1, h1 = (1 << (lgn - 1)) - 1;
    const int c = (int)(t >> (3 * lgn - 1));
    const int q = (int)(t & h1);
    j = (int)((t >> (lgn - 1)) & n1);
    i = (int)((t >> (2 * lgn - 1)) & n1);
    k = 2 * q + ((i + j + c) & 1);
}

template <typename T>
__device__ __forceinline__ T nbsum(const T *__restrict__ u, int lgn, int i, int j, int k)
{
    const int m = (1 << lgn) - 1;
    return u[sidx(lgn, (i + 1) & m, j, k)] + u[sidx(lgn, (i - 1) & m, j, k)] + u[sidx(lgn, i, (j + 1) & m, k)] +
           u[sidx(lgn, i, (j - 1) & m, k)] + u[sidx(lgn, i, j, (k + 1) & m)] + u[sidx(lgn, i, j, (k - 1) & m)];
}

// L(u) at one cell: u value uc, neighbour sum nb, coefficients at the cell
template <typename T, int KIND>
__device__ __forceinline__ T op_cell(T uc, T nb, T ih2, T c0, T c1, T rho)
{
    T lap = (nb - T(6) * uc) * ih2;
    if (KIND == KPOISSON) return lap;
    if (KIND == KHELM) return lap - c0 * uc;
    const double v = 1.0 + (double)uc, iv = 1.0 / v, iv2 = iv * iv, iv4 = iv2 * iv2;
    const double v2 = v * v, v4 = v2 * v2;
    return (T)((double)lap + 2.0 * kPi * (double)c0 * iv + 0.125 * (double)c1 * (iv4 * iv2 * iv) -
               2.0 * kPi * (double)rho * (v4 * v));
}

template <typename T, int KIND>
__device__ __forceinline__ T resid_cell(const T *__restrict__ u, const T *__restrict__ f, const T *__restrict__ c0,
                                        const T *__restrict__ c1, int lgn, int i, int j, int k, T ih2, T rho)
{
    const int64_t id = sidx(lgn, i, j, k);
    const T a0 = (KIND == KPOISSON) ? T(0) : c0[id];
    const T a1 = (KIND == KPSI) ? c1[id] : T(0);
    return op_cell<T, KIND>(u[id], nbsum(u, lgn, i, j, k), ih2, a0, a1, rho) - f[id];
}

// ---------------------------------------------------------------- sweep
template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock)
    k_sweep(int lgn, T *__restrict__ u, const T *__restrict__ f, const T *__restrict__ c0, const T *__restrict__ c1,
            T h2, T ih2, T rho, int color)
{
    pdl_begin();
    const int lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int64_t half = (int64_t)1 << (3 * lgn - 1);
    const int64_t off = color ? half : 0;
    T *__restrict__ own = u + off;
    const T *__restrict__ oth = u + (half - off);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < half; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t & mh);
        const int j = (int)((t >> lgh) & mn);
        const int i = (int)(t >> (lgh + lgn));
        const int p = (i + j + color) & 1;
        const int64_t r0 = t - q;
        const int64_t ri = (int64_t)j << lgh;
        const int64_t rip = ((int64_t)((i + 1) & mn) << (lgn + lgh)) + ri;
        const int64_t rim = ((int64_t)((i - 1) & mn) << (lgn + lgh)) + ri;
        const int64_t rj = (int64_t)i << (lgn + lgh);
        const int64_t rjp = rj + ((int64_t)((j + 1) & mn) << lgh);
        const int64_t rjm = rj + ((int64_t)((j - 1) & mn) << lgh);
        const int qs = (q + (p ? 1 : -1)) & mh;
        const T nb = oth[rip + q] + oth[rim + q] + oth[rjp + q] + oth[rjm + q] + oth[r0 + q] + oth[r0 + qs];
        const int64_t c = off + t;
        if (KIND == KPOISSON) {
            own[t] = (nb - h2 * f[c]) * T(1.0 / 6.0);
        } else if (KIND == KHELM) {
            own[t] = (nb - h2 * f[c]) * c1[c];  // c1 = 1/(6 + h^2 m)
        } else {
            const double uc = (double)own[t];
            const double v = 1.0 + uc, iv = 1.0 / v, iv2 = iv * iv, iv4 = iv2 * iv2, iv8 = iv4 * iv4;
            const double v2 = v * v, v4 = v2 * v2;
            const double s0 = (double)c0[c], aa = (double)c1[c], ihd = (double)ih2, rh = (double)rho;
            const double g = ((double)nb - 6.0 * uc) * ihd + 2.0 * kPi * s0 * iv + 0.125 * aa * (iv4 * iv2 * iv) -
                             2.0 * kPi * rh * (v4 * v) - (double)f[c];
            const double dg = -6.0 * ihd - 2.0 * kPi * s0 * iv2 - 0.875 * aa * iv8 - 10.0 * kPi * rh * v4;
            own[t] = (T)(uc - g / dg);
        }
    }
}

// FP32 colour pass, four consecutive half-indices per thread (float4): the
// rows (i +- 1, j), (i, j +- 1) and the own row of the other colour are read
// as float4; the shifted own-row neighbour q + (p ? 1 : -1) takes one extra
// scalar load.  Needs n >= 8 (rows of at least four half-indices).
template <int KIND>
__global__ void __launch_bounds__(kBlock) k_sweep4(int lgn, float *__restrict__ u, const float *__restrict__ f,
                                                   const float *__restrict__ c1, float h2, int color, int rev)
{
    pdl_begin();
    const int lgh = lgn - 1, mn = (1 << lgn) - 1, mh = (1 << lgh) - 1;
    const int64_t half = (int64_t)1 << (3 * lgn - 1);
    const int64_t off = color ? half : 0;
    float *__restrict__ own = u + off;
    const float *__restrict__ oth = u + (half - off);
    const int64_t nvec = half >> 2;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvec; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (rev ? nvec - 1 - v : v) << 2;
        const int q = (int)(t & mh);
        const int j = (int)((t >> lgh) & mn);
        const int i = (int)(t >> (lgh + lgn));
        const int p = (i + j + color) & 1;
        const int64_t r0 = t - q;
        const int64_t ri = (int64_t)j << lgh;
        const int64_t rip = ((int64_t)((i + 1) & mn) << (lgn + lgh)) + ri;
        const int64_t rim = ((int64_t)((i - 1) & mn) << (lgn + lgh)) + ri;
        const int64_t rj = (int64_t)i << (lgn + lgh);
        const int64_t rjp = rj + ((int64_t)((j + 1) & mn) << lgh);
        const int64_t rjm = rj + ((int64_t)((j - 1) & mn) << lgh);
        const float4 A = *reinterpret_cast<const float4 *>(oth + rip + q);
        const float4 B = *reinterpret_cast<const float4 *>(oth + rim + q);
        const float4 C = *reinterpret_cast<const float4 *>(oth + rjp + q);
        const float4 D = *reinterpret_cast<const float4 *>(oth + rjm + q);
        const float4 E = *reinterpret_cast<const float4 *>(oth + r0 + q);
        const float4 F = *reinterpret_cast<const float4 *>(f + off + t);
        const float x = oth[r0 + ((q + (p ? 4 : -1)) & mh)];
        const float4 Sh = p ? make_float4(E.y, E.z, E.w, x) : make_float4(x, E.x, E.y, E.z);
        float4 nb;
        nb.x = A.x + B.x + C.x + D.x + E.x + Sh.x;
        nb.y = A.y + B.y + C.y + D.y + E.y + Sh.y;
        nb.z = A.z + B.z + C.z + D.z + E.z + Sh.z;
        nb.w = A.w + B.w + C.w + D.w + E.w + Sh.w;
        // nb - h^2 f as one fused multiply-add (the fused three-pass kernel,
        // smooth3.cu, forms it the same way, bit for bit)
        float4 out;
        if (KIND == KPOISSON) {
            const float s6 = 1.0f / 6.0f;
            out = make_float4(__fmaf_rn(-h2, F.x, nb.x) * s6, __fmaf_rn(-h2, F.y, nb.y) * s6,
                              __fmaf_rn(-h2, F.z, nb.z) * s6, __fmaf_rn(-h2, F.w, nb.w) * s6);
        } else {
            const float4 G = *reinterpret_cast<const float4 *>(c1 + off + t);
            out = make_float4(__fmaf_rn(-h2, F.x, nb.x) * G.x, __fmaf_rn(-h2, F.y, nb.y) * G.y,
                              __fmaf_rn(-h2, F.z, nb.z) * G.z, __fmaf_rn(-h2, F.w, nb.w) * G.w);
        }
        *reinterpret_cast<float4 *>(own + t) = out;
    }
}

// ---------------------------------------------------------------- residual + restriction
// One thread per coarse cell (I, J, K).  Its 8 children sit at half-index K
// of the fine rows (2I + a, 2J + b), a, b in {0, 1}; their residuals need the
// 32 values of those rows at k = 2K - 1 .. 2K + 2 and of the 8 side rows at
// k = 2K, 2K + 1, which are loaded once into registers.  In a fine row (i, j)
// the value at k = 2K + c has colour (i + j + c) & 1 and half-index K - 1,
// K, K or K + 1 for c = -1, 0, 1, 2.
// RED = 1: right after a black Gauss-Seidel pass of a linear equation the
// black cells' residuals are zero up to rounding, so only the four red
// children are evaluated (the black ones count as zero in the average); the
// loads that only black children need are then dead and dropped.
// FIRST = 1 (correction form): instead of zeroing the coarse correction, write
// the result of the coarse level's first red relaxation from zero,
// -h_c^2 fc / 6 (KPOISSON) or -h_c^2 fc cinv (KHELM, cinv = 1/(6 + h_c^2 m_c)),
// on red coarse cells and 0 on black ones, so that pass can be skipped.
template <typename T, int KIND, int FAS, int RED = 0, int FIRST = 0>
__global__ void __launch_bounds__(kBlock)
    k_resid_restrict(int lgf, const T *__restrict__ u, const T *__restrict__ f, const T *__restrict__ c0,
                     const T *__restrict__ c1, T ih2, T rho, T *__restrict__ uc, T *__restrict__ fc,
                     T *__restrict__ urc, const T *__restrict__ cinv = nullptr, T h2c = T(0), int rev = 0)
{
    pdl_begin();
    const int lgc = lgf - 1;
    const int mf = (1 << lgf) - 1, mc = (1 << lgc) - 1;
    const int half = 1 << (3 * lgf - 1);
    const int ncells = 1 << (3 * lgc);
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < ncells; tt += gridDim.x * blockDim.x) {
        const int t = rev ? ncells - 1 - tt : tt;
        const int K = t & mc, J = (t >> lgc) & mc, I = t >> (2 * lgc);
        const int qm = (K - 1) & mc, qp = (K + 1) & mc;
        T v[4][4][4];  // v[a + 1][b + 1][c + 1]
#pragma unroll
        for (int a = -1; a <= 2; a++)
#pragma unroll
            for (int b = -1; b <= 2; b++) {
                if ((a == -1 || a == 2) && (b == -1 || b == 2)) continue;
                const int i = (2 * I + a) & mf, j = (2 * J + b) & mf;
                const int row = ((i << lgf) + j) << lgc;
                const int c0h = ((i + j) & 1) ? half : 0, c1h = half - c0h;  // colour of k even / odd
                const bool central = a >= 0 && a <= 1 && b >= 0 && b <= 1;
                v[a + 1][b + 1][1] = u[c0h + row + K];
                v[a + 1][b + 1][2] = u[c1h + row + K];
                if (central) {
                    v[a + 1][b + 1][0] = u[c1h + row + qm];  // k = 2K - 1 (odd)
                    v[a + 1][b + 1][3] = u[c0h + row + qp];  // k = 2K + 2 (even)
                }
            }
        T s = T(0), su = T(0);
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const int row = (((2 * I + a) << lgf) + 2 * J + b) << lgc;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    if (RED && ((a + b + c) & 1)) continue;
                    const int id = (((a + b + c) & 1) ? half : 0) + row + K;
                    const T uc0 = v[a + 1][b + 1][c + 1];
                    const T nb = v[a + 2][b + 1][c + 1] + v[a][b + 1][c + 1] + v[a + 1][b + 2][c + 1] +
                                 v[a + 1][b][c + 1] + v[a + 1][b + 1][c + 2] + v[a + 1][b + 1][c];
                    const T a0 = (KIND == KPOISSON) ? T(0) : c0[id];
                    const T a1 = (KIND == KPSI) ? c1[id] : T(0);
                    s += op_cell<T, KIND>(uc0, nb, ih2, a0, a1, rho) - f[id];
                    if (FAS) su += uc0;
                }
            }
        const int cid = sidx32(lgc, I, J, K);
        if (FAS) {
            fc[cid] = T(0.125) * s;
            uc[cid] = T(0.125) * su;
            urc[cid] = T(0.125) * su;
        } else {
            const T rc = -(T(0.125) * s);
            fc[cid] = rc;
            T e0 = T(0);
            if (FIRST && !((I + J + K) & 1)) e0 = -h2c * rc * (KIND == KHELM ? cinv[cid] : T(1.0 / 6.0));
            uc[cid] = e0;
        }
    }
}

// FP32 red-children restriction (correction form, after a black pass), one
// thread per pair of coarse cells K = 2Q, 2Q + 1 of coarse row (I, J): their
// red children lie at fine k = 4Q + d, d = 0..3, of the four central fine rows
// (2I + a, 2J + b).  Per central row the six values at d = -1 .. 4 are two
// two-element vectors and two scalars (one colour holds even, the other odd k);
// each of the eight side rows (a or b in {-1, 2}) contributes the two black
// values facing the red children of its central neighbour, one vector.  About
// half the loads and a third of the index arithmetic of one thread per coarse
// cell.  FIRST as in k_resid_restrict.
template <int KIND, int FIRST>
__global__ void __launch_bounds__(kBlock, KIND == KPOISSON ? 5 : 4)
    k_restrict_red2(int lgf, const float *__restrict__ e, const float *__restrict__ r, const float *__restrict__ m,
                    float ih2, float *__restrict__ ec, float *__restrict__ rc, const float *__restrict__ cinv,
                    float h2c, int rev)
{
    pdl_begin();
    using V2 = float2;
    const int lgc = lgf - 1, mc = (1 << lgc) - 1, hcl = lgc - 1, mq = (1 << hcl) - 1;
    const int mf = (1 << lgf) - 1, mhf = (1 << (lgf - 1)) - 1;
    const int halff = 1 << (3 * lgf - 1), halfc = 1 << (3 * lgc - 1);
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < halfc; tt += gridDim.x * blockDim.x) {
        const int t = rev ? halfc - 1 - tt : tt;
        const int Q = t & mq, J = (t >> hcl) & mc, I = t >> (hcl + lgc);
        const int h0 = 2 * Q;  // fine half-index of k = 4Q
        auto base = [&](int a, int b) {
            const int fi = (2 * I + a) & mf, fj = (2 * J + b) & mf;
            return ((fi << lgf) + fj) << (lgf - 1);
        };
        // central rows: c[a][b][d + 1] = e at k = 4Q + d, d = -1 .. 4
        float c[2][2][6];
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const int rb = base(a, b);
                const int pr = (a + b) & 1;  // colour of even k in this row
                const int ev = pr ? halff : 0, od = halff - ev;
                const V2 E = *reinterpret_cast<const V2 *>(e + ev + rb + h0);  // k = 4Q, 4Q + 2
                const V2 O = *reinterpret_cast<const V2 *>(e + od + rb + h0);  // k = 4Q + 1, 4Q + 3
                c[a][b][1] = E.x;
                c[a][b][3] = E.y;
                c[a][b][2] = O.x;
                c[a][b][4] = O.y;
                c[a][b][0] = e[od + rb + ((h0 - 1) & mhf)];  // k = 4Q - 1
                c[a][b][5] = e[ev + rb + ((h0 + 2) & mhf)];  // k = 4Q + 4
            }
        // side rows: the black values at the red children's k of the adjacent central row
        // si[b][0]: row (-1, b), si[b][1]: row (2, b); sj[a][0]: row (a, -1), sj[a][1]: row (a, 2)
        V2 si[2][2], sj[2][2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            si[q][0] = *reinterpret_cast<const V2 *>(e + halff + base(-1, q) + h0);
            si[q][1] = *reinterpret_cast<const V2 *>(e + halff + base(2, q) + h0);
            sj[q][0] = *reinterpret_cast<const V2 *>(e + halff + base(q, -1) + h0);
            sj[q][1] = *reinterpret_cast<const V2 *>(e + halff + base(q, 2) + h0);
        }
        float s[2] = {0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const int pr = (a + b) & 1;  // red children of this row: d = pr, pr + 2
                const int rb = base(a, b);
                const V2 R = *reinterpret_cast<const V2 *>(r + rb + h0);  // red r at d = pr, pr + 2
                V2 M = make_float2(0.0f, 0.0f);
                if (KIND == KHELM) M = *reinterpret_cast<const V2 *>(m + rb + h0);
#pragma unroll
                for (int w = 0; w < 2; w++) {
                    const int d = pr + 2 * w;
                    const float uc = c[a][b][d + 1];
                    // i neighbours: a - 1 and a + 1 (a side row when outside 0..1)
                    const float ia = a == 0 ? (w ? si[b][0].y : si[b][0].x) : c[0][b][d + 1];
                    const float ib = a == 1 ? (w ? si[b][1].y : si[b][1].x) : c[1][b][d + 1];
                    const float ja = b == 0 ? (w ? sj[a][0].y : sj[a][0].x) : c[a][0][d + 1];
                    const float jb = b == 1 ? (w ? sj[a][1].y : sj[a][1].x) : c[a][1][d + 1];
                    const float nb = ia + ib + ja + jb + c[a][b][d] + c[a][b][d + 2];
                    float lap = (nb - 6.0f * uc) * ih2;
                    if (KIND == KHELM) lap -= (w ? M.y : M.x) * uc;
                    s[w] += lap - (w ? R.y : R.x);
                }
            }
        const int off = ((I << lgc) + J) << hcl;
        const int c0 = (I + J) & 1;  // colour of coarse K = 2Q
#pragma unroll
        for (int w = 0; w < 2; w++) {
            const int cid = ((c0 ^ w) ? halfc : 0) + off + Q;
            const float rcv = -(0.125f * s[w]);
            rc[cid] = rcv;
            float e0 = 0.0f;
            if (FIRST && !(c0 ^ w)) e0 = -h2c * rcv * (KIND == KHELM ? cinv[cid] : (1.0f / 6.0f));
            ec[cid] = e0;
        }
    }
}

__global__ void __launch_bounds__(kBlock)
    k_fas_rhs(int lgc, const double *__restrict__ uc, double *__restrict__ fc, const double *__restrict__ c0,
              const double *__restrict__ c1, double ih2, double rho)
{
    pdl_begin();
    const int64_t ncells = (int64_t)1 << (3 * lgc);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncells;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgc, t, i, j, k);
        fc[t] = op_cell<double, KPSI>(uc[t], nbsum(uc, lgc, i, j, k), ih2, c0[t], c1[t], rho) - fc[t];
    }
}

__global__ void k_fas_diff(int64_t cnt, double *__restrict__ uc, const double *__restrict__ urc)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        uc[t] -= urc[t];
}

// ---------------------------------------------------------------- prolongation
// One thread per pair of coarse cells K = 2Q, 2Q + 1 of coarse row (I, J):
// the 3 x 3 coarse rows around it, at K - 1 .. K + 2, give the 16 children by
// separable trilinear interpolation (3/4 from the parent, 1/4 from the
// neighbour on the child's side, per axis).  The children lie at fine
// k = 4Q .. 4Q + 3 of the fine rows (2I + a, 2J + b); per fine row the two
// red and the two black children are adjacent half-indices 2Q, 2Q + 1 of
// their colour, so each colour takes one two-element vector update.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// BLACK = 1 corrects the black children only: when a red Gauss-Seidel pass of
// a linear equation follows, the red values are overwritten without being
// read (the point update does not use the old value), so their correction
// would be dead work.
template <typename T, int BLACK = 0>
__global__ void __launch_bounds__(kBlock) k_prolong_add(int lgf, T *__restrict__ u, const T *__restrict__ uc, int rev = 0)
{
    pdl_begin();
    using V2 = typename Vec2<T>::type;
    const int lgc = lgf - 1, mc = (1 << lgc) - 1, hc = lgc - 1, mq = (1 << hc) - 1;
    const int halfc = 1 << (3 * lgc - 1), halff = 1 << (3 * lgf - 1);
    const T w0 = T(0.25), w1 = T(0.75);
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < halfc; tt += gridDim.x * blockDim.x) {
        const int t = rev ? halfc - 1 - tt : tt;
        const int Q = t & mq, J = (t >> hc) & mc, I = t >> (hc + lgc);
        const int Qm = (Q - 1) & mq, Qp = (Q + 1) & mq;
        T z[3][3][4];  // interpolated along k: fine k = 4Q + m
#pragma unroll
        for (int x = 0; x < 3; x++)
#pragma unroll
            for (int y = 0; y < 3; y++) {
                const int Ii = (I + x - 1) & mc, Jj = (J + y - 1) & mc;
                const int base = ((Ii << lgc) + Jj) << hc;
                const int ce = ((Ii + Jj) & 1) ? halfc : 0;  // colour array of the even coarse k
                const int co = halfc - ce;
                const T cm = uc[co + base + Qm];   // K - 1 = 2Q - 1
                const T c0 = uc[ce + base + Q];    // 2Q
                const T c1 = uc[co + base + Q];    // 2Q + 1
                const T cp = uc[ce + base + Qp];   // 2Q + 2
                z[x][y][0] = w0 * cm + w1 * c0;
                z[x][y][1] = w1 * c0 + w0 * c1;
                z[x][y][2] = w0 * c0 + w1 * c1;
                z[x][y][3] = w1 * c1 + w0 * cp;
            }
#pragma unroll
        for (int b = 0; b < 2; b++) {
            T yv[3][4];  // along j
#pragma unroll
            for (int x = 0; x < 3; x++)
#pragma unroll
                for (int m = 0; m < 4; m++)
                    yv[x][m] = b ? (w1 * z[x][1][m] + w0 * z[x][2][m]) : (w0 * z[x][0][m] + w1 * z[x][1][m]);
#pragma unroll
            for (int a = 0; a < 2; a++) {
                T val[4];  // along i
#pragma unroll
                for (int m = 0; m < 4; m++) val[m] = a ? (w1 * yv[1][m] + w0 * yv[2][m]) : (w0 * yv[0][m] + w1 * yv[1][m]);
                const int row = (((2 * I + a) << lgf) + 2 * J + b) << (lgf - 1);
                // fine cell 4Q + m has colour (a + b + m) & 1 and half-index 2Q + (m >> 1)
                const int p = (a + b) & 1;
                V2 *blk = reinterpret_cast<V2 *>(u + halff + row + 2 * Q);
                V2 k = *blk;
                k.x += val[1 - p];
                k.y += val[3 - p];
                *blk = k;
                if (!BLACK) {
                    V2 *red = reinterpret_cast<V2 *>(u + row + 2 * Q);
                    V2 r = *red;
                    r.x += val[p];
                    r.y += val[2 + p];
                    *red = r;
                }
            }
        }
    }
}

// black-children prolongation over four coarse cells K = 4P .. 4P + 3 of a
// coarse row per thread: fine k = 8P .. 8P + 7, whose black cells in each of
// the four fine rows are one float4 of the black half-array; the coarse row's
// values K = 4P - 1 .. 4P + 4 are two float2 and two scalar loads per
// neighbouring coarse row
__global__ void __launch_bounds__(kBlock, 5) k_prolong_black4(int lgf, float *__restrict__ u, const float *__restrict__ uc,
                                                           int rev)
{
    pdl_begin();
    const int lgc = lgf - 1, mc = (1 << lgc) - 1, hc = lgc - 1, mq = (1 << hc) - 1;
    const int halfc = 1 << (3 * lgc - 1), halff = 1 << (3 * lgf - 1);
    const int lp = lgc - 2, mp = (1 << lp) - 1;  // P: coarse row / 4
    const int cnt = 1 << (3 * lgc - 2);
    const float w0 = 0.25f, w1 = 0.75f;
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < cnt; tt += gridDim.x * blockDim.x) {
        const int t = rev ? cnt - 1 - tt : tt;
        const int P = t & mp, J = (t >> lp) & mc, I = t >> (lp + lgc);
        float z[3][3][8];
#pragma unroll
        for (int x = 0; x < 3; x++)
#pragma unroll
            for (int y = 0; y < 3; y++) {
                const int Ii = (I + x - 1) & mc, Jj = (J + y - 1) & mc;
                const int base = ((Ii << lgc) + Jj) << hc;
                const int ce = ((Ii + Jj) & 1) ? halfc : 0;  // colour array of the even coarse K
                const int co = halfc - ce;
                const float2 ev = *reinterpret_cast<const float2 *>(uc + ce + base + 2 * P);  // K = 4P, 4P + 2
                const float2 od = *reinterpret_cast<const float2 *>(uc + co + base + 2 * P);  // K = 4P + 1, 4P + 3
                const float om = uc[co + base + ((2 * P - 1) & mq)];                         // K = 4P - 1
                const float ep = uc[ce + base + ((2 * P + 2) & mq)];                         // K = 4P + 4
                const float c[6] = {om, ev.x, od.x, ev.y, od.y, ep};
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    const int t0 = (m >> 1) + 1, t1 = (m & 1) ? t0 + 1 : t0 - 1;
                    z[x][y][m] = w1 * c[t0] + w0 * c[t1];
                }
            }
#pragma unroll
        for (int b = 0; b < 2; b++) {
            float yv[3][8];
#pragma unroll
            for (int x = 0; x < 3; x++)
#pragma unroll
                for (int m = 0; m < 8; m++)
                    yv[x][m] = b ? (w1 * z[x][1][m] + w0 * z[x][2][m]) : (w0 * z[x][0][m] + w1 * z[x][1][m]);
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const int kp = (a + b + 1) & 1;  // parity of the black fine k in this row
                float val[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int m = kp + 2 * q;
                    val[q] = a ? (w1 * yv[1][m] + w0 * yv[2][m]) : (w0 * yv[0][m] + w1 * yv[1][m]);
                }
                const int row = (((2 * I + a) << lgf) + 2 * J + b) << (lgf - 1);
                float4 *blk = reinterpret_cast<float4 *>(u + halff + row + 4 * P);
                float4 k4 = *blk;
                k4.x += val[0];
                k4.y += val[1];
                k4.z += val[2];
                k4.w += val[3];
                *blk = k4;
            }
        }
    }
}


// ---------------------------------------------------------------- 2^3 level
// Linear kinds: the exact solve (coarsest_exact).  KPSI: Newton red-black
// sweeps, each followed by the zero-mode shift.
template <typename T, int KIND>
__global__ void k_coarsest(T *__restrict__ u, T *__restrict__ f, const T *__restrict__ c0, const T *__restrict__ c1,
                           double h2, double ih2, double rho)
{
    pdl_begin();
    __shared__ double su[8], sf[8], s0[8], s1[8];
    const int t = threadIdx.x;
    if (t < 8) {
        su[t] = (double)u[t];
        sf[t] = (double)f[t];
        s0[t] = (KIND == KPOISSON) ? 0.0 : (double)c0[t];
        s1[t] = (KIND == KPSI) ? (double)c1[t] : 0.0;
    }
    __syncthreads();
    if (KIND == KPOISSON && t == 0) {
        double m = 0.0;
        for (int q = 0; q < 8; q++) m += sf[q];
        m *= 0.125;
        for (int q = 0; q < 8; q++) sf[q] -= m;
    }
    __syncthreads();
    if (KIND != KPSI) {
        // lane x holds cell x = 4i + 2j + k, split index 4 ((i + j + k) & 1) + 2i + j
        const int x = t & 7, i = x >> 2, j = (x >> 1) & 1, k = x & 1;
        const int id = 4 * ((i + j + k) & 1) + 2 * i + j;
        const double e = coarsest_exact<KIND>(sf[id], s0[id], h2);
        if (t < 8) su[id] = e;
        __syncthreads();
    } else {
        // on 2^3 the split index of (i, j, k) is 4 c + 2 i + j; every
        // neighbour along an axis is the same cell, counted twice
        for (int sweep = 0; sweep < kCoarsestSweeps; sweep++) {
            for (int color = 0; color < 2; color++) {
                if (t < 4) {
                    const int i = t >> 1, j = t & 1;
                    const int id = 4 * color + t;
                    const int o = 4 * (color ^ 1);
                    const double nb = 2.0 * (su[o + 2 * (i ^ 1) + j] + su[o + 2 * i + (j ^ 1)] + su[o + 2 * i + j]);
                    const double uc = su[id], v = 1.0 + uc, v2 = v * v, v4 = v2 * v2;
                    const double g = (nb - 6.0 * uc) * ih2 + 2.0 * kPi * s0[id] / v + s1[id] / (8.0 * v4 * v2 * v) -
                                     2.0 * kPi * rho * v4 * v - sf[id];
                    const double dg =
                        -6.0 * ih2 - 2.0 * kPi * s0[id] / v2 - 7.0 * s1[id] / (8.0 * v4 * v4) - 10.0 * kPi * rho * v4;
                    su[id] = uc - g / dg;
                }
                __syncthreads();
            }
            // zero mode: the constant shift that zeroes the sum of the eight
            // residuals to first order, u -= sum(f - N(u)) / sum(-dN/du) (a
            // sweep damps the constant error only by 1/(1 + h^2 m / 6), slowly
            // where the non-Laplacian coefficient m is small)
            __shared__ double zr[8], zm[8];
            if (t < 8) {
                const int c = t >> 2, i = (t >> 1) & 1, j = t & 1, o = 4 * (c ^ 1);
                const double nb = 2.0 * (su[o + 2 * (i ^ 1) + j] + su[o + 2 * i + (j ^ 1)] + su[o + 2 * i + j]);
                const double uc = su[t];
                const double v = 1.0 + uc, v2 = v * v, v4 = v2 * v2;
                zr[t] = sf[t] - ((nb - 6.0 * uc) * ih2 + 2.0 * kPi * s0[t] / v + s1[t] / (8.0 * v4 * v2 * v) -
                                 2.0 * kPi * rho * v4 * v);
                zm[t] = 2.0 * kPi * s0[t] / v2 + 7.0 * s1[t] / (8.0 * v4 * v4) + 10.0 * kPi * rho * v4;
            }
            __syncthreads();
            if (t < 8) {
                double sr = 0.0, sm = 0.0;
                for (int q = 0; q < 8; q++) {
                    sr += zr[q];
                    sm += zm[q];
                }
                if (sm > 0.0) su[t] -= sr / sm;
            }
            __syncthreads();
        }
    }
    if (KIND == KPOISSON && t == 0) {
        double m = 0.0;
        for (int q = 0; q < 8; q++) m += su[q];
        m *= 0.125;
        for (int q = 0; q < 8; q++) su[q] -= m;
    }
    __syncthreads();
    if (t < 8) {
        u[t] = (T)su[t];
        f[t] = (T)sf[t];
    }
}

// ---------------------------------------------------------------- plain restriction
// coarse = 8-child average of fine (split layout), e.g. a right-hand side
template <typename T>
__global__ void __launch_bounds__(kBlock) k_restrict_avg(int lgf, const T *__restrict__ fine, T *__restrict__ coarse)
{
    pdl_begin();
    const int lgc = lgf - 1, mc = (1 << lgc) - 1;
    const int ncells = 1 << (3 * lgc);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncells; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lgc) & mc, I = t >> (2 * lgc);
        T s = T(0);
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++)
#pragma unroll
                for (int c = 0; c < 2; c++) s += fine[sidx32(lgf, 2 * I + a, 2 * J + b, 2 * K + c)];
        coarse[sidx32(lgc, I, J, K)] = T(0.125) * s;
    }
}

// ---------------------------------------------------------------- coefficients
template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock) k_restrict_coef(int lgf, const T *__restrict__ c0f, const T *__restrict__ c1f,
                                                          T *__restrict__ c0c, T *__restrict__ c1c, T h2c)
{
    pdl_begin();
    const int lgc = lgf - 1, mc = (1 << lgc) - 1;
    const int64_t ncells = (int64_t)1 << (3 * lgc);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncells;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int K = (int)(t & mc), J = (int)((t >> lgc) & mc), I = (int)(t >> (2 * lgc));
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++)
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const int64_t id = sidx(lgf, 2 * I + a, 2 * J + b, 2 * K + c);
                    s0 += c0f[id];
                    if (KIND == KPSI) s1 += c1f[id];
                }
        const int64_t cid = lgc > 0 ? sidx(lgc, I, J, K) : 0;
        c0c[cid] = T(0.125) * s0;
        if (KIND == KPSI)
            c1c[cid] = T(0.125) * s1;
        else
            c1c[cid] = T(1) / (T(6) + h2c * (T(0.125) * s0));
    }
}

template <typename T>
__global__ void k_helm_invdiag(int64_t cnt, const T *__restrict__ c0, T *__restrict__ c1, T h2)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        c1[t] = T(1) / (T(6) + h2 * c0[t]);
}

// ---------------------------------------------------------------- reductions
template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock)
    k_resid_norm(int lgn, const T *__restrict__ u, const T *__restrict__ f, const T *__restrict__ c0,
                 const T *__restrict__ c1, T ih2, T rho, double *__restrict__ partials, double *__restrict__ eps_nat)
{
    pdl_begin();
    const int64_t ncells = (int64_t)1 << (3 * lgn);
    double s2 = 0.0, su = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncells;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        const double e = (double)resid_cell<T, KIND>(u, f, c0, c1, lgn, i, j, k, ih2, rho);
        s2 += e * e;
        su += (double)u[t];
        if (eps_nat) eps_nat[((((int64_t)i << lgn) + j) << lgn) + k] = e;
    }
    block_sum2(s2, su, partials);
}

__global__ void __launch_bounds__(kBlock) k_finalize(const double *__restrict__ partials, int nblk,
                                                     double *__restrict__ out)
{
    pdl_begin();
    // one block, fixed summation order: out[0], out[1] = block_sum2's slots of block 0
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblk; q += kBlock) {
        a += partials[2 * q];
        b += partials[2 * q + 1];
    }
    block_sum2(a, b, out);
}

// cnt (<= 32) doubles from device memory to host-mapped pinned memory: the
// host reads them after a stream synchronisation without a copy-engine
// transfer, which would queue behind large copies in flight on other streams
__global__ void k_scalars_out(const double *__restrict__ src, double *dst, int cnt)
{
    pdl_begin();
    if ((int)threadIdx.x < cnt) dst[threadIdx.x] = src[threadIdx.x];
    __threadfence_system();
}

// ---------------------------------------------------------------- mixed precision
template <int KIND>
__global__ void __launch_bounds__(kBlock)
    k_mixed_resid(int lgn, const double *__restrict__ u, const double *__restrict__ f, const double *__restrict__ c0,
                  const double *__restrict__ c1, double ih2, double h2, double rho, float *__restrict__ r32,
                  float *__restrict__ m32, float *__restrict__ inv32, double *__restrict__ partials)
{
    pdl_begin();
    const int64_t ncells = (int64_t)1 << (3 * lgn);
    double s2 = 0.0, su = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncells;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        const double e = resid_cell<double, KIND>(u, f, c0, c1, lgn, i, j, k, ih2, rho);
        s2 += e * e;
        su += u[t];
        r32[t] = (float)(-e);
        if (KIND == KPSI) {
            const double v = 1.0 + u[t], iv = 1.0 / v, iv2 = iv * iv, iv4 = iv2 * iv2, v2 = v * v;
            const double mj = 2.0 * kPi * c0[t] * iv2 + 0.875 * c1[t] * (iv4 * iv4) + 10.0 * kPi * rho * (v2 * v2);
            const float mf = (float)mj;
            m32[t] = mf;
            inv32[t] = 1.0f / (6.0f + (float)h2 * mf);
        }
    }
    block_sum2(s2, su, partials);
}

__global__ void k_mixed_update(int64_t cnt, double *__restrict__ u, const float *__restrict__ e)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        u[t] += (double)e[t];
}

__global__ void k_to_float(int64_t cnt, const double *__restrict__ a, float *__restrict__ b)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}

}  // namespace

// ================================================================ launchers
template <typename T>
void sweep_colour(int kind, int n, T *u, const T *f, const T *c0, const T *c1, double h2, double ih2, double rho,
                  int color, cudaStream_t st, int rev)
{
    const int lgn = log2i(n);
    if (sizeof(T) == 4 && n >= 8 && kind != KPSI) {
        float *uf = (float *)u;
        const float *ff = (const float *)f, *cf = (const float *)c1;
        const int64_t threads = (int64_t)n * n * n / 8;
        if (kind == KPOISSON)
            GR_LAUNCH(k_sweep4<KPOISSON>, wave_grid(k_sweep4<KPOISSON>, threads), kBlock, st, lgn, uf, ff, cf,
                      (float)h2, color, rev);
        else
            GR_LAUNCH(k_sweep4<KHELM>, wave_grid(k_sweep4<KHELM>, threads), kBlock, st, lgn, uf, ff, cf, (float)h2,
                      color, rev);
        return;
    }
    const int g = grid_for((int64_t)n * n * n / 2);
    if (kind == KPOISSON)
        GR_LAUNCH((k_sweep<T, KPOISSON>), g, kBlock, st, lgn, u, f, c0, c1, (T)h2, (T)ih2, (T)rho, color);
    else if (kind == KHELM)
        GR_LAUNCH((k_sweep<T, KHELM>), g, kBlock, st, lgn, u, f, c0, c1, (T)h2, (T)ih2, (T)rho, color);
    else
        GR_LAUNCH((k_sweep<T, KPSI>), g, kBlock, st, lgn, u, f, c0, c1, (T)h2, (T)ih2, (T)rho, color);
}

template <typename T>
void resid_restrict(int kind, int nf, const T *u, const T *f, const T *c0, const T *c1, double ih2, double rho, T *uc,
                    T *fc, T *urc, int fas, cudaStream_t st)
{
    const int lgf = log2i(nf);
    const int g = grid_for((int64_t)nf * nf * nf / 8);
    if (kind == KPOISSON)
        GR_LAUNCH((k_resid_restrict<T, KPOISSON, 0>), g, kBlock, st, lgf, u, f, c0, c1, (T)ih2, (T)rho, uc, fc, urc, nullptr, T(0), 0);
    else if (kind == KHELM)
        GR_LAUNCH((k_resid_restrict<T, KHELM, 0>), g, kBlock, st, lgf, u, f, c0, c1, (T)ih2, (T)rho, uc, fc, urc, nullptr, T(0), 0);
    else if (fas)
        GR_LAUNCH((k_resid_restrict<T, KPSI, 1>), g, kBlock, st, lgf, u, f, c0, c1, (T)ih2, (T)rho, uc, fc, urc, nullptr, T(0), 0);
    else
        GR_LAUNCH((k_resid_restrict<T, KPSI, 0>), g, kBlock, st, lgf, u, f, c0, c1, (T)ih2, (T)rho, uc, fc, urc, nullptr, T(0), 0);
}

void resid_restrict_red(int kind, int nf, const float *e, const float *r, const float *m, double ih2, float *ec,
                        float *rc, const float *cinv, double h2c, cudaStream_t st, int rev)
{
    const int lgf = log2i(nf);
    const int64_t threads = (int64_t)nf * nf * nf / 8;
    const float hc = (float)h2c;
    // a fixed 16 blocks per SM: measured faster here than a single wave
    const int g = grid_for(threads);
    if (nf >= 8) {  // two coarse cells per thread
        const int g2 = grid_for(threads / 2);
#define GR_RR2(K, F) \
    GR_LAUNCH((k_restrict_red2<K, F>), g2, kBlock, st, lgf, e, r, m, (float)ih2, ec, rc, cinv, hc, rev)
        if (kind == KPOISSON) {
            if (cinv || h2c > 0) GR_RR2(KPOISSON, 1);
            else GR_RR2(KPOISSON, 0);
        } else {
            if (h2c > 0) GR_RR2(KHELM, 1);
            else GR_RR2(KHELM, 0);
        }
#undef GR_RR2
        return;
    }
#define GR_RR(K, F)                                                                                          \
    GR_LAUNCH((k_resid_restrict<float, K, 0, 1, F>), g, kBlock, st, lgf, e, r, m, nullptr, (float)ih2, 0.0f, ec, \
              rc, nullptr, cinv, hc, rev)
    if (kind == KPOISSON) {
        if (cinv || h2c > 0) GR_RR(KPOISSON, 1);
        else GR_RR(KPOISSON, 0);
    } else {
        if (h2c > 0) GR_RR(KHELM, 1);
        else GR_RR(KHELM, 0);
    }
#undef GR_RR
}

void fas_rhs(int nc, const double *uc, double *fc, const double *c0, const double *c1, double ih2, double rho,
             cudaStream_t st)
{
    GR_LAUNCH(k_fas_rhs, grid_for((int64_t)nc * nc * nc), kBlock, st, log2i(nc), uc, fc, c0, c1, ih2, rho);
}

void fas_diff(int nc, double *uc, const double *urc, cudaStream_t st)
{
    const int64_t cnt = (int64_t)nc * nc * nc;
    GR_LAUNCH(k_fas_diff, grid_for(cnt), kBlock, st, cnt, uc, urc);
}

void restrict_avg(int nf, const float *fine, float *coarse, cudaStream_t st)
{
    GR_LAUNCH((k_restrict_avg<float>), grid_for((int64_t)nf * nf * nf / 8), kBlock, st, log2i(nf), fine, coarse);
}

void prolong_add_black(int nf, float *u, const float *uc, cudaStream_t st, int rev)
{
    if (nf >= 16)
        GR_LAUNCH(k_prolong_black4, wave_grid(k_prolong_black4, (int64_t)nf * nf * nf / 32), kBlock, st, log2i(nf), u,
                  uc, rev);
    else
        GR_LAUNCH((k_prolong_add<float, 1>), wave_grid(k_prolong_add<float, 1>, (int64_t)nf * nf * nf / 16), kBlock,
                  st, log2i(nf), u, uc, rev);
}

template <typename T>
void prolong_add(int nf, T *u, const T *uc, cudaStream_t st)
{
    GR_LAUNCH((k_prolong_add<T>), wave_grid(k_prolong_add<T>, (int64_t)nf * nf * nf / 16), kBlock, st, log2i(nf), u,
              uc, 0);
}

template <typename T>
void coarsest(int kind, T *u, T *f, const T *c0, const T *c1, double h2, double ih2, double rho, cudaStream_t st)
{
    if (kind == KPOISSON)
        GR_LAUNCH((k_coarsest<T, KPOISSON>), 1, 32, st, u, f, c0, c1, h2, ih2, rho);
    else if (kind == KHELM)
        GR_LAUNCH((k_coarsest<T, KHELM>), 1, 32, st, u, f, c0, c1, h2, ih2, rho);
    else
        GR_LAUNCH((k_coarsest<T, KPSI>), 1, 32, st, u, f, c0, c1, h2, ih2, rho);
}

template <typename T>
void restrict_coef(int kind, int nf, const T *c0f, const T *c1f, T *c0c, T *c1c, double h2c, cudaStream_t st)
{
    const int g = grid_for((int64_t)nf * nf * nf / 8);
    if (kind == KPSI)
        GR_LAUNCH((k_restrict_coef<T, KPSI>), g, kBlock, st, log2i(nf), c0f, c1f, c0c, c1c, (T)h2c);
    else
        GR_LAUNCH((k_restrict_coef<T, KHELM>), g, kBlock, st, log2i(nf), c0f, c1f, c0c, c1c, (T)h2c);
}

template <typename T>
void helm_invdiag(int n, const T *c0, T *c1, double h2, cudaStream_t st)
{
    const int64_t cnt = (int64_t)n * n * n;
    GR_LAUNCH((k_helm_invdiag<T>), grid_for(cnt), kBlock, st, cnt, c0, c1, (T)h2);
}

static int red_grid(int64_t cnt)
{
    int g = grid_for(cnt);
    return g > kMaxRedBlocks ? kMaxRedBlocks : g;
}

template <typename T>
int resid_norm(int kind, int n, const T *u, const T *f, const T *c0, const T *c1, double ih2, double rho,
               double *partials, double *eps_nat, cudaStream_t st)
{
    const int lgn = log2i(n);
    const int g = red_grid((int64_t)n * n * n);
    if (kind == KPOISSON)
        GR_LAUNCH((k_resid_norm<T, KPOISSON>), g, kBlock, st, lgn, u, f, c0, c1, (T)ih2, (T)rho, partials, eps_nat);
    else if (kind == KHELM)
        GR_LAUNCH((k_resid_norm<T, KHELM>), g, kBlock, st, lgn, u, f, c0, c1, (T)ih2, (T)rho, partials, eps_nat);
    else
        GR_LAUNCH((k_resid_norm<T, KPSI>), g, kBlock, st, lgn, u, f, c0, c1, (T)ih2, (T)rho, partials, eps_nat);
    return g;
}

void finalize(const double *partials, int nblk, double *out, cudaStream_t st)
{
    GR_LAUNCH(k_finalize, 1, kBlock, st, partials, nblk, out);
}

void scalars_out(const double *src, double *dst_mapped, int cnt, cudaStream_t st)
{
    GR_LAUNCH(k_scalars_out, 1, 32, st, src, dst_mapped, cnt);
}

int mixed_resid(int kind, int n, const double *u, const double *f, const double *c0, const double *c1, double ih2,
                double h2, double rho, float *r32, float *m32, float *inv32, double *partials, cudaStream_t st)
{
    const int lgn = log2i(n);
    const int g = red_grid((int64_t)n * n * n);
    if (kind == KPOISSON)
        GR_LAUNCH((k_mixed_resid<KPOISSON>), g, kBlock, st, lgn, u, f, c0, c1, ih2, h2, rho, r32, m32, inv32, partials);
    else if (kind == KHELM)
        GR_LAUNCH((k_mixed_resid<KHELM>), g, kBlock, st, lgn, u, f, c0, c1, ih2, h2, rho, r32, m32, inv32, partials);
    else
        GR_LAUNCH((k_mixed_resid<KPSI>), g, kBlock, st, lgn, u, f, c0, c1, ih2, h2, rho, r32, m32, inv32, partials);
    return g;
}

void mixed_update(int n, double *u, const float *e, cudaStream_t st)
{
    const int64_t cnt = (int64_t)n * n * n;
    GR_LAUNCH(k_mixed_update, grid_for(cnt), kBlock, st, cnt, u, e);
}

void to_float(int64_t cnt, const double *a, float *b, cudaStream_t st)
{
    GR_LAUNCH(k_to_float, grid_for(cnt), kBlock, st, cnt, a, b);
}

#define GR_INST(T)                                                                                                  \
    template void sweep_colour<T>(int, int, T *, const T *, const T *, const T *, double, double, double, int,     \
                                  cudaStream_t, int);                                                              \
    template void resid_restrict<T>(int, int, const T *, const T *, const T *, const T *, double, double, T *, T *, \
                                    T *, int, cudaStream_t);                                                       \
    template void prolong_add<T>(int, T *, const T *, cudaStream_t);                                               \
    template void coarsest<T>(int, T *, T *, const T *, const T *, double, double, double, cudaStream_t);           \
    template void restrict_coef<T>(int, int, const T *, const T *, T *, T *, double, cudaStream_t);                \
    template void helm_invdiag<T>(int, const T *, T *, double, cudaStream_t);                                      \
    template int resid_norm<T>(int, int, const T *, const T *, const T *, const T *, double, double, double *,     \
                               double *, cudaStream_t);
GR_INST(double)
GR_INST(float)

// ================================================================ coarse tail
// Levels 16^3 down to 2^3 and back up of one FP32 correction V-cycle
// (correction form, KPOISSON or KHELM) inside one thread block, with every
// level's e, r, m and 1/(6 + h^2 m) in shared memory.  The block runs the
// same operations in the same order as the per-level kernels (red then black
// sweeps, residual-restriction, FP64 2^3 solve, trilinear prolongation), so
// the coarse levels cost one launch per cycle instead of about thirty.
namespace {

// gl: the global arrays of levels 2^3 .. 16^3 (index 0 = 2^3); e/r of 16^3
// in and out, m/inv read for KHELM.
struct TailArgs {
    float *e[4], *r[4];
    const float *m[4], *inv[4];
    float h2[4];
};

template <int KIND>
__global__ void __launch_bounds__(kTailThreads) k_coarse_tail(TailArgs g, int nu1, int nu2)
{
    pdl_begin();
    extern __shared__ float sh[];
    TailLevel L[4];
    float *res = sh;  // residual scratch of the finest tail level (16^3 cells)
    float *p = sh + (1 << 12);
#pragma unroll
    for (int l = 0; l < 4; l++) {
        const int cells = 1 << (3 * (l + 1));
        L[l].lg = l + 1;
        L[l].h2 = g.h2[l];
        L[l].ih2 = 1.0f / g.h2[l];
        L[l].e = p;
        L[l].r = p + cells;
        L[l].m = p + 2 * cells;
        L[l].inv = p + 3 * cells;
        p += 4 * cells;
        for (int t = threadIdx.x; t < cells; t += blockDim.x) {
            if (l == 3) {
                L[l].e[t] = g.e[3][t];
                L[l].r[t] = g.r[3][t];
            }
            if (KIND == KHELM) {
                L[l].m[t] = g.m[l][t];
                L[l].inv[t] = g.inv[l][t];
            }
        }
    }
    __syncthreads();
    tail_cycle<KIND>(L, res, nu1, nu2);
    for (int t = threadIdx.x; t < (1 << 12); t += blockDim.x) g.e[3][t] = L[3].e[t];
}

}  // namespace

int coarse_tail_n() { return kTailN; }

void coarse_tail(int kind, float *const *e, float *const *r, const float *const *m, const float *const *inv,
                 const double *h2, int nu1, int nu2, cudaStream_t st)
{
    TailArgs a;
    for (int l = 0; l < 4; l++) {
        a.e[l] = e[l];
        a.r[l] = r[l];
        a.m[l] = m[l];
        a.inv[l] = inv[l];
        a.h2[l] = (float)h2[l];
    }
    const size_t smem = sizeof(float) * (4096 + 4 * (8 + 64 + 512 + 4096));  // residual scratch + e, r, m, inv
    // once per kernel (function-local statics are initialised once, even with several host threads)
    if (kind == KPOISSON) {
        static const bool attr = cudaFuncSetAttribute(k_coarse_tail<KPOISSON>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
        (void)attr;
        GR_LAUNCH_SMEM(k_coarse_tail<KPOISSON>, 1, kTailThreads, smem, st, a, nu1, nu2);
    } else {
        static const bool attr = cudaFuncSetAttribute(k_coarse_tail<KHELM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)smem) == cudaSuccess;
        (void)attr;
        GR_LAUNCH_SMEM(k_coarse_tail<KHELM>, 1, kTailThreads, smem, st, a, nu1, nu2);
    }
}

}  // namespace gr
