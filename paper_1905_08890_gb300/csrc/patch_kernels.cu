// patch_kernels.cu - static nested refinement patches: the kernels of the
// composite-grid FAS solve (cloud-in-cell deposit at a patch's resolution,
// parent windows, ghost interpolation, relaxation, residual, restriction,
// injection into the parent with flux matching, the solvability constant of
// the periodic Poisson-type equations, and the per-equation set-up).
//
// A patch of n^3 cells is stored natural-layout with two ghost layers,
// (n + 4)^3 values per array, index ((i + 2) m + (j + 2)) m + (k + 2), m = n + 4,
// -2 <= i, j, k < n + 2.  It refines the parent block o .. o + n/2 - 1 (per
// axis) by 2; the parent window is the (n/2 + 4)^3 block of parent cells
// o - 2 .. o + n/2 + 1, which every interpolation and correction of the
// patch reads.  The transfers and the coupling run in FP64; the relaxation
// and the residual run in FP64 (GR_PREC_FP64) or, in the mixed modes, on
// double-float pairs with the base's stencil operator, since GB300 issues
// FP64 at 1/58 of the FP32 rate and an FP64 colour pass is FP64-issue bound.
//
// The paper runs its solver on an adaptive grid (Sec. 3, Sec. 4.3) without
// stating how a refined region couples to its parent; these kernels follow
// the multilevel FAS reading: ghosts = trilinear interpolation of the parent,
// the parent takes u = R u_patch and f = L(u) - R eps_patch on the covered
// cells (FAS, Sec. 4.3.2.1), the coarse flux through each face of the
// covered block is replaced by the mean of the four fine fluxes, and the
// patch takes the parent's correction P(u_new - u_old).
#include "df64.cuh"
#include "gr_internal.cuh"
#include "df_stencil.cuh"

namespace gr {
namespace {

constexpr int PG = 2;  // ghost layers

// 32-bit: a patch array has at most (512 + 4)^3 < 2^31 cells
__device__ __forceinline__ int gxi(int m, int i, int j, int k)
{
    return ((i + PG) * m + (j + PG)) * m + (k + PG);
}

// natural and split-layout indices on the periodic base (n = 2^lgn; the
// coordinates wrap)
__device__ __forceinline__ int64_t bnat(int lgn, int i, int j, int k)
{
    const int mk = (1 << lgn) - 1;
    return ((((int64_t)(i & mk) << lgn) + (j & mk)) << lgn) + (k & mk);
}

__device__ __forceinline__ int64_t bsplit(int lgn, int i, int j, int k)
{
    const int mk = (1 << lgn) - 1;
    i &= mk, j &= mk, k &= mk;
    return ((int64_t)((i + j + k) & 1) << (3 * lgn - 1)) + ((((int64_t)i << lgn) + j) << (lgn - 1)) + (k >> 1);
}

// ---------------------------------------------------------------- base access
template <int FMT>
__device__ __forceinline__ double b_u(const PBase &B, int i, int j, int k)
{
    if (FMT == PB_NAT) return B.nat[bnat(B.lgn, i, j, k)];
    const int64_t s = bsplit(B.lgn, i, j, k);
    if (FMT == PB_SPLIT) return B.u[s];
    return join_double({B.uh[s], B.ul[s]});
}

template <int FMT>
__device__ __forceinline__ void b_set_u(const PBase &B, int i, int j, int k, double v)
{
    const int64_t s = bsplit(B.lgn, i, j, k);
    if (FMT == PB_SPLIT) {
        B.u[s] = v;
    } else {
        const df d = split_double(v);
        B.uh[s] = d.hi;
        B.ul[s] = d.lo;
    }
}

// the base right-hand side at a split index, unscaled (the double-float
// arrays hold h^2 f)
template <int FMT>
__device__ __forceinline__ double b_f(const PBase &B, int64_t s)
{
    if (FMT == PB_SPLIT) return B.f[s];
    return join_double({B.fh[s], B.fl[s]}) * B.ih2;
}

template <int FMT>
__device__ __forceinline__ void b_set_f(const PBase &B, int64_t s, double v)
{
    if (FMT == PB_SPLIT) {
        B.f[s] = v;
    } else {
        const df d = split_double(v * B.h2);
        B.fh[s] = d.hi;
        B.fl[s] = d.lo;
    }
}

// L(u) of the base equation at one cell (the oracle's operator: Poisson
// lap u; Helmholtz lap u - m u; psi lap u + 2 pi s0/psi + AA/(8 psi^7) -
// 2 pi rho psi^5 with psi = 1 + u); the double-float arrays hold the
// h^2-scaled coefficients a' = h^2 m or 2 pi h^2 s0 and b' = h^2 AA / 8
template <int FMT, int KIND>
__device__ __forceinline__ double b_op(const PBase &B, int i, int j, int k)
{
    const double u = b_u<FMT>(B, i, j, k);
    const double nb = b_u<FMT>(B, i + 1, j, k) + b_u<FMT>(B, i - 1, j, k) + b_u<FMT>(B, i, j + 1, k) +
                      b_u<FMT>(B, i, j - 1, k) + b_u<FMT>(B, i, j, k + 1) + b_u<FMT>(B, i, j, k - 1);
    const int64_t s = bsplit(B.lgn, i, j, k);
    if (FMT == PB_SPLIT) {
        const double lap = (nb - 6.0 * u) * B.ih2;
        if (KIND == KPOISSON) return lap;
        if (KIND == KHELM) return lap - B.c0[s] * u;
        const double v = 1.0 + u, v2 = v * v, v4 = v2 * v2;
        return lap + 2.0 * kPi * B.c0[s] / v + B.c1[s] / (8.0 * v4 * v2 * v) - 2.0 * kPi * B.rho * v4 * v;
    }
    double S = nb - 6.0 * u;
    if (KIND == KHELM) {
        S -= join_double({B.ah[s], B.al[s]}) * u;
    } else if (KIND == KPSI) {
        const double v = 1.0 + u, v2 = v * v, v4 = v2 * v2;
        S += join_double({B.ah[s], B.al[s]}) / v + join_double({B.bh[s], B.bl[s]}) / (v4 * v2 * v) -
             2.0 * kPi * B.rho * B.h2 * v4 * v;
    }
    return S * B.ih2;
}

// ---------------------------------------------------------------- patch access
// The working unknown of a patch is FP64 (u) or, with DF, a double-float pair
// (uh, ul: the mixed modes, where the relaxation runs in FP32 instructions).
template <bool DF>
__device__ __forceinline__ double pu_get(const PPatch &P, int64_t c)
{
    if (DF) return join_double({P.uh[c], P.ul[c]});
    return P.u[c];
}

template <bool DF>
__device__ __forceinline__ void pu_set(const PPatch &P, int64_t c, double v)
{
    if (DF) {
        const df d = split_double(v);
        P.uh[c] = d.hi;
        P.ul[c] = d.lo;
    } else {
        P.u[c] = v;
    }
}

template <bool DF>
__device__ __forceinline__ double p_nb(const PPatch &P, int i, int j, int k)
{
    const int m = P.m, mm = m * m, c = gxi(m, i, j, k);
    return pu_get<DF>(P, c + mm) + pu_get<DF>(P, c - mm) + pu_get<DF>(P, c + m) + pu_get<DF>(P, c - m) +
           pu_get<DF>(P, c + 1) + pu_get<DF>(P, c - 1);
}

// L(u) at a patch cell in FP64 (the oracle's operator; FP64 coefficients c0, c1)
template <int KIND, bool DF = false>
__device__ __forceinline__ double p_op(const PPatch &P, int i, int j, int k)
{
    const int64_t c = gxi(P.m, i, j, k);
    const double u = pu_get<DF>(P, c);
    const double lap = (p_nb<DF>(P, i, j, k) - 6.0 * u) * P.ih2;
    if (KIND == KPOISSON) return lap;
    if (KIND == KHELM) return lap - P.c0[c] * u;
    const double v = 1.0 + u, v2 = v * v, v4 = v2 * v2, iv = 1.0 / v, iv2 = iv * iv;
    return lap + 2.0 * kPi * P.c0[c] * iv + 0.125 * P.c1[c] * (iv2 * iv2 * iv2 * iv) - 2.0 * kPi * P.rho * v4 * v;
}

// whether the child patch covers cell (i, j, k)
__device__ __forceinline__ bool p_covered(const PPatch &P, int i, int j, int k)
{
    return P.cnc > 0 && (unsigned)(i - P.co[0]) < (unsigned)P.cnc && (unsigned)(j - P.co[1]) < (unsigned)P.cnc &&
           (unsigned)(k - P.co[2]) < (unsigned)P.cnc;
}

// h^2 eps = h^2 (L(u) - f) at a patch cell in double-float (the base's stencil
// operator on the pair arrays; f' = h^2 f, plus h^2 lambda where no child
// covers the cell); KPSI also the Newton inverse diagonal
template <int KIND>
__device__ __forceinline__ df p_cell_df(const PPatch &P, df lam2, int i, int j, int k, float *inv)
{
    const int m = P.m, mm = m * m;
    const int c = gxi(m, i, j, k);
    const int nb[6] = {c + mm, c - mm, c + m, c - m, c + 1, c - 1};
    float nh[6], nl[6];
#pragma unroll
    for (int q = 0; q < 6; q++) {
        nh[q] = P.uh[nb[q]];
        nl[q] = P.ul[nb[q]];
    }
    df f = {P.fh[c], P.fl[c]};
    if (P.lam && !p_covered(P, i, j, k)) f = df_add(f, lam2);
    const df a = KIND == KPOISSON ? df{0.0f, 0.0f} : df{P.ah[c], P.al[c]};
    const df b = KIND == KPSI ? df{P.bh[c], P.bl[c]} : df{0.0f, 0.0f};
    float mj = 0.0f;
    return df_cell<KIND>(nh, nl, {P.uh[c], P.ul[c]}, f, a, b, P.cpr, P.c5, &mj, inv);
}

// right-hand side of a patch cell: f, plus the solvability constant lambda
// where the child patch does not cover the cell
__device__ __forceinline__ double p_rhs(const PPatch &P, int i, int j, int k)
{
    const double f = P.f[gxi(P.m, i, j, k)];
    if (!P.lam) return f;
    return p_covered(P, i, j, k) ? f : f + *P.lam;
}

// interior cell t (0 <= t < n^3) of an n^3 patch, n = 2^lgn
__device__ __forceinline__ void p_cell(int lgn, int64_t t, int &i, int &j, int &k)
{
    const int mk = (1 << lgn) - 1;
    k = (int)(t & mk);
    j = (int)((t >> lgn) & mk);
    i = (int)(t >> (2 * lgn));
}

// trilinear interpolation of a w^3 window at patch cell (i, j, k): fine
// cell i sits in parent cell floor(i/2) (window index floor(i/2) + 2) and
// leans 1/4 towards the neighbour on the side of its half
__device__ __forceinline__ double interp(const double *win, int w, int i, int j, int k)
{
    int I[2], J[2], K[2];
    I[0] = (i >> 1) + 2;
    I[1] = I[0] + ((i & 1) ? 1 : -1);
    J[0] = (j >> 1) + 2;
    J[1] = J[0] + ((j & 1) ? 1 : -1);
    K[0] = (k >> 1) + 2;
    K[1] = K[0] + ((k & 1) ? 1 : -1);
    const double wt[2] = {0.75, 0.25};
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int c = 0; c < 2; c++) {
                s += wt[a] * wt[b] * wt[c] * win[(I[a] * w + J[b]) * w + K[c]];
            }
    return s;
}

// ---------------------------------------------------------------- deposit
// The particles whose clouds may meet a box of base cells: base cell of the
// position within [lo, lo + len) (mod n0) on every axis (the caller grows the
// box by one cell on every side for the cloud's reach); their indices are
// appended to list (order not kept), count holds how many.
__global__ void __launch_bounds__(kBlock)
    k_pselect(int64_t np, const double *__restrict__ x, double sn0, int n0, int lo0, int lo1, int lo2, int len,
              int *__restrict__ list, unsigned *__restrict__ count)
{
    pdl_begin();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool in = p < np;
    const int lo[3] = {lo0, lo1, lo2};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!in) break;
        const int c = (int)floor(x[d * np + p] * sn0);
        in = ((c - lo[d]) & (n0 - 1)) < len;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, in);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (in) list[base + __popc(mask & ((1u << lane) - 1))] = (int)p;
}

// CIC at resolution N (spacing L/N; the base deposit's formulas in plain
// FP64) onto the nw^3 window of cells O + a (mod N) of one particle
__device__ __forceinline__ void pdeposit_one(int64_t p, int64_t np, const double *__restrict__ x,
                                             const double *__restrict__ u, double mass, double L, int N, int O0,
                                             int O1, int O2, int nw, double *__restrict__ s0,
                                             double *__restrict__ sx, double *__restrict__ sy,
                                             double *__restrict__ sz, double *__restrict__ sig)
{
    // positions scaled by 1/L and N/L (multiplications: the FP64 divide is
    // the slowest FP64 instruction, and every particle passes here)
    const double iL = 1.0 / L, sN = (double)N / L, ivol = sN * sN * sN;
    const int O[3] = {O0, O1, O2};
    int r[3];
    double fplus[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double xp = x[d * np + p];
        xp -= L * floor(xp * iL);
        const double t = xp * sN - 0.5;
        const double fl = floor(t);
        fplus[d] = 1.0 - (t - fl);
        r[d] = ((int)fl - O[d]) & (N - 1);  // window coordinate of the lower cloud cell
        if (r[d] >= nw && ((r[d] + 1) & (N - 1)) >= nw) return;  // the cloud misses the window
    }
    const double ux = u[p], uy = u[np + p], uz = u[2 * np + p];
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double W = sqrt(1.0 + u2);
    const double mv = mass * ivol;
    const double q0 = mv * W, qx = mv * ux, qy = mv * uy, qz = mv * uz;
    const double qs = mv * u2 / W;
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const int ra = (r[0] + a) & (N - 1);
        if (ra >= nw) continue;
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int rb = (r[1] + b) & (N - 1);
            if (rb >= nw) continue;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int rc = (r[2] + c) & (N - 1);
                if (rc >= nw) continue;
                const double w =
                    (a ? 1.0 - fplus[0] : fplus[0]) * (b ? 1.0 - fplus[1] : fplus[1]) * (c ? 1.0 - fplus[2] : fplus[2]);
                const int64_t id = ((int64_t)ra * nw + rb) * nw + rc;
                atomicAdd(s0 + id, q0 * w);
                atomicAdd(sx + id, qx * w);
                atomicAdd(sy + id, qy * w);
                atomicAdd(sz + id, qz * w);
                atomicAdd(sig + id, qs * w);
            }
        }
    }
}

// one thread per particle, or (list given) a grid-stride loop over the count
// particles whose indices list holds
__global__ void __launch_bounds__(kBlock)
    k_pdeposit(int64_t np, const double *__restrict__ x, const double *__restrict__ u, double mass, double L, int N,
               int O0, int O1, int O2, int nw, double *__restrict__ s0, double *__restrict__ sx,
               double *__restrict__ sy, double *__restrict__ sz, double *__restrict__ sig,
               const int *__restrict__ list, const unsigned *__restrict__ count)
{
    pdl_begin();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (!list) {
        if (t < np) pdeposit_one(t, np, x, u, mass, L, N, O0, O1, O2, nw, s0, sx, sy, sz, sig);
        return;
    }
    const int64_t cnt = (int64_t)*count;
    for (int64_t e = t; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
        pdeposit_one(list[e], np, x, u, mass, L, N, O0, O1, O2, nw, s0, sx, sy, sz, sig);
}

// ---------------------------------------------------------------- windows
// win = the parent's values on the window; with dold, also dold := win - dold
// (the parent's change since dold was gathered)
// (d32, if given, receives the change rounded to FP32: the double-float
// patches add its interpolation in FP32, since it is small)
template <int FMT>
__global__ void __launch_bounds__(kBlock) k_gather_base(PBase B, int o0, int o1, int o2, int w, double *__restrict__ win,
                                                        double *__restrict__ dold, float *__restrict__ d32)
{
    pdl_begin();
    const int W = w * w * w;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < W; t += gridDim.x * blockDim.x) {
        const int x = t / (w * w), r = t - x * w * w, y = r / w, z = r - y * w;
        const double v = b_u<FMT>(B, o0 - 2 + x, o1 - 2 + y, o2 - 2 + z);
        win[t] = v;
        if (dold) {
            const double d = v - dold[t];
            dold[t] = d;
            if (d32) d32[t] = (float)d;
        }
    }
}

template <bool DF>
__global__ void __launch_bounds__(kBlock) k_gather_patch(PPatch par, int o0, int o1, int o2, int w,
                                                         double *__restrict__ win, double *__restrict__ dold,
                                                         float *__restrict__ d32)
{
    pdl_begin();
    const int W = w * w * w;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < W; t += gridDim.x * blockDim.x) {
        const int x = t / (w * w), r = t - x * w * w, y = r / w, z = r - y * w;
        const double v = pu_get<DF>(par, gxi(par.m, o0 - 2 + x, o1 - 2 + y, o2 - 2 + z));
        win[t] = v;
        if (dold) {
            const double d = v - dold[t];
            dold[t] = d;
            if (d32) d32[t] = (float)d;
        }
    }
}

// trilinear interpolation of a float window (the weights of interp)
__device__ __forceinline__ float interp32(const float *d, int w, int i, int j, int k)
{
    int I[2], J[2], K[2];
    I[0] = (i >> 1) + 2;
    I[1] = I[0] + ((i & 1) ? 1 : -1);
    J[0] = (j >> 1) + 2;
    J[1] = J[0] + ((j & 1) ? 1 : -1);
    K[0] = (k >> 1) + 2;
    K[1] = K[0] + ((k & 1) ? 1 : -1);
    const float wt[2] = {0.75f, 0.25f};
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int c = 0; c < 2; c++) s += wt[a] * wt[b] * wt[c] * d[(I[a] * w + J[b]) * w + K[c]];
    return s;
}

// interior of the patch's unknown += P(d), d the parent's change on the
// window (FP64 d, or its FP32 copy d32 for the double-float unknown)
template <bool DF>
__global__ void __launch_bounds__(kBlock)
    k_interp_in(int lgn, PPatch P, const double *__restrict__ d, const float *__restrict__ d32, int w)
{
    pdl_begin();
    const int N = 1 << (3 * lgn), m = (1 << lgn) + 2 * PG;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(lgn, t, i, j, k);
        const int64_t c = gxi(m, i, j, k);
        if (DF) {
            const df s = df_plus_f(P.uh[c], P.ul[c], interp32(d32, w, i, j, k));
            P.uh[c] = s.hi;
            P.ul[c] = s.lo;
        } else {
            P.u[c] += interp(d, w, i, j, k);
        }
    }
}

// ghost cells of a ghosted patch array = P(win): the shell of the (n + 4)^3
// block, enumerated as the six slabs i < 0, i >= n (all j, k), then 0 <= i < n
// with j < 0 or j >= n (all k), then 0 <= i, j < n with k < 0 or k >= n
template <bool DF>
__global__ void __launch_bounds__(kBlock) k_interp_ghost(int n, const double *__restrict__ win, int w, PPatch P)
{
    pdl_begin();
    const int m = n + 2 * PG;
    const int a = 2 * PG * m * m;        // i slabs
    const int b = n * 2 * PG * m;        // j slabs
    const int cnt = a + b + n * n * 2 * PG;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        int i, j, k;
        if (t < a) {
            const int s = t / (m * m), r = t - s * m * m;
            i = s < PG ? s - PG : n + s - PG;
            j = r / m - PG;
            k = r - (r / m) * m - PG;
        } else if (t < a + b) {
            const int q = t - a, s = q / (n * m), r = q - s * n * m;  // s in [0, 2 PG)
            i = r / m;
            j = s < PG ? s - PG : n + s - PG;
            k = r - i * m - PG;
        } else {
            const int q = t - a - b, s = q / (n * n), r = q - s * n * n;
            i = r / n;
            j = r - i * n;
            k = s < PG ? s - PG : n + s - PG;
        }
        pu_set<DF>(P, gxi(m, i, j, k), interp(win, w, i, j, k));
    }
}

// ---------------------------------------------------------------- relaxation, residual
// one red-black colour over the interior (local colour (i + j + k) & 1): the
// point update of the base relaxation (Newton step for psi).  DF: the update
// u += h^2 eps / (6 + h^2 m) of the double-float unknown, h^2 eps from the
// stencil operator in FP32 instructions, the divisor in FP32 (it scales a
// correction that vanishes at the fixed point)
template <int KIND, bool DF>
__global__ void __launch_bounds__(kBlock) k_pgs(PPatch P, int color)
{
    pdl_begin();
    const int half = 1 << (3 * P.lgn - 1);
    const int lh = P.lgn - 1, mk = (1 << P.lgn) - 1;
    df lam2 = {0.0f, 0.0f};
    if (DF && P.lam) lam2 = split_double(*P.lam * P.h2);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < half; t += gridDim.x * blockDim.x) {
        const int kk = t & ((1 << lh) - 1), j = (t >> lh) & mk, i = t >> (lh + P.lgn);
        const int k = 2 * kk + ((i + j + color) & 1);
        const int64_t c = gxi(P.m, i, j, k);
        if (DF) {
            float inv = 1.0f / 6.0f;
            const df e = p_cell_df<KIND>(P, lam2, i, j, k, &inv);  // h^2 eps
            if (KIND == KHELM) inv = 1.0f / (6.0f + P.ah[c]);
            const df s = df_plus_f(P.uh[c], P.ul[c], (e.hi + e.lo) * inv);
            P.uh[c] = s.hi;
            P.ul[c] = s.lo;
            continue;
        }
        const double nb = p_nb<false>(P, i, j, k);
        const double f = p_rhs(P, i, j, k);
        if (KIND == KPOISSON) {
            P.u[c] = (nb - P.h2 * f) * (1.0 / 6.0);
        } else if (KIND == KHELM) {
            P.u[c] = (nb - P.h2 * f) * P.c1[c];  // c1 = 1 / (6 + h^2 m), written by the set-up
        } else {
            // one Newton step on g(u) = L(u) - f (the oracle's update, with 1/psi formed once)
            const double u = P.u[c], w = 1.0 + u, w2 = w * w, w4 = w2 * w2, iw = 1.0 / w, iw2 = iw * iw,
                         iw4 = iw2 * iw2;
            const double c0 = P.c0[c], c1 = P.c1[c];
            const double g = (nb - 6.0 * u) * P.ih2 + 2.0 * kPi * c0 * iw + 0.125 * c1 * (iw4 * iw2 * iw) -
                             2.0 * kPi * P.rho * w4 * w - f;
            const double dg = -6.0 * P.ih2 - 2.0 * kPi * c0 * iw2 - 0.875 * c1 * (iw4 * iw4) - 10.0 * kPi * P.rho * w4;
            P.u[c] = u - g / dg;
        }
    }
}

// eps = L(u) - f on the interior (ghosted eps array) and block sums of eps^2
template <int KIND, bool DF>
__global__ void __launch_bounds__(kBlock) k_presid(PPatch P, double *__restrict__ eps, double *__restrict__ partials)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * P.lgn);
    df lam2 = {0.0f, 0.0f};
    if (DF && P.lam) lam2 = split_double(*P.lam * P.h2);
    double s2 = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(P.lgn, t, i, j, k);
        double e;
        if (DF) {
            float inv;
            e = join_double(p_cell_df<KIND>(P, lam2, i, j, k, &inv)) * P.ih2;
        } else {
            e = p_op<KIND>(P, i, j, k) - p_rhs(P, i, j, k);
        }
        eps[gxi(P.m, i, j, k)] = e;
        s2 += e * e;
    }
    block_sum2(s2, 0.0, partials);
}

// 8-child averages of u and eps over the nc^3 parent cells the patch covers
template <bool DF>
__global__ void __launch_bounds__(kBlock) k_prestrict(int n, PPatch P, const double *__restrict__ eps,
                                                      double *__restrict__ Ru, double *__restrict__ Re)
{
    pdl_begin();
    const int nc = n / 2, m = n + 2 * PG;
    const int Nc = nc * nc * nc, lc = 31 - __clz(nc), mc = nc - 1;  // nc a power of two
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        double su = 0.0, se = 0.0;
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++)
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const int64_t id = gxi(m, 2 * I + a, 2 * J + b, 2 * K + c);
                    su += pu_get<DF>(P, id);
                    se += eps[id];
                }
        Ru[t] = 0.125 * su;
        Re[t] = 0.125 * se;
    }
}

// ---------------------------------------------------------------- injection
template <int FMT>
__global__ void __launch_bounds__(kBlock) k_inject_u_base(PBase B, int o0, int o1, int o2, int nc, const double *__restrict__ Ru)
{
    pdl_begin();
    const int Nc = nc * nc * nc, lc = 31 - __clz(nc), mc = nc - 1;  // nc a power of two
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        b_set_u<FMT>(B, o0 + I, o1 + J, o2 + K, Ru[t]);
    }
}

// f = L(u) - R eps on the covered base cells (the double-float arrays store
// h^2 (f - lambda) so that the residual kernel's uniform + lambda restores
// it); block sums of f for the mean of the Poisson right-hand side
template <int FMT, int KIND>
__global__ void __launch_bounds__(kBlock) k_inject_f_base(PBase B, int o0, int o1, int o2, int nc,
                                                          const double *__restrict__ Re, const double *__restrict__ lam,
                                                          double *__restrict__ partials)
{
    pdl_begin();
    const int Nc = nc * nc * nc, lc = 31 - __clz(nc), mc = nc - 1;  // nc a power of two
    const double l = (FMT == PB_DF && lam) ? *lam : 0.0;
    double sf = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        const int i = o0 + I, j = o1 + J, k = o2 + K;
        const double f = b_op<FMT, KIND>(B, i, j, k) - Re[t];
        b_set_f<FMT>(B, bsplit(B.lgn, i, j, k), f - l);
        sf += f;
    }
    if (partials) block_sum2(sf, 0.0, partials);
}

// the base right-hand side summed over the covered cells (unscaled)
template <int FMT>
__global__ void __launch_bounds__(kBlock) k_sum_f_base(PBase B, int o0, int o1, int o2, int nc, double *__restrict__ partials)
{
    pdl_begin();
    const int Nc = nc * nc * nc, lc = 31 - __clz(nc), mc = nc - 1;  // nc a power of two
    double sf = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        sf += b_f<FMT>(B, bsplit(B.lgn, o0 + I, o1 + J, o2 + K));
    }
    block_sum2(sf, 0.0, partials);
}

template <bool DF>
__global__ void __launch_bounds__(kBlock) k_inject_u_patch(PPatch par, int o0, int o1, int o2, int nc,
                                                           const double *__restrict__ Ru)
{
    pdl_begin();
    const int Nc = nc * nc * nc, lc = 31 - __clz(nc), mc = nc - 1;  // nc a power of two
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        pu_set<DF>(par, gxi(par.m, o0 + I, o1 + J, o2 + K), Ru[t]);
    }
}

// (the double-float parent stores h^2 f as a pair)
template <int KIND, bool DF>
__global__ void __launch_bounds__(kBlock) k_inject_f_patch(PPatch par, int o0, int o1, int o2, int nc,
                                                           const double *__restrict__ Re)
{
    pdl_begin();
    const int Nc = nc * nc * nc, lc = 31 - __clz(nc), mc = nc - 1;  // nc a power of two
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc; t += gridDim.x * blockDim.x) {
        const int K = t & mc, J = (t >> lc) & mc, I = t >> (2 * lc);
        const int i = o0 + I, j = o1 + J, k = o2 + K;
        const int64_t g = gxi(par.m, i, j, k);
        const double f = p_op<KIND, DF>(par, i, j, k) - Re[t];
        if (DF) {
            const df d = split_double(f * par.h2);
            par.fh[g] = d.hi;
            par.fl[g] = d.lo;
        } else {
            par.f[g] = f;
        }
    }
}

// Flux matching on the 6 nc^2 parent cells next to the covered block: the
// coarse flux (u_in - u_out)/h_c through the shared face is replaced by the
// mean of the four fine fluxes (u_inner - u_ghost)/h_f, as the change
// corr = -(T_f - T_c)/h_c of the parent's right-hand side there; flux[q]
// keeps the correction in force.  PARENT: 0 a patch (ghosted arrays in par),
// else the base in format PARENT; DF: the patches' unknowns (and a patch
// parent's right-hand side) are double-float pairs.
__device__ __forceinline__ void shell_cell(int q, int nc, int n, int in[3], int out[3], int fi[4][3], int fg[4][3])
{
    const int per = nc * nc;
    const int face = q / per, r = q % per;
    const int ax = face >> 1, sd = (face & 1) ? 1 : -1;
    const int t1 = r / nc, t2 = r % nc;
    const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
    in[ax] = sd < 0 ? 0 : nc - 1;
    in[b1] = t1;
    in[b2] = t2;
    for (int d = 0; d < 3; d++) out[d] = in[d] + (d == ax ? sd : 0);
    for (int e = 0; e < 4; e++) {
        fi[e][ax] = sd < 0 ? 0 : n - 1;
        fg[e][ax] = sd < 0 ? -1 : n;
        fi[e][b1] = fg[e][b1] = 2 * t1 + (e >> 1);
        fi[e][b2] = fg[e][b2] = 2 * t2 + (e & 1);
    }
}

template <int PARENT, bool DF>
__global__ void __launch_bounds__(kBlock) k_reflux(PBase B, PPatch par, PPatch ch, int o0, int o1, int o2, int n,
                                                   double hc, double *__restrict__ flux)
{
    pdl_begin();
    const int nc = n / 2, m = n + 2 * PG;
    const int nq = 6 * nc * nc;
    const double hf = 0.5 * hc;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        int in[3], out[3], fi[4][3], fg[4][3];
        shell_cell(q, nc, n, in, out, fi, fg);
        const int ii = o0 + in[0], ij = o1 + in[1], ik = o2 + in[2];
        const int oi = o0 + out[0], oj = o1 + out[1], ok = o2 + out[2];
        double uin, uout;
        if (PARENT == 0) {
            uin = pu_get<DF>(par, gxi(par.m, ii, ij, ik));
            uout = pu_get<DF>(par, gxi(par.m, oi, oj, ok));
        } else {
            uin = b_u<PARENT>(B, ii, ij, ik);
            uout = b_u<PARENT>(B, oi, oj, ok);
        }
        const double Tc = (uin - uout) / hc;
        double Tf = 0.0;
        for (int e = 0; e < 4; e++)
            Tf += (pu_get<DF>(ch, gxi(m, fi[e][0], fi[e][1], fi[e][2])) -
                   pu_get<DF>(ch, gxi(m, fg[e][0], fg[e][1], fg[e][2]))) / hf;
        Tf *= 0.25;
        const double corr = -(Tf - Tc) / hc;
        const double d = corr - flux[q];
        flux[q] = corr;
        if (PARENT == 0) {
            const int64_t g = gxi(par.m, oi, oj, ok);
            if (DF) {
                const df v = split_double(join_double({par.fh[g], par.fl[g]}) + d * par.h2);
                par.fh[g] = v.hi;
                par.fl[g] = v.lo;
            } else {
                par.f[g] += d;
            }
        } else {
            const int64_t s = bsplit(B.lgn, oi, oj, ok);
            b_set_f<PARENT>(B, s, b_f<PARENT>(B, s) + d);
        }
    }
}

// The Poisson solvability constant after an injection into the base:
// m = mean of the base right-hand side with the patches at lambda, i.e.
// (sum_cov f' - sum_cov f_orig + sum_shell corr + (N - N_cov) lambda) / N
// (the original right-hand side is mean-free); lambda -= m.  sc[0] = sum_cov
// f_orig, sc[2] = sum_cov f' (finalized block sums); m goes to sc[4].
__global__ void __launch_bounds__(kBlock) k_lambda(double *__restrict__ sc, const double *__restrict__ flux, int nq,
                                                   double N, double Ncov, double *__restrict__ lam)
{
    pdl_begin();
    double s = 0.0;
    for (int q = threadIdx.x; q < nq; q += kBlock) s += flux[q];
    block_sum2(s, 0.0, sc + 6);  // sc[6] = sum of the shell corrections
    if (threadIdx.x == 0) {
        const double l = *lam;
        const double m = (sc[2] - sc[0] + sc[6] + (N - Ncov) * l) / N;
        sc[4] = m;
        *lam = l - m;
    }
}

__global__ void __launch_bounds__(kBlock) k_sub_scalar(int64_t cnt, double *__restrict__ a, const double *__restrict__ m)
{
    pdl_begin();
    const double v = *m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        a[t] -= v;
}

// ---------------------------------------------------------------- copies
// ghosted interior <- natural n^3 (+ add)
__global__ void __launch_bounds__(kBlock) k_to_ghosted(int lgn, const double *__restrict__ in, double *__restrict__ out, double add)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * lgn);
    const int m = (1 << lgn) + 2 * PG;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(lgn, t, i, j, k);
        out[gxi(m, i, j, k)] = in[t] + add;
    }
}

// the working unknown's interior <- natural n^3 (+ add)
template <bool DF>
__global__ void __launch_bounds__(kBlock) k_u_load(int lgn, const double *__restrict__ in, PPatch P, double add)
{
    pdl_begin();
    const int N = 1 << (3 * lgn);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(lgn, t, i, j, k);
        pu_set<DF>(P, gxi(P.m, i, j, k), in[t] + add);
    }
}

// natural n^3 (and the interior of the ghosted FP64 copy keep) <- the working
// unknown + add - usum[0] * scale (usum may be NULL)
template <bool DF>
__global__ void __launch_bounds__(kBlock) k_u_store(int lgn, PPatch P, double *__restrict__ out,
                                                    double *__restrict__ keep, double add,
                                                    const double *__restrict__ usum, double scale)
{
    pdl_begin();
    const int N = 1 << (3 * lgn);
    const double sh = add - (usum ? usum[0] * scale : 0.0);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(lgn, t, i, j, k);
        const int64_t g = gxi(P.m, i, j, k);
        const double v = pu_get<DF>(P, g) + sh;
        out[t] = v;
        if (keep) keep[g] = v;
    }
}

// the double-float relaxation's right-hand side and coefficients, scaled by
// h^2 as the stencil operator takes them: f' = h^2 f; Helmholtz a' = h^2 m;
// psi a' = 2 pi h^2 s0, b' = h^2 AA / 8
template <int KIND>
__global__ void __launch_bounds__(kBlock) k_pcoef_df(PPatch P)
{
    pdl_begin();
    const int N = 1 << (3 * P.lgn);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(P.lgn, t, i, j, k);
        const int64_t g = gxi(P.m, i, j, k);
        df d = split_double(P.f[g] * P.h2);
        P.fh[g] = d.hi, P.fl[g] = d.lo;
        if (KIND == KPOISSON) continue;
        d = split_double(P.c0[g] * P.h2 * (KIND == KPSI ? 2.0 * kPi : 1.0));
        P.ah[g] = d.hi, P.al[g] = d.lo;
        if (KIND == KPSI) {
            d = split_double(P.c1[g] * P.h2 * 0.125);
            P.bh[g] = d.hi, P.bl[g] = d.lo;
        }
    }
}

// ---------------------------------------------------------------- set-up
__device__ __forceinline__ int64_t gxs(int m, int i, int j, int k, int a, int s)
{
    return gxi(m, i + (a == 0 ? s : 0), j + (a == 1 ? s : 0), k + (a == 2 ? s : 0));
}

// A_ij (xx yy zz xy xz yz) at a patch cell from ghosted V, U (the base's
// stencils: 3-point first derivatives, 3-point second difference on the
// diagonal, 4-cell cross derivative; Eqs. Aij-discrete-2, U-cross-deriv)
__device__ void aij_at(int m, const double *const V[3], const double *U, double nh, int i, int j, int k, double A[6])
{
    const double i2h = 0.5 * nh, ih2 = nh * nh;
    double D[3][3];
    for (int a = 0; a < 3; a++)
        for (int l = 0; l < 3; l++) D[a][l] = (V[l][gxs(m, i, j, k, a, 1)] - V[l][gxs(m, i, j, k, a, -1)]) * i2h;
    const double divV = D[0][0] + D[1][1] + D[2][2];
    const double u0 = U[gxi(m, i, j, k)];
    for (int a = 0; a < 3; a++) {
        const double Uaa = (U[gxs(m, i, j, k, a, 1)] - 2.0 * u0 + U[gxs(m, i, j, k, a, -1)]) * ih2;
        A[a] = 2.0 * D[a][a] - 0.5 * divV + 2.0 * Uaa;
    }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int p = 0; p < 3; p++) {
        const int a = pa[p], b = pb[p];
        double s = 0.0;
        for (int sa = -1; sa <= 1; sa += 2)
            for (int sb = -1; sb <= 1; sb += 2) {
                int c[3] = {i, j, k};
                c[a] += sa;
                c[b] += sb;
                s += (double)(sa * sb) * U[gxi(m, c[0], c[1], c[2])];
            }
        A[3 + p] = D[a][b] + D[b][a] + 2.0 * s * 0.25 * ih2;
    }
}

// A_ij on the interior and the first ghost layer (what the set-ups read),
// six ghosted arrays A6[q * M + cell]
__global__ void __launch_bounds__(kBlock) k_paij(int n, double nh, PSetFld G, double *__restrict__ A6)
{
    pdl_begin();
    const int m = n + 2 * PG, e = n + 2;
    const int64_t M = (int64_t)m * m * m;
    const double *V[3] = {G.g[0], G.g[1], G.g[2]};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < e * e * e; t += gridDim.x * blockDim.x) {
        const int i = t / (e * e) - 1, r = t - (i + 1) * e * e, j = r / e - 1, k = r - (j + 1) * e - 1;
        double A[6];
        aij_at(m, V, G.g[3], nh, i, j, k, A);
        const int64_t g = gxi(m, i, j, k);
        for (int q = 0; q < 6; q++) A6[q * M + g] = A[q];
    }
}

__device__ __forceinline__ double aa_of(const double A[6])
{
    return A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + 2.0 * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]);
}

// Right-hand side and coefficients of equation eq (solve order) on a patch's
// interior (ghosted f, c0, c1), with block sums of the square of the
// reference quantity: the momentum sources 8 pi (s_i - smean); the
// divergence sources -div/4; psi: c0 = s0, c1 = AA, f = 0 (reference s0);
// alpha psi: c0 = m, c1 = 1/(6 + h^2 m), f = m - psi^5 Kdot (reference psi^5 Kdot); B^i:
// 2 d_j (alpha psi psi^-7 A^ij).  G: ghosted fields in the order V_x V_y V_z
// U psi apsi B^x B^y B^z b.
__global__ void __launch_bounds__(kBlock)
    k_pset(int eq, int lgn, double nh, PSetSrc S, PSetFld G, const double *__restrict__ A6, double smean, double K2,
           double Kdot, double *__restrict__ f, double *__restrict__ c0, double *__restrict__ c1,
           double *__restrict__ partials)
{
    pdl_begin();
    const int64_t N = (int64_t)1 << (3 * lgn);
    const int m = (1 << lgn) + 2 * PG;
    const int64_t M = (int64_t)m * m * m;
    const double i2h = 0.5 * nh;
    double s2 = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        p_cell(lgn, t, i, j, k);
        const int64_t g = gxi(m, i, j, k);
        if (eq <= 2) {
            f[g] = 8.0 * kPi * (S.s[1 + eq][t] - smean);
            s2 += f[g] * f[g];
        } else if (eq == 3 || eq == 9) {
            const int b = eq == 3 ? 0 : 6;
            double s = 0.0;
            for (int a = 0; a < 3; a++) s += G.g[b + a][gxs(m, i, j, k, a, 1)] - G.g[b + a][gxs(m, i, j, k, a, -1)];
            f[g] = -0.25 * s * i2h;
            s2 += f[g] * f[g];
        } else if (eq == 4) {
            double A[6];
            for (int q = 0; q < 6; q++) A[q] = A6[q * M + g];
            c1[g] = aa_of(A);
            c0[g] = S.s[0][t];
            f[g] = 0.0;
            s2 += S.s[0][t] * S.s[0][t];
        } else if (eq == 5) {
            double A[6];
            for (int q = 0; q < 6; q++) A[q] = A6[q * M + g];
            const double aa = aa_of(A);
            const double p = G.g[4][g], p2 = p * p, p4 = p2 * p2, p8 = p4 * p4;
            c0[g] = 2.0 * kPi / p2 * (S.s[0][t] + 2.0 * S.s[4][t] / p4) + 0.875 * aa / p8 + (5.0 / 12.0) * p4 * K2;
            c1[g] = 1.0 / (6.0 + c0[g] / (nh * nh));  // the inverse diagonal of the relaxation
            const double fk = -p4 * p * Kdot;
            s2 += fk * fk;
            f[g] = fk + c0[g];
        } else {
            const int tab[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
            double s = 0.0;
            for (int l = 0; l < 3; l++)
                for (int sg = -1; sg <= 1; sg += 2) {
                    int c[3] = {i, j, k};
                    c[l] += sg;
                    const int64_t q = gxi(m, c[0], c[1], c[2]);
                    const double p = G.g[4][q], p2 = p * p, p4 = p2 * p2;
                    s += (double)sg * G.g[5][q] / (p4 * p2 * p) * A6[tab[eq - 6][l] * M + q];
                }
            f[g] = 2.0 * s * i2h;
            s2 += f[g] * f[g];
        }
    }
    block_sum2(s2, 0.0, partials);
}

inline int blocks_for(int64_t work, int cap = kMaxRedBlocks)
{
    int64_t b = (work + kBlock - 1) / kBlock;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

inline int lg2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

// ---------------------------------------------------------------- launchers
void patch_deposit(int64_t np, const double *x, const double *u, double mass, double L, int N, const int O[3], int nw,
                   const PSetSrc &out, cudaStream_t st)
{
    if (np <= 0) return;
    const int64_t g = (np + kBlock - 1) / kBlock;
    GR_LAUNCH(k_pdeposit, (unsigned)g, kBlock, st, np, x, u, mass, L, N, O[0], O[1], O[2], nw, out.s[0], out.s[1],
              out.s[2], out.s[3], out.s[4], (const int *)nullptr, (const unsigned *)nullptr);
}

void patch_select(int64_t np, const double *x, double L, int n0, const int lo[3], int len, int *list,
                  unsigned *count, cudaStream_t st)
{
    cudaMemsetAsync(count, 0, sizeof(unsigned), st);
    if (np <= 0) return;
    const int64_t g = (np + kBlock - 1) / kBlock;
    GR_LAUNCH(k_pselect, (unsigned)g, kBlock, st, np, x, n0 / L, n0, lo[0], lo[1], lo[2], len, list, count);
}

void patch_deposit_list(int64_t np, const int *list, const unsigned *count, const double *x, const double *u,
                        double mass, double L, int N, const int O[3], int nw, const PSetSrc &out, cudaStream_t st)
{
    if (np <= 0) return;
    GR_LAUNCH(k_pdeposit, wave_grid(k_pdeposit, np), kBlock, st, np, x, u, mass, L, N, O[0], O[1], O[2], nw,
              out.s[0], out.s[1], out.s[2], out.s[3], out.s[4], list, count);
}

void patch_gather_base(int fmt, const PBase &B, const int o[3], int w, double *win, cudaStream_t st, double *dold,
                       float *d32)
{
    const int g = blocks_for((int64_t)w * w * w);
    if (fmt == PB_NAT) GR_LAUNCH(k_gather_base<PB_NAT>, g, kBlock, st, B, o[0], o[1], o[2], w, win, dold, d32);
    else if (fmt == PB_SPLIT) GR_LAUNCH(k_gather_base<PB_SPLIT>, g, kBlock, st, B, o[0], o[1], o[2], w, win, dold, d32);
    else GR_LAUNCH(k_gather_base<PB_DF>, g, kBlock, st, B, o[0], o[1], o[2], w, win, dold, d32);
}

void patch_gather_patch(const PPatch &par, bool pdf, const int o[3], int w, double *win, cudaStream_t st,
                        double *dold, float *d32)
{
    const int g = blocks_for((int64_t)w * w * w);
    if (pdf) GR_LAUNCH(k_gather_patch<true>, g, kBlock, st, par, o[0], o[1], o[2], w, win, dold, d32);
    else GR_LAUNCH(k_gather_patch<false>, g, kBlock, st, par, o[0], o[1], o[2], w, win, dold, d32);
}

void patch_interp(const PPatch &P, bool pdf, const double *win, const double *d, const float *d32, cudaStream_t st)
{
    const int n = 1 << P.lgn, m = n + 2 * PG, w = n / 2 + 4;
    const int gi = blocks_for((int64_t)n * n * n), gg = blocks_for((int64_t)m * m * m - (int64_t)n * n * n);
    if (pdf) {
        if (d) GR_LAUNCH(k_interp_in<true>, gi, kBlock, st, P.lgn, P, d, d32, w);
        GR_LAUNCH(k_interp_ghost<true>, gg, kBlock, st, n, win, w, P);
    } else {
        if (d) GR_LAUNCH(k_interp_in<false>, gi, kBlock, st, P.lgn, P, d, d32, w);
        GR_LAUNCH(k_interp_ghost<false>, gg, kBlock, st, n, win, w, P);
    }
}

void patch_gs(int kind, const PPatch &P, bool pdf, int color, cudaStream_t st)
{
    const int g = blocks_for((int64_t)1 << (3 * P.lgn - 1));
#define GR_PGS(K, D) GR_LAUNCH((k_pgs<K, D>), g, kBlock, st, P, color)
    if (pdf) {
        if (kind == KPOISSON) GR_PGS(KPOISSON, true);
        else if (kind == KHELM) GR_PGS(KHELM, true);
        else GR_PGS(KPSI, true);
    } else {
        if (kind == KPOISSON) GR_PGS(KPOISSON, false);
        else if (kind == KHELM) GR_PGS(KHELM, false);
        else GR_PGS(KPSI, false);
    }
#undef GR_PGS
}

int patch_resid(int kind, const PPatch &P, bool pdf, double *eps, double *partials, cudaStream_t st)
{
    const int g = blocks_for((int64_t)1 << (3 * P.lgn));
#define GR_PRES(K, D) GR_LAUNCH((k_presid<K, D>), g, kBlock, st, P, eps, partials)
    if (pdf) {
        if (kind == KPOISSON) GR_PRES(KPOISSON, true);
        else if (kind == KHELM) GR_PRES(KHELM, true);
        else GR_PRES(KPSI, true);
    } else {
        if (kind == KPOISSON) GR_PRES(KPOISSON, false);
        else if (kind == KHELM) GR_PRES(KHELM, false);
        else GR_PRES(KPSI, false);
    }
#undef GR_PRES
    return g;
}

void patch_restrict(const PPatch &P, bool pdf, const double *eps, double *Ru, double *Re, cudaStream_t st)
{
    const int n = 1 << P.lgn, nc = n / 2;
    const int g = blocks_for((int64_t)nc * nc * nc);
    if (pdf) GR_LAUNCH(k_prestrict<true>, g, kBlock, st, n, P, eps, Ru, Re);
    else GR_LAUNCH(k_prestrict<false>, g, kBlock, st, n, P, eps, Ru, Re);
}

void patch_inject_u_base(int fmt, const PBase &B, const int o[3], int nc, const double *Ru, cudaStream_t st)
{
    const int g = blocks_for((int64_t)nc * nc * nc);
    if (fmt == PB_SPLIT) GR_LAUNCH(k_inject_u_base<PB_SPLIT>, g, kBlock, st, B, o[0], o[1], o[2], nc, Ru);
    else GR_LAUNCH(k_inject_u_base<PB_DF>, g, kBlock, st, B, o[0], o[1], o[2], nc, Ru);
}

int patch_inject_f_base(int fmt, int kind, const PBase &B, const int o[3], int nc, const double *Re, const double *lam,
                        double *partials, cudaStream_t st)
{
    const int g = blocks_for((int64_t)nc * nc * nc);
#define GR_INJ(F, K) GR_LAUNCH((k_inject_f_base<F, K>), g, kBlock, st, B, o[0], o[1], o[2], nc, Re, lam, partials)
    if (fmt == PB_SPLIT) {
        if (kind == KPOISSON) GR_INJ(PB_SPLIT, KPOISSON);
        else if (kind == KHELM) GR_INJ(PB_SPLIT, KHELM);
        else GR_INJ(PB_SPLIT, KPSI);
    } else {
        if (kind == KPOISSON) GR_INJ(PB_DF, KPOISSON);
        else if (kind == KHELM) GR_INJ(PB_DF, KHELM);
        else GR_INJ(PB_DF, KPSI);
    }
#undef GR_INJ
    return g;
}

int patch_sum_f_base(int fmt, const PBase &B, const int o[3], int nc, double *partials, cudaStream_t st)
{
    const int g = blocks_for((int64_t)nc * nc * nc);
    if (fmt == PB_SPLIT) GR_LAUNCH(k_sum_f_base<PB_SPLIT>, g, kBlock, st, B, o[0], o[1], o[2], nc, partials);
    else GR_LAUNCH(k_sum_f_base<PB_DF>, g, kBlock, st, B, o[0], o[1], o[2], nc, partials);
    return g;
}

void patch_inject_u_patch(const PPatch &par, bool pdf, const int o[3], int nc, const double *Ru, cudaStream_t st)
{
    const int g = blocks_for((int64_t)nc * nc * nc);
    if (pdf) GR_LAUNCH(k_inject_u_patch<true>, g, kBlock, st, par, o[0], o[1], o[2], nc, Ru);
    else GR_LAUNCH(k_inject_u_patch<false>, g, kBlock, st, par, o[0], o[1], o[2], nc, Ru);
}

void patch_inject_f_patch(int kind, const PPatch &par, bool pdf, const int o[3], int nc, const double *Re,
                          cudaStream_t st)
{
    const int g = blocks_for((int64_t)nc * nc * nc);
#define GR_PINJ(K, D) GR_LAUNCH((k_inject_f_patch<K, D>), g, kBlock, st, par, o[0], o[1], o[2], nc, Re)
    if (pdf) {
        if (kind == KPOISSON) GR_PINJ(KPOISSON, true);
        else if (kind == KHELM) GR_PINJ(KHELM, true);
        else GR_PINJ(KPSI, true);
    } else {
        if (kind == KPOISSON) GR_PINJ(KPOISSON, false);
        else if (kind == KHELM) GR_PINJ(KHELM, false);
        else GR_PINJ(KPSI, false);
    }
#undef GR_PINJ
}

void patch_reflux(int parent_fmt, const PBase &B, const PPatch &par, const PPatch &ch, bool pdf, const int o[3],
                  double hc, double *flux, cudaStream_t st)
{
    const int n = 1 << ch.lgn, nc = n / 2;
    const int g = blocks_for((int64_t)6 * nc * nc);
#define GR_RFX(F, D) GR_LAUNCH((k_reflux<F, D>), g, kBlock, st, B, par, ch, o[0], o[1], o[2], n, hc, flux)
    if (pdf) {
        if (parent_fmt < 0) GR_RFX(0, true);
        else if (parent_fmt == PB_SPLIT) GR_RFX(PB_SPLIT, true);
        else GR_RFX(PB_DF, true);
    } else {
        if (parent_fmt < 0) GR_RFX(0, false);
        else if (parent_fmt == PB_SPLIT) GR_RFX(PB_SPLIT, false);
        else GR_RFX(PB_DF, false);
    }
#undef GR_RFX
}

void patch_lambda(double *sc, const double *flux, int nq, double N, double Ncov, double *lam, cudaStream_t st)
{
    GR_LAUNCH(k_lambda, 1, kBlock, st, sc, flux, nq, N, Ncov, lam);
}

void sub_scalar(int64_t cnt, double *a, const double *m, cudaStream_t st)
{
    GR_LAUNCH(k_sub_scalar, blocks_for(cnt), kBlock, st, cnt, a, m);
}

void patch_to_ghosted(int n, const double *in, double *out, double add, cudaStream_t st)
{
    GR_LAUNCH(k_to_ghosted, blocks_for((int64_t)n * n * n), kBlock, st, lg2(n), in, out, add);
}

void patch_u_load(const PPatch &P, bool pdf, const double *in, double add, cudaStream_t st)
{
    const int g = blocks_for((int64_t)1 << (3 * P.lgn));
    if (pdf) GR_LAUNCH(k_u_load<true>, g, kBlock, st, P.lgn, in, P, add);
    else GR_LAUNCH(k_u_load<false>, g, kBlock, st, P.lgn, in, P, add);
}

void patch_u_store(const PPatch &P, bool pdf, double *out, double *keep, double add, const double *usum, double scale,
                   cudaStream_t st)
{
    const int g = blocks_for((int64_t)1 << (3 * P.lgn));
    if (pdf) GR_LAUNCH(k_u_store<true>, g, kBlock, st, P.lgn, P, out, keep, add, usum, scale);
    else GR_LAUNCH(k_u_store<false>, g, kBlock, st, P.lgn, P, out, keep, add, usum, scale);
}

void patch_coef_df(int kind, const PPatch &P, cudaStream_t st)
{
    const int g = blocks_for((int64_t)1 << (3 * P.lgn));
    if (kind == KPOISSON) GR_LAUNCH(k_pcoef_df<KPOISSON>, g, kBlock, st, P);
    else if (kind == KHELM) GR_LAUNCH(k_pcoef_df<KHELM>, g, kBlock, st, P);
    else GR_LAUNCH(k_pcoef_df<KPSI>, g, kBlock, st, P);
}

void patch_aij(int n, double nh, const PSetFld &G, double *A6, cudaStream_t st)
{
    GR_LAUNCH(k_paij, blocks_for((int64_t)(n + 2) * (n + 2) * (n + 2)), kBlock, st, n, nh, G, A6);
}

int patch_setup(int eq, int n, double nh, const PSetSrc &S, const PSetFld &G, const double *A6, double smean,
                double K2, double Kdot, double *f, double *c0, double *c1, double *partials, cudaStream_t st)
{
    const int g = blocks_for((int64_t)n * n * n);
    GR_LAUNCH(k_pset, g, kBlock, st, eq, lg2(n), nh, S, G, A6, smean, K2, Kdot, f, c0, c1, partials);
    return g;
}

}  // namespace gr
