// coarse_cluster.cu - levels 64^3 .. 2^3 of the FP32 correction V-cycle in
// one thread-block cluster of 16 CTAs, one per SM.
//
// CTA r keeps planes [4r, 4r + 4) of the 64^3 level and [2r, 2r + 2) of the
// 32^3 level (e and r, both colours) in its shared memory.  A cell's i +- 1
// neighbours on the first and last plane of a slab are read from the
// adjacent CTAs' shared memory (distributed shared memory), and a cluster
// barrier takes the place of each kernel boundary of the per-level path.
// Cell by cell, the colour passes, the red-children restriction with the
// coarse first red pass and the black-children prolongation perform the
// operations of k_sweep4, k_restrict_red2 and k_prolong_black4 in their
// order, so the fields are those of the per-level path bit for bit.  The
// 32^3 level restricts into the 16^3 level kept by CTA 0, which runs the
// single-block tail (16^3 .. 2^3, coarse_tail.cuh) while the others wait.
// Measured at 512^3 it is slower than the about 22 per-level launches it
// replaces (68 against 65 us per Poisson cycle): with programmatic dependent
// launch those cost about 1.5 us each, while a slab pass here takes 0.8-1.9 us
// plus its cluster barrier, and the 16^3 prolongation reads CTA 0's shared
// memory from all sixteen CTAs.  It runs only when GR_COARSE_CLUSTER=1.
#include <cooperative_groups.h>

#include "coarse_tail.cuh"
#include "gr_internal.cuh"

namespace cg = cooperative_groups;

namespace gr {
namespace {

constexpr int kClusterCtas = 16;
constexpr int kClusterThreads = 1024;
constexpr int kSlabA = 4 * 64 * 64;  // cells of a CTA's 64^3 slab
constexpr int kSlabB = 2 * 32 * 32;  // cells of a CTA's 32^3 slab
// e and r of both slabs, the tail's residual scratch, e and r of the tail
// levels, and m, 1/(6 + h^2 m) of levels 2^3 .. 8^3 (KHELM)
constexpr int kTailCells = 8 + 64 + 512 + 4096;
constexpr size_t kClusterSmem =
    sizeof(float) * (2 * kSlabA + 2 * kSlabB + 4096 + 2 * kTailCells + 2 * (8 + 64 + 512));

// A level spread over the cluster in slabs of 2^lgp planes: the slab of CTA
// `owner` holds planes [owner << lgp, (owner + 1) << lgp), colour c at
// c * coff and row (il, j) at (il * n + j) * (n / 2).  lgp = lg: the whole
// level is held by CTA 0.  base: the array in this CTA's shared memory (the
// same offset in every CTA).
struct View {
    float *base;
    int lg, lgp, coff;
};

// row (i, j), colour 0, of the level seen through v, in the owning CTA's shared memory
__device__ __forceinline__ float *view_row(cg::cluster_group &cl, unsigned me, const View &v, int i, int j)
{
    const int owner = i >> v.lgp, il = i & ((1 << v.lgp) - 1);
    float *b = owner == (int)me ? v.base : cl.map_shared_rank(v.base, owner);
    return b + (((il << v.lg) + j) << (v.lg - 1));
}

template <int W>
__device__ __forceinline__ void ldw(const float *p, float (&v)[W])
{
    if (W == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
#pragma unroll
        for (int e = 0; e < W; e++) v[e] = p[e];
    }
}

// One colour pass over this CTA's planes of E (r: the slab's right-hand
// side; inv_g: the level's global 1/(6 + h^2 m), KHELM), W cells per item:
// per cell the operations of k_sweep4, then a cluster barrier.
template <int KIND, int W>
__device__ void slab_sweep(cg::cluster_group &cl, unsigned me, const View &E, const float *R, const float *inv_g,
                           float h2, int color)
{
    const int lg = E.lg, lgh = lg - 1, mn = (1 << lg) - 1, mh = (1 << lgh) - 1;
    const int i0 = (int)me << E.lgp;
    const int off = color ? E.coff : 0, oth = E.coff - off;
    const int half_g = 1 << (3 * lg - 1);
    for (int v = threadIdx.x; v < E.coff / W; v += blockDim.x) {
        const int t = v * W;
        const int q = t & mh, j = (t >> lgh) & mn, il = t >> (lgh + lg);
        const int i = i0 + il;
        const int p = (i + j + color) & 1;
        const float *rE = E.base + oth + (((il << lg) + j) << lgh);
        float A[W], B[W], C[W], D[W], Ev[W], F[W], G[W];
        ldw<W>(view_row(cl, me, E, (i + 1) & mn, j) + oth + q, A);
        ldw<W>(view_row(cl, me, E, (i - 1) & mn, j) + oth + q, B);
        ldw<W>(E.base + oth + (((il << lg) + ((j + 1) & mn)) << lgh) + q, C);
        ldw<W>(E.base + oth + (((il << lg) + ((j - 1) & mn)) << lgh) + q, D);
        ldw<W>(rE + q, Ev);
        ldw<W>(R + off + t, F);
        const float x = rE[(q + (p ? W : -1)) & mh];
        if (KIND == KHELM) ldw<W>(inv_g + (color ? half_g : 0) + (((i << lg) + j) << lgh) + q, G);
        float out[W];
#pragma unroll
        for (int e = 0; e < W; e++) {
            const float sh = p ? (e + 1 < W ? Ev[e + 1 < W ? e + 1 : 0] : x) : (e > 0 ? Ev[e > 0 ? e - 1 : 0] : x);
            const float nb = A[e] + B[e] + C[e] + D[e] + Ev[e] + sh;
            out[e] = __fmaf_rn(-h2, F[e], nb) * (KIND == KPOISSON ? 1.0f / 6.0f : G[e]);
        }
        float *o = E.base + off + t;
        if (W == 4) *reinterpret_cast<float4 *>(o) = make_float4(out[0], out[1], out[2], out[3]);
        else
#pragma unroll
            for (int e = 0; e < W; e++) o[e] = out[e];
    }
    cl.sync();
}

// Residual of the red children of this CTA's coarse cells and their 8-child
// average into (ec, rc), two coarse cells per item, per cell the operations
// of k_restrict_red2 (FIRST: the coarse first red relaxation from zero on red
// coarse cells, 0 on black ones; else 0).  Output layout: colour offset
// halfo, coarse plane I at row ((I - Ioff) * nc + J) * (nc / 2); m_g, cinv_g:
// global arrays of the fine and the coarse level (KHELM).
template <int KIND, int FIRST>
__device__ void slab_restrict(cg::cluster_group &cl, unsigned me, const View &Ef, const float *Rf, const float *m_g,
                              float ih2, float *ec, float *rc, int halfo, int Ioff, const float *cinv_g, float h2c)
{
    using V2 = float2;
    const int lgf = Ef.lg, lgc = lgf - 1, mc = (1 << lgc) - 1, hcl = lgc - 1, mq = (1 << hcl) - 1;
    const int mf = (1 << lgf) - 1, mhf = (1 << (lgf - 1)) - 1;
    const int lpc = Ef.lgp - 1, i0f = (int)me << Ef.lgp;
    const int halfc = 1 << (3 * lgc - 1);
    const int items = 1 << (lpc + lgc + hcl);
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int Q = t & mq, J = (t >> hcl) & mc, I = ((int)me << lpc) + (t >> (hcl + lgc));
        const int h0 = 2 * Q;  // fine half-index of k = 4Q
        auto row = [&](int a, int b) { return view_row(cl, me, Ef, (2 * I + a) & mf, (2 * J + b) & mf); };
        float c[2][2][6];
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const float *rb = row(a, b);
                const int pr = (a + b) & 1;  // colour of even k in this row
                const int ev = pr ? Ef.coff : 0, od = Ef.coff - ev;
                const V2 E = *reinterpret_cast<const V2 *>(rb + ev + h0);  // k = 4Q, 4Q + 2
                const V2 O = *reinterpret_cast<const V2 *>(rb + od + h0);  // k = 4Q + 1, 4Q + 3
                c[a][b][1] = E.x;
                c[a][b][3] = E.y;
                c[a][b][2] = O.x;
                c[a][b][4] = O.y;
                c[a][b][0] = rb[od + ((h0 - 1) & mhf)];  // k = 4Q - 1
                c[a][b][5] = rb[ev + ((h0 + 2) & mhf)];  // k = 4Q + 4
            }
        V2 si[2][2], sj[2][2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            si[q][0] = *reinterpret_cast<const V2 *>(row(-1, q) + Ef.coff + h0);
            si[q][1] = *reinterpret_cast<const V2 *>(row(2, q) + Ef.coff + h0);
            sj[q][0] = *reinterpret_cast<const V2 *>(row(q, -1) + Ef.coff + h0);
            sj[q][1] = *reinterpret_cast<const V2 *>(row(q, 2) + Ef.coff + h0);
        }
        float s[2] = {0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const int pr = (a + b) & 1;  // red children of this row: d = pr, pr + 2
                const int fl = (((2 * I + a - i0f) << lgf) + ((2 * J + b) & mf)) << (lgf - 1);
                const V2 R = *reinterpret_cast<const V2 *>(Rf + fl + h0);  // red r at d = pr, pr + 2
                V2 M = make_float2(0.0f, 0.0f);
                if (KIND == KHELM)
                    M = *reinterpret_cast<const V2 *>(m_g + ((((2 * I + a) << lgf) + ((2 * J + b) & mf)) << (lgf - 1)) +
                                                      h0);
#pragma unroll
                for (int w = 0; w < 2; w++) {
                    const int d = pr + 2 * w;
                    const float uc = c[a][b][d + 1];
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
        const int c0 = (I + J) & 1;  // colour of coarse K = 2Q
#pragma unroll
        for (int w = 0; w < 2; w++) {
            const int cid = ((c0 ^ w) ? halfo : 0) + ((((I - Ioff) << lgc) + J) << hcl) + Q;
            const float rcv = -(0.125f * s[w]);
            rc[cid] = rcv;
            float e0 = 0.0f;
            if (FIRST && !(c0 ^ w))
                e0 = -h2c * rcv *
                     (KIND == KHELM ? cinv_g[((c0 ^ w) ? halfc : 0) + (((I << lgc) + J) << hcl) + Q] : (1.0f / 6.0f));
            ec[cid] = e0;
        }
    }
    cl.sync();
}

// The coarse correction Ec prolonged trilinearly onto the black cells of
// this CTA's slab of the finer level (e: its slab array, 2^lpf planes), four
// coarse cells of a row per item, per cell the operations of k_prolong_black4.
__device__ void slab_prolong(cg::cluster_group &cl, unsigned me, const View &Ec, float *ef, int lpf)
{
    const int lgc = Ec.lg, lgf = lgc + 1, mc = (1 << lgc) - 1, hc = lgc - 1, mq = (1 << hc) - 1;
    const int lp = lgc - 2, mp = (1 << lp) - 1;  // P: coarse row / 4
    const int lpc = lpf - 1, i0f = (int)me << lpf;
    const int cofff = 1 << (lpf + 2 * lgf - 1);
    const int items = 1 << (lpc + lgc + lp);
    const float w0 = 0.25f, w1 = 0.75f;
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int P = t & mp, J = (t >> lp) & mc, I = ((int)me << lpc) + (t >> (lp + lgc));
        float z[3][3][8];
#pragma unroll
        for (int x = 0; x < 3; x++)
#pragma unroll
            for (int y = 0; y < 3; y++) {
                const int Ii = (I + x - 1) & mc, Jj = (J + y - 1) & mc;
                const float *rc = view_row(cl, me, Ec, Ii, Jj);
                const int ce = ((Ii + Jj) & 1) ? Ec.coff : 0;  // colour array of the even coarse K
                const int co = Ec.coff - ce;
                const float2 ev = *reinterpret_cast<const float2 *>(rc + ce + 2 * P);  // K = 4P, 4P + 2
                const float2 od = *reinterpret_cast<const float2 *>(rc + co + 2 * P);  // K = 4P + 1, 4P + 3
                const float om = rc[co + ((2 * P - 1) & mq)];                         // K = 4P - 1
                const float ep = rc[ce + ((2 * P + 2) & mq)];                         // K = 4P + 4
                const float cv[6] = {om, ev.x, od.x, ev.y, od.y, ep};
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    const int t0 = (m >> 1) + 1, t1 = (m & 1) ? t0 + 1 : t0 - 1;
                    z[x][y][m] = w1 * cv[t0] + w0 * cv[t1];
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
                const int row = (((2 * I + a - i0f) << lgf) + 2 * J + b) << (lgf - 1);
                float4 *blk = reinterpret_cast<float4 *>(ef + cofff + row + 4 * P);
                float4 k4 = *blk;
                k4.x += val[0];
                k4.y += val[1];
                k4.z += val[2];
                k4.w += val[3];
                *blk = k4;
            }
        }
    }
    cl.sync();
}

// level arrays of 2^3 .. 64^3 (index 0 = 2^3), global split layout; h2 and
// ih2 rounded from the level's double values as the per-level launches round them
struct ClusterArgs {
    float *e[6], *r[6];
    const float *m[6], *inv[6];
    float h2[6], ih2[6];
};

template <int KIND>
__global__ void __launch_bounds__(kClusterThreads, 1) k_coarse_cluster(ClusterArgs g, int nu1, int nu2)
{
    pdl_begin();
    cg::cluster_group cl = cg::this_cluster();
    const unsigned me = cl.block_rank();
    extern __shared__ float4 sh4[];
    float *sh = reinterpret_cast<float *>(sh4);
    float *Ae = sh, *Ar = Ae + kSlabA, *Be = Ar + kSlabA, *Br = Be + kSlabB;
    float *res = Br + kSlabB;  // residual scratch of the tail's 16^3 level (CTA 0)
    float *p = res + 4096;
    TailLevel L[4];
#pragma unroll
    for (int l = 0; l < 4; l++) {
        const int cells = 1 << (3 * (l + 1));
        L[l].lg = l + 1;
        L[l].h2 = g.h2[l];
        L[l].ih2 = 1.0f / g.h2[l];
        L[l].e = p;
        L[l].r = p + cells;
        p += 2 * cells;
        if (KIND == KHELM && l < 3) {
            L[l].m = p;
            L[l].inv = p + cells;
            p += 2 * cells;
            if (me == 0)
                for (int t = threadIdx.x; t < cells; t += blockDim.x) {
                    L[l].m[t] = g.m[l][t];
                    L[l].inv[t] = g.inv[l][t];
                }
        } else {  // the 16^3 coefficients are read from global memory (KHELM)
            L[l].m = const_cast<float *>(g.m[l]);
            L[l].inv = const_cast<float *>(g.inv[l]);
        }
    }
    // this CTA's 64^3 slab of e (first red pass made by the restriction) and r
    {
        const int i0 = (int)me * 4 * 64 * 32, hg = 64 * 64 * 32;
        for (int v = threadIdx.x; v < kSlabA / 4; v += blockDim.x) {
            const int c = v >= kSlabA / 8, t = 4 * v - (c ? kSlabA / 2 : 0);
            const int gi = (c ? hg : 0) + i0 + t;
            *reinterpret_cast<float4 *>(Ae + 4 * v) = *reinterpret_cast<const float4 *>(g.e[5] + gi);
            *reinterpret_cast<float4 *>(Ar + 4 * v) = *reinterpret_cast<const float4 *>(g.r[5] + gi);
        }
    }
    cl.sync();
    const View VA{Ae, 6, 2, kSlabA / 2}, VB{Be, 5, 1, kSlabB / 2}, VT{L[3].e, 4, 4, 2048};
    // 64^3 pre-smoothing: black, then nu1 - 1 red-black sweeps
    slab_sweep<KIND, 4>(cl, me, VA, Ar, g.inv[5], g.h2[5], 1);
    for (int s = 1; s < nu1; s++) {
        slab_sweep<KIND, 4>(cl, me, VA, Ar, g.inv[5], g.h2[5], 0);
        slab_sweep<KIND, 4>(cl, me, VA, Ar, g.inv[5], g.h2[5], 1);
    }
    slab_restrict<KIND, 1>(cl, me, VA, Ar, g.m[5], g.ih2[5], Be, Br, kSlabB / 2, (int)me * 2, g.inv[4], g.h2[4]);
    // 32^3 pre-smoothing, the first red pass made by the restriction
    slab_sweep<KIND, 1>(cl, me, VB, Br, g.inv[4], g.h2[4], 1);
    for (int s = 1; s < nu1; s++) {
        slab_sweep<KIND, 1>(cl, me, VB, Br, g.inv[4], g.h2[4], 0);
        slab_sweep<KIND, 1>(cl, me, VB, Br, g.inv[4], g.h2[4], 1);
    }
    // into CTA 0's 16^3 level (e = 0, r = the red children's average)
    {
        float *te = me == 0 ? L[3].e : cl.map_shared_rank(L[3].e, 0);
        float *tr = me == 0 ? L[3].r : cl.map_shared_rank(L[3].r, 0);
        slab_restrict<KIND, 0>(cl, me, VB, Br, g.m[4], g.ih2[4], te, tr, 2048, 0, nullptr, 0.0f);
    }
    if (me == 0) tail_cycle<KIND>(L, res, nu1, nu2);
    cl.sync();
    slab_prolong(cl, me, VT, Be, 1);
    for (int s = 0; s < nu2; s++) {
        slab_sweep<KIND, 1>(cl, me, VB, Br, g.inv[4], g.h2[4], 0);
        slab_sweep<KIND, 1>(cl, me, VB, Br, g.inv[4], g.h2[4], 1);
    }
    slab_prolong(cl, me, VB, Ae, 2);
    for (int s = 0; s < nu2; s++) {
        slab_sweep<KIND, 4>(cl, me, VA, Ar, g.inv[5], g.h2[5], 0);
        slab_sweep<KIND, 4>(cl, me, VA, Ar, g.inv[5], g.h2[5], 1);
    }
    // the 64^3 correction back to global memory for the prolongation onto 128^3
    {
        const int i0 = (int)me * 4 * 64 * 32, hg = 64 * 64 * 32;
        for (int v = threadIdx.x; v < kSlabA / 4; v += blockDim.x) {
            const int c = v >= kSlabA / 8, t = 4 * v - (c ? kSlabA / 2 : 0);
            *reinterpret_cast<float4 *>(g.e[5] + (c ? hg : 0) + i0 + t) = *reinterpret_cast<const float4 *>(Ae + 4 * v);
        }
    }
}

template <int KIND>
cudaLaunchConfig_t cluster_config(cudaStream_t st, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = kClusterSmem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCtas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cfg;
}

// once per kind: the 16-CTA cluster (beyond the portable 8) and its shared
// memory are allowed, and the device can hold one such cluster
template <int KIND>
bool cluster_usable()
{
    static const bool ok = [] {
        auto k = k_coarse_cluster<KIND>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        cudaLaunchAttribute at[2];
        cudaLaunchConfig_t cfg = cluster_config<KIND>(nullptr, at);
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, (const void *)k, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return nc >= 1;
    }();
    return ok;
}

template <int KIND>
void launch_cluster(const ClusterArgs &a, int nu1, int nu2, cudaStream_t st)
{
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config<KIND>(st, at);
    if (cudaLaunchKernelEx(&cfg, k_coarse_cluster<KIND>, a, nu1, nu2) != cudaSuccess) {
        cudaGetLastError();  // without programmatic serialization; an error of this launch stays recorded
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_coarse_cluster<KIND>, a, nu1, nu2);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

}  // namespace

bool coarse_cluster_ok(int kind)
{
    if (kind == KPOISSON) return cluster_usable<KPOISSON>();
    if (kind == KHELM) return cluster_usable<KHELM>();
    return false;
}

void coarse_cluster(int kind, float *const *e, float *const *r, const float *const *m, const float *const *inv,
                    const double *h2, const double *ih2, int nu1, int nu2, cudaStream_t st)
{
    ClusterArgs a;
    for (int l = 0; l < 6; l++) {
        a.e[l] = e[l];
        a.r[l] = r[l];
        a.m[l] = m[l];
        a.inv[l] = inv[l];
        a.h2[l] = (float)h2[l];
        a.ih2[l] = (float)ih2[l];
    }
    if (kind == KPOISSON) launch_cluster<KPOISSON>(a, nu1, nu2, st);
    else launch_cluster<KHELM>(a, nu1, nu2, st);
}

}  // namespace gr
