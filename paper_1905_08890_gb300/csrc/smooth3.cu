// smooth3.cu - three red-black Gauss-Seidel colour passes of the FP32
// correction equation (Sec. 3.1: lap e - m e = r, Poisson m = 0) in one pass
// over HBM.
//
// The separate colour passes of the correction cycle each read the other
// colour and the right-hand side of the updated colour and write the updated
// colour: 6 bytes per cell for Poisson, 8 with the Helmholtz inverse diagonal,
// so three passes cost 18 (24) bytes per cell.  This kernel reads the input
// colour once, the right-hand side (and inverse diagonal) of both colours
// once, and writes both colours once: 10 (14) bytes per cell.
//
// Passes: P1 updates colour c1 from the input colour c2, P2 colour c2 from P1,
// P3 colour c1 from P2; the result is (c1: P3, c2: P2), bit for bit what the
// three separate passes give (same operands, same order of additions, the
// same fused multiply-add).  It is written to a second buffer, because the
// input colour is overwritten by P2 while neighbouring tiles still read it.
//
// Work split: each block owns a column tile of TJ rows (j) by 32 half-indices
// (q) and marches along i over the whole periodic range, one plane per step.
// At step s it makes P1 on plane s, P2 on plane s - 1 and P3 on plane s - 2
// (each pass needs its predecessor on the planes on both sides), over halos of
// two, one and zero cells in j and q.  The planes of the input colour and of
// the right-hand sides arrive in shared-memory rings by asynchronous copies
// (cp.async) kD planes ahead; each thread keeps its own strip of four
// half-indices of the last three planes of the input, P1 and P2 in registers
// (the i neighbours), and P1 and P2 go to small shared-memory rings for the j
// and q neighbours.  One barrier per plane.  Block count: two blocks on every
// SM; the i range is walked in full from plane -2 to n + 1 (periodic), so the
// only redundant work is four planes of P1 and two of P2 per column.
//
// Measured at 512^3 it moves its algorithmic DRAM bytes but takes as long as
// the three separate passes (373 against 371 us): both are bound by the SM's
// L1/shared-memory pipe, which here carries the staged halos, the j
// neighbours of every pass and the P1/P2 rings (about 450 shared-memory
// wavefronts per block and plane), where the separate passes, at the copy
// rate, read the same neighbours through L1.  The library therefore uses it
// only when asked (GR_SMOOTH3=1).
#include "gr_internal.cuh"

namespace gr {
namespace {

constexpr int kQ = 32;            // half-indices per tile row
constexpr int kGC = kQ / 4 + 2;   // float4 groups computed per row (one halo group each side)
constexpr int kGL = kGC + 2;      // float4 groups held per row of the input, P1 and P2 (two halo groups)
constexpr int kTJMax = 14;        // tallest tile (rows)
constexpr int kLanes = kGL;       // lanes per tile row: a row's float4 accesses are consecutive (no bank conflicts)
constexpr int kThreads = 256;     // >= (kTJMax + 4) kLanes

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// one colour update of four consecutive half-indices: neighbours in the other
// colour at i + 1 (a), i - 1 (b), j + 1 (c), j - 1 (d), the own row (e) and
// the own row shifted by +1 (p = 1; x = the value after the strip) or -1
// (p = 0; x = the value before it); the same expression as the single pass
template <int KIND>
__device__ __forceinline__ float4 relax(float4 a, float4 b, float4 c, float4 d, float4 e, float x, int p, float4 f,
                                        float4 g, float h2)
{
    const float4 sh = p ? make_float4(e.y, e.z, e.w, x) : make_float4(x, e.x, e.y, e.z);
    float4 nb;
    nb.x = a.x + b.x + c.x + d.x + e.x + sh.x;
    nb.y = a.y + b.y + c.y + d.y + e.y + sh.y;
    nb.z = a.z + b.z + c.z + d.z + e.z + sh.z;
    nb.w = a.w + b.w + c.w + d.w + e.w + sh.w;
    if (KIND == KPOISSON) g = make_float4(1.0f / 6.0f, 1.0f / 6.0f, 1.0f / 6.0f, 1.0f / 6.0f);
    return make_float4(__fmaf_rn(-h2, f.x, nb.x) * g.x, __fmaf_rn(-h2, f.y, nb.y) * g.y,
                       __fmaf_rn(-h2, f.z, nb.z) * g.z, __fmaf_rn(-h2, f.w, nb.w) * g.w);
}

struct S3Args {
    const float *ein;  // input e (split layout); colour c2 is read
    float *eout;       // output e, both colours
    const float *f;    // right-hand side, both colours
    const float *g;    // KHELM: 1 / (6 + h^2 m), both colours
    float h2;
    int lgn, c1, rt;   // log2 n, first updated colour, row tiles
};

// ring sizes and shared-memory layout (float4 units) for TJM rows per tile
template <int KIND, int D>
struct S3Layout {
    static constexpr int R = D + 4;  // planes s - 2 .. s + 1 in use, s + 2 .. s + D + 1 in flight
    int tjm;
    __host__ __device__ int in_sz() const { return R * (tjm + 6) * kGL; }
    __host__ __device__ int f1_sz() const { return R * (tjm + 4) * kGC; }
    __host__ __device__ int f2_sz() const { return R * (tjm + 2) * kGC; }
    __host__ __device__ int p1_sz() const { return 2 * (tjm + 4) * kGL; }
    __host__ __device__ int p2_sz() const { return 2 * (tjm + 2) * kGL; }
    // + a tail: lanes outside a pass's domain load (and discard) values up to
    // two rows past their ring slot
    __host__ __device__ int total() const
    {
        return in_sz() + f1_sz() + f2_sz() + (KIND == KHELM ? f1_sz() + f2_sz() : 0) + p1_sz() + p2_sz() + 4 * kGL;
    }
};

// slot of plane s +- k in a ring of R slots, from the slot of plane s
template <int R>
__device__ __forceinline__ int ring_add(int sl, int k)
{
    const int v = sl + k;
    return v >= R ? v - R : (v < 0 ? v + R : v);
}

// Per-thread state of the march and one step of it.  Lane (r, gg) works on
// group gg - 1 of row j0 - 2 + r for gg < 10 (groups -1 .. 8, the halo of one
// group included), so a row's float4 accesses are consecutive; the two spare
// lanes of each row and the rows past the tallest tile only copy.  Every working lane runs all three
// passes (the warps mix lanes inside and outside each pass's domain, so
// branching would not skip work); lanes outside a domain compute values no
// output depends on, and their stores are predicated off.  EVEN: parity of the
// step s, which fixes the P1/P2 ring slots and flips the shift direction.
template <int KIND, int D>
struct S3Thread {
    static constexpr int R = D + 4;
    static constexpr int kMaxG = KIND == KHELM ? 4 : 3;  // copies per thread and plane: ceil(staged granules / threads)
    const float4 *In, *F1, *F2, *G1, *G2;
    float4 *P1, *P2;
    int in_pl, f1_pl, f2_pl, p1_pl, p2_pl;
    int o_in, o_f1, o_f2, o_p1, o_p2;
    int pa;                   // own-row shift direction at even steps (all three passes)
    bool work, act1, act2, act3;
    float *out1, *out2;       // output strips (colours c1, c2) of the plane of the next P3
    size_t plane;             // floats per colour plane
    float h2;
    const float *gsrc[kMaxG];
    unsigned gdst[kMaxG], gstr[kMaxG];
    int ng, mn, lgpl;

    __device__ __forceinline__ void issue(int p, int sl) const
    {
        const size_t po = (size_t)(p & mn) << lgpl;
#pragma unroll
        for (int k = 0; k < kMaxG; k++)
            if (k < ng)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(gdst[k] + sl * gstr[k]),
                             "l"(gsrc[k] + po)
                             : "memory");
        cp_commit();
    }

    // step s with the queues (x0, x1, x2) = input at s - 1, s, s + 1 (x2 loaded
    // here), (y0, y1, y2) = P1 at s - 2, s - 1, s (y2 made here), (z0, z1, z2) =
    // P2 at s - 3, s - 2, s - 1 (z2 made here); sl = ring slot of plane s
    // (w0, w1, w2), (v0, v1, v2): f and KHELM's inverse diagonal of colour c1
    // at s - 2, s - 1, s (w2, v2 loaded here for P1; P3 takes w0, v0)
    template <bool EVEN, bool DO2, bool DO3>
    __device__ __forceinline__ void step(int sl, float4 &x0, float4 &x1, float4 &x2, float4 &y0, float4 &y1,
                                         float4 &y2, float4 &z0, float4 &z1, float4 &z2, float4 &w0, float4 &w2,
                                         float4 &v0, float4 &v2) const
    {
        if (!work) return;
        const int p = EVEN ? pa : 1 - pa;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        // every operand of the three passes first: no pass reads a ring slot
        // that another pass writes in this step, so the loads need not wait for
        // the stores, and their latencies overlap
        const float4 *I = In + sl * in_pl + o_in;
        const float4 *Q1 = P1 + (EVEN ? 1 : 0) * p1_pl + o_p1;  // P1 on plane s - 1
        const float4 *Q2 = P2 + (EVEN ? 0 : 1) * p2_pl + o_p2;  // P2 on plane s - 2
        const int s1 = ring_add<R>(sl, -1);
        x2 = In[ring_add<R>(sl, 1) * in_pl + o_in];
        // the shifted own-row neighbour: the next group's first value (p = 1)
        // or the previous group's last (p = 0)
        const float4 n1 = I[p ? 1 : -1];
        const float4 c1v = I[kGL], d1v = I[-kGL];
        w2 = F1[sl * f1_pl + o_f1];
        if (KIND == KHELM) v2 = G1[sl * f1_pl + o_f1];
        float4 n2 = zero4, c2v = zero4, d2v = zero4, f2 = zero4, g2 = zero4;
        float4 n3 = zero4, c3v = zero4, d3v = zero4;
        if (DO2) {
            n2 = Q1[p ? 1 : -1];
            c2v = Q1[kGL], d2v = Q1[-kGL];
            f2 = F2[s1 * f2_pl + o_f2];
            if (KIND == KHELM) g2 = G2[s1 * f2_pl + o_f2];
        }
        if (DO3) {
            n3 = Q2[p ? 1 : -1];
            c3v = Q2[kGL], d3v = Q2[-kGL];
        }
        // P1 on plane s (colour c1), P2 on plane s - 1 (colour c2), P3 on plane
        // s - 2 (colour c1)
        y2 = relax<KIND>(x2, x0, c1v, d1v, x1, p ? n1.x : n1.w, p, w2, v2, h2);
        if (DO2) z2 = relax<KIND>(y2, y0, c2v, d2v, y1, p ? n2.x : n2.w, p, f2, g2, h2);
        float4 v3 = zero4;
        if (DO3) v3 = relax<KIND>(z2, z0, c3v, d3v, z1, p ? n3.x : n3.w, p, w0, v0, h2);
        if (act1) P1[(EVEN ? 0 : 1) * p1_pl + o_p1] = y2;
        if (DO2 && act2) P2[(EVEN ? 1 : 0) * p2_pl + o_p2] = z2;
        if (DO3 && act3) {
            *reinterpret_cast<float4 *>(out1) = v3;
            *reinterpret_cast<float4 *>(out2) = z1;
        }
    }
};

template <int KIND, int D>
__device__ __forceinline__ void smooth3_body(const S3Args &a)
{
    extern __shared__ float4 sm[];
    using T = S3Thread<KIND, D>;
    constexpr int R = T::R;
    constexpr int kMaxG = T::kMaxG;
    const int n = 1 << a.lgn, mn = n - 1, lgh = a.lgn - 1;
    const int qt_n = n >> 6;  // q tiles (32 half-indices each)
    const int qt = blockIdx.x % qt_n, rti = blockIdx.x / qt_n;
    const int j0 = (int)(((long long)rti * n) / a.rt), TJ = (int)(((long long)(rti + 1) * n) / a.rt) - j0;
    // laid out for the tallest tile whatever this tile's height: lanes outside
    // a pass's domain (rows up to 19) then read inside the allocation
    const S3Layout<KIND, D> L{kTJMax};
    T t;
    float4 *In = sm;
    float4 *F1 = In + L.in_sz();
    float4 *F2 = F1 + L.f1_sz();
    float4 *G1 = F2 + L.f2_sz();
    float4 *G2 = G1 + (KIND == KHELM ? L.f1_sz() : 0);
    float4 *P1 = G2 + (KIND == KHELM ? L.f2_sz() : 0);
    float4 *P2 = P1 + L.p1_sz();
    t.In = In, t.F1 = F1, t.F2 = F2, t.G1 = G1, t.G2 = G2, t.P1 = P1, t.P2 = P2;
    t.in_pl = (L.tjm + 6) * kGL, t.f1_pl = (L.tjm + 4) * kGC, t.f2_pl = (L.tjm + 2) * kGC;
    t.p1_pl = (L.tjm + 4) * kGL, t.p2_pl = (L.tjm + 2) * kGL;
    t.mn = mn;
    t.lgpl = 2 * a.lgn - 1;  // log2 of a colour plane's size (n^2 / 2 floats)
    t.plane = (size_t)1 << t.lgpl;
    t.h2 = a.h2;

    const int c1 = a.c1, c2 = 1 - c1;
    const size_t half = (size_t)1 << (3 * a.lgn - 1);
    const int gmask = (n >> 3) - 1;  // float4 groups per row - 1
    const int gq = qt * (kQ / 4);    // first interior group of the tile

    // zero the P1 and P2 rings and the tail
    for (int i = threadIdx.x; i < L.p1_sz() + L.p2_sz() + 4 * kGL; i += kThreads) P1[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    // this thread's share of the staged granules of one plane, the same for
    // every plane: source within a plane (periodic row and group), destination
    // in ring slot 0 and the slot stride (bytes)
    const int n_in = (TJ + 6) * kGC, n_f1 = (TJ + 4) * kGC, n_f2 = (TJ + 2) * kGC;
    const int n_all = n_in + (KIND == KHELM ? 2 : 1) * (n_f1 + n_f2);
    t.ng = 0;
#pragma unroll
    for (int k = 0; k < kMaxG; k++) {
        const int u0 = threadIdx.x + k * kThreads;
        t.gsrc[k] = a.f;
        t.gdst[k] = t.gstr[k] = 0;
        if (u0 >= n_all) continue;
        t.ng = k + 1;
        if (u0 < n_in) {
            // groups -1 .. 8 into columns 1 .. 10: the outer columns (groups -2
            // and 9) would only feed values that no output depends on
            const int rr = u0 / kGC, cc = u0 - rr * kGC;
            const int jw = (j0 - 3 + rr) & mn, gw = (gq - 1 + cc) & gmask;
            t.gsrc[k] = a.ein + (c2 ? half : 0) + ((size_t)jw << lgh) + 4 * gw;
            t.gdst[k] = (unsigned)__cvta_generic_to_shared(In + rr * kGL + cc + 1);
            t.gstr[k] = t.in_pl * 16;
        } else {
            int u = u0 - n_in, arr = 0;  // 0: f c1, 1: f c2, 2: g c1, 3: g c2
            if (u >= n_f1) {
                u -= n_f1;
                arr = 1;
                if (KIND == KHELM && u >= n_f2) {
                    u -= n_f2;
                    arr = 2;
                    if (u >= n_f1) {
                        u -= n_f1;
                        arr = 3;
                    }
                }
            }
            const int rr = u / kGC, cc = u - rr * kGC;
            const bool first = arr == 0 || arr == 2;  // colour c1 arrays: rows from j0 - 2, else j0 - 1
            const int jw = (j0 - (first ? 2 : 1) + rr) & mn, gw = (gq - 1 + cc) & gmask;
            const float *base = (arr < 2 ? a.f : a.g) + ((first ? c1 : c2) ? half : 0);
            t.gsrc[k] = base + ((size_t)jw << lgh) + 4 * gw;
            float4 *d0 = arr == 0 ? F1 : arr == 1 ? F2 : arr == 2 ? G1 : G2;
            t.gdst[k] = (unsigned)__cvta_generic_to_shared(d0 + u);
            t.gstr[k] = (first ? t.f1_pl : t.f2_pl) * 16;
        }
    }

    const int tid = threadIdx.x;
    const int r = tid / kLanes, gg = tid - (tid / kLanes) * kLanes;  // group gg - 1
    t.work = gg < kGC && r < kTJMax + 4;
    const int j = j0 - 2 + r;  // row of this thread's strip (may lie outside [0, n))
    t.act1 = r < TJ + 4;
    t.act2 = r >= 1 && r < TJ + 3;
    t.act3 = r >= 2 && r < TJ + 2 && gg >= 1 && gg <= kGC - 2;
    t.pa = (j + c1) & 1;  // the step parity enters as s + j + c1 (P2: s - 1 + j + c2 has the same parity)
    t.o_in = (r + 1) * kGL + gg + 1;  // input, own strip (rows from j0 - 3, groups from -2)
    t.o_f1 = r * kGC + gg, t.o_f2 = (r - 1) * kGC + gg;  // groups from -1
    t.o_p1 = r * kGL + gg + 1;        // P1 rows from j0 - 2
    t.o_p2 = (r - 1) * kGL + gg + 1;  // P2 rows from j0 - 1
    // output strips of P3 threads, plane 0
    const size_t o_out = ((size_t)(j & mn) << lgh) + 4 * ((gq + gg - 1) & gmask);
    t.out1 = a.eout + (c1 ? half : 0) + o_out;
    t.out2 = a.eout + (c2 ? half : 0) + o_out;

    // prologue: planes -3 .. D - 2 (D + 2 groups); -3 .. -1 complete after the wait
    for (int p = -3; p <= D - 2; p++) t.issue(p, (p + 3 * R) % R);
    cp_wait<D - 1>();
    __syncthreads();
    int sl = (3 * R - 2) % R;  // slot of plane s = -2
    float4 qa = make_float4(0.f, 0.f, 0.f, 0.f), qb = qa;
    if (t.work) {
        qa = In[ring_add<R>(sl, -1) * t.in_pl + t.o_in];
        qb = In[sl * t.in_pl + t.o_in];
    }
    float4 qc = qa;
    float4 ya = qa, yb = qa, yc = qa, za = qa, zb = qa, zc = qa;
    float4 Wya = qa, Wyb = qa, Wyc = qa, Vya = qa, Vyb = qa, Vyc = qa;  // f, inverse diagonal of c1 (rotate as P1)
    // one step: wait for plane s + 1, run it, issue plane s + D + 1 into the slot
    // of plane s - 3 (which no lane reads at step s), advance
#define S3_STEP(EVEN, DO2, DO3, X0, X1, X2, Y0, Y1, Y2, Z0, Z1, Z2)                     \
    do {                                                                                \
        cp_wait<D - 1>();                                                               \
        __syncthreads();                                                                \
        t.template step<EVEN, DO2, DO3>(sl, X0, X1, X2, Y0, Y1, Y2, Z0, Z1, Z2, W##Y0, W##Y2, \
                                        V##Y0, V##Y2);                                  \
        if (DO3) {                                                                      \
            t.out1 += t.plane;                                                          \
            t.out2 += t.plane;                                                          \
        }                                                                               \
        if (s + D + 1 <= n + 2) t.issue(s + D + 1, ring_add<R>(sl, D + 1));             \
        else cp_commit();                                                               \
        sl = ring_add<R>(sl, 1);                                                        \
        ++s;                                                                            \
    } while (0)
    int s = -2;
    S3_STEP(true, false, false, qa, qb, qc, ya, yb, yc, za, zb, zc);   // s = -2
    S3_STEP(false, false, false, qb, qc, qa, yb, yc, ya, zb, zc, za);  // s = -1
    S3_STEP(true, true, false, qc, qa, qb, yc, ya, yb, zc, za, zb);    // s = 0
    S3_STEP(false, true, false, qa, qb, qc, ya, yb, yc, za, zb, zc);   // s = 1
    // s = 2 .. n + 1, six steps per pass of the loop (parity and queue rotation static)
    while (true) {
        S3_STEP(true, true, true, qb, qc, qa, yb, yc, ya, zb, zc, za);
        if (s > n + 1) break;
        S3_STEP(false, true, true, qc, qa, qb, yc, ya, yb, zc, za, zb);
        if (s > n + 1) break;
        S3_STEP(true, true, true, qa, qb, qc, ya, yb, yc, za, zb, zc);
        if (s > n + 1) break;
        S3_STEP(false, true, true, qb, qc, qa, yb, yc, ya, zb, zc, za);
        if (s > n + 1) break;
        S3_STEP(true, true, true, qc, qa, qb, yc, ya, yb, zc, za, zb);
        if (s > n + 1) break;
        S3_STEP(false, true, true, qa, qb, qc, ya, yb, yc, za, zb, zc);
        if (s > n + 1) break;
    }
#undef S3_STEP
    cp_wait<0>();
}

// entry points (the Poisson kernel stages three ring planes ahead, the
// Helmholtz kernel, which also stages the inverse diagonals, two), two blocks
// per SM
__global__ void __launch_bounds__(kThreads, 2) k_smooth3_poisson(S3Args a)
{
    pdl_begin();
    smooth3_body<KPOISSON, 3>(a);
}
__global__ void __launch_bounds__(kThreads, 2) k_smooth3_helm(S3Args a)
{
    pdl_begin();
    smooth3_body<KHELM, 2>(a);
}

template <int KIND, int D>
void launch_s3(void (*kern)(S3Args), int n, const float *ein, float *eout, const float *f, const float *g, double h2,
               int c1, int rt, cudaStream_t st)
{
    const S3Layout<KIND, D> L{kTJMax};
    const size_t smem = (size_t)L.total() * sizeof(float4);
    // once per kernel (a function-local static is initialised once, even with several host threads)
    static const bool attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                             cudaSuccess;
    (void)attr;
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    S3Args a{ein, eout, f, g, (float)h2, lgn, c1, rt};
    GR_LAUNCH_SMEM(kern, (n >> 6) * rt, kThreads, smem, st, a);
}

}  // namespace

// Row tiles for an n^3 grid: two blocks on every SM where the tile height
// stays within [4, 14] rows, else the nearest height in that range.
int smooth3_row_tiles(int n, int sms)
{
    const int qt = n >> 6;
    int rt = (2 * sms + qt - 1) / qt;
    const int lo = (n + kTJMax - 1) / kTJMax, hi = n / 4;
    if (rt < lo) rt = lo;
    if (rt > hi) rt = hi;
    return rt;
}

bool smooth3_fits(int kind, int n) { return (kind == KPOISSON || kind == KHELM) && n >= 64 && n <= 1024; }

void smooth3(int kind, int n, const float *ein, float *eout, const float *f, const float *inv, double h2, int c1,
             int rt, cudaStream_t st)
{
    if (kind == KPOISSON) launch_s3<KPOISSON, 3>(k_smooth3_poisson, n, ein, eout, f, nullptr, h2, c1, rt, st);
    else launch_s3<KHELM, 2>(k_smooth3_helm, n, ein, eout, f, inv, h2, c1, rt, st);
}

}  // namespace gr
