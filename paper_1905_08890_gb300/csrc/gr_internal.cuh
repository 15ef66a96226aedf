// gr_internal.cuh - shared definitions of the CUDA library (not part of the C ABI).
//
// Multigrid level arrays use a red-black split layout: on a level of extent
// n (a power of two, n >= 2) the cell (i, j, k) of colour c = (i + j + k) & 1
// lives at
//     c * n^3/2 + (i * n + j) * (n/2) + (k >> 1).
// A red cell's six neighbours are black cells at the same half-index q = k>>1
// in rows (i +- 1, j) and (i, j +- 1), and at q and q + (p ? 1 : -1) in its own
// row, p = (i + j + c) & 1 the parity of k.  A colour pass therefore reads one
// contiguous half-array and writes the other, with no idle threads, and the
// 8 children of a coarse cell (I, J, K) all sit at q = K in rows (2I + a, 2J + b).
// Caller-facing fields and sources use the natural [n][n][n] layout.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include <atomic>
#include <mutex>
#include <unordered_map>

#include "df64.cuh"

namespace gr {

// kernels launched by this library since load; every launch goes through GR_LAUNCH
extern std::atomic<long long> g_launches;

// Every kernel is launched with programmatic dependent launch: the next kernel
// of the stream may be scheduled onto the SMs while its predecessor drains
// (its launch latency and block start-up overlap the predecessor's last
// blocks), and every kernel begins with pdl_begin(), which waits for the
// predecessor's completion and memory before anything else, so the stream's
// order of effects is that of plain launches.
template <class T>
struct ident {
    using type = T;
};
template <typename... KArgs>
inline void launch_pdl(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st,
                       typename ident<KArgs>::type... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k, args...) != cudaSuccess) {
        // a stream that takes no programmatic serialization (the legacy default
        // stream may not): a plain launch, whose error, if any, stays recorded
        cudaGetLastError();
        cfg.numAttrs = 0;
        cudaLaunchKernelEx(&cfg, k, args...);
    }
}
#define GR_LAUNCH(kernel, grid, block, stream, ...)                              \
    do {                                                                         \
        ::gr::launch_pdl(kernel, (grid), (block), 0, (stream), __VA_ARGS__);      \
        ::gr::g_launches.fetch_add(1, std::memory_order_relaxed);                \
    } while (0)
#define GR_LAUNCH_SMEM(kernel, grid, block, smem, stream, ...)                   \
    do {                                                                         \
        ::gr::launch_pdl(kernel, (grid), (block), (smem), (stream), __VA_ARGS__); \
        ::gr::g_launches.fetch_add(1, std::memory_order_relaxed);                \
    } while (0)

#ifdef __CUDACC__
// first statement of every kernel: let the stream's next kernel launch, then
// wait for the previous one (a no-op for a kernel launched without the attribute)
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.launch_dependents;\n\tgriddepcontrol.wait;" ::: "memory");
}
#endif

// Kernels of the finest level take `rev`: nonzero walks their index range
// from the end, so a launch that follows one walking forward starts where it
// stopped, on data still in L2.

// Blocks for a grid-stride kernel over `threads` threads: one full wave (as
// many blocks per SM as the kernel's registers allow, on every SM) or fewer
// when the work is smaller.  Every block then takes the same number of
// grid-stride iterations to within one, where a fixed block count that is not
// a multiple of the wave leaves a partial last wave with most SMs idle.
inline int wave_grid_of(const void *kernel, int64_t threads, int block)
{
    static std::mutex mu;
    static std::unordered_map<const void *, int> per_sm;
    static int sms = 0;
    int b = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (sms == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (sms <= 0) sms = 1;
        }
        auto it = per_sm.find(kernel);
        if (it == per_sm.end()) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, 0) != cudaSuccess || b <= 0) {
                cudaGetLastError();
                b = 1;
            }
            per_sm[kernel] = b;
        } else {
            b = it->second;
        }
    }
    const int64_t need = (threads + block - 1) / block;
    const int64_t wave = (int64_t)sms * b;
    return (int)(need < 1 ? 1 : (need < wave ? need : wave));
}

template <class Kernel>
int wave_grid(Kernel kernel, int64_t threads, int block = 256)
{
    return wave_grid_of(reinterpret_cast<const void *>(kernel), threads, block);
}

// sets the thread's message returned by gr_last_error()
void set_last_error(const char *msg);

constexpr double kPi = 3.14159265358979323846;

enum Kind : int { KPOISSON = 0, KHELM = 1, KPSI = 2 };

constexpr int kBlock = 256;
constexpr int kMaxRedBlocks = 152 * 16;  // blocks of the norm/mean reductions (16 per SM)
constexpr int kCoarsestSweeps = 32;  // red-black sweeps on the 2^3 level

#ifdef __CUDACC__
// Block sums of a and b (blockDim.x == kBlock) into out[2 blockIdx.x + 0/1],
// in a fixed order.
__device__ __forceinline__ void block_sum2(double a, double b, double *out)
{
    __shared__ double sa[kBlock / 32], sb[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int q = 0; q < kBlock / 32; q++) {
            ta += sa[q];
            tb += sb[q];
        }
        out[2 * blockIdx.x] = ta;
        out[2 * blockIdx.x + 1] = tb;
    }
}

// The same for FP32 inputs: warp sums in FP32 (for norms, where the rounding
// of partial sums is harmless), the per-warp totals in FP64.  GB300's FP64
// pipe is narrow enough that a full FP64 warp reduction per thread costs a
// noticeable share of a memory-sized kernel.
__device__ __forceinline__ void block_sum2f(float a, float b, double *out)
{
    __shared__ double sa[kBlock / 32], sb[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = (double)a;
        sb[w] = (double)b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int q = 0; q < kBlock / 32; q++) {
            ta += sa[q];
            tb += sb[q];
        }
        out[2 * blockIdx.x] = ta;
        out[2 * blockIdx.x + 1] = tb;
    }
}
#endif

// ---- multigrid kernels (templated on the working precision T) ---------------
// One Gauss-Seidel pass over colour `color` of a level.  KPOISSON: f;
// KHELM: f and c1 = 1/(6 + h^2 m); KPSI (double only): f, c0 = s0, c1 = AA,
// unknown u = psi - 1, one Newton step per cell.
template <typename T>
void sweep_colour(int kind, int n, T *u, const T *f, const T *c0, const T *c1, double h2, double ih2, double rho,
                  int color, cudaStream_t st, int rev = 0);

// Residual eps = L(u) - f of the fine level restricted to the coarse level.
// Correction form (fas = 0): fc = -R eps, uc = 0.  FAS (fas = 1, KPSI):
// fc = R eps, uc = urc = R u.  c0 is m for KHELM (the operator), s0 for KPSI.
template <typename T>
void resid_restrict(int kind, int nf, const T *u, const T *f, const T *c0, const T *c1, double ih2, double rho, T *uc,
                    T *fc, T *urc, int fas, cudaStream_t st);
// FP32 correction form of the same (KPOISSON or KHELM with m) right after a
// black relaxation pass: only the red children's residuals enter the average,
// the black ones being zero up to rounding.  h2c > 0: the coarse correction
// ec receives the coarse level's first red relaxation from zero instead of
// zeros (cinv: the coarse KHELM inverse diagonal), so that pass is skipped.
void resid_restrict_red(int kind, int nf, const float *e, const float *r, const float *m, double ih2, float *ec,
                        float *rc, const float *cinv, double h2c, cudaStream_t st, int rev = 0);

// FAS coarse right-hand side: fc = N(uc) - fc (KPSI, double).
void fas_rhs(int nc, const double *uc, double *fc, const double *c0, const double *c1, double ih2, double rho,
             cudaStream_t st);
// uc -= urc (the FAS coarse correction).
void fas_diff(int nc, double *uc, const double *urc, cudaStream_t st);

// Fine u += P(uc), cell-centred trilinear.
template <typename T>
void prolong_add(int nf, T *u, const T *uc, cudaStream_t st);
// FP32, black children only (a red relaxation of a linear equation follows)
void prolong_add_black(int nf, float *u, const float *uc, cudaStream_t st, int rev = 0);
// FP32 coarse = 8-child average of fine (a right-hand side going down)
void restrict_avg(int nf, const float *fine, float *coarse, cudaStream_t st);

// The 2^3 level in FP64 (any T storage).  KPOISSON, KHELM: solved exactly
// (Walsh-Hadamard diagonalisation; Gauss-Jordan elimination), Poisson with
// the source mean removed before and the solution mean after; KHELM reads
// c0 = m.  KPSI: kCoarsestSweeps Newton red-black sweeps, each followed by
// the constant shift that zeroes the sum of the eight residuals to first
// order (the Laplacian leaves that mode to the weak non-Laplacian terms).
template <typename T>
void coarsest(int kind, T *u, T *f, const T *c0, const T *c1, double h2, double ih2, double rho, cudaStream_t st);

// Coarse coefficients.  KPSI: c0c = R c0f, c1c = R c1f.  KHELM: c0c = R c0f
// (m) and c1c = 1/(6 + h2c c0c).
template <typename T>
void restrict_coef(int kind, int nf, const T *c0f, const T *c1f, T *c0c, T *c1c, double h2c, cudaStream_t st);
// KHELM inverse diagonal on one level: c1 = 1/(6 + h2 c0).
template <typename T>
void helm_invdiag(int n, const T *c0, T *c1, double h2, cudaStream_t st);

// Block partial sums of eps^2 and of u over a level (split layout);
// eps_nat (may be null) receives eps in natural layout (double).
// Partials: 2 doubles per block; returns the number of blocks.
template <typename T>
int resid_norm(int kind, int n, const T *u, const T *f, const T *c0, const T *c1, double ih2, double rho,
               double *partials, double *eps_nat, cudaStream_t st);
// out[0] = sum of partials[2b], out[1] = sum of partials[2b + 1].
void finalize(const double *partials, int nblk, double *out, cudaStream_t st);
// dst_mapped[0 .. cnt) = src[0 .. cnt) (cnt <= 32): dst_mapped is the device
// alias of pinned host memory allocated with cudaHostAllocMapped.
void scalars_out(const double *src, double *dst_mapped, int cnt, cudaStream_t st);

// The FP32 correction cycle's levels coarse_tail_n()^3 .. 2^3 in one thread
// block (shared memory): e/r/m/inv of levels 2^3, 4^3, 8^3, 16^3 (index 0 =
// 2^3); e and r of the top tail level in and e out; h2 per level.
int coarse_tail_n();
void coarse_tail(int kind, float *const *e, float *const *r, const float *const *m, const float *const *inv,
                 const double *h2, int nu1, int nu2, cudaStream_t st);

// The FP32 correction cycle's levels 64^3 .. 2^3 in one 16-CTA thread-block
// cluster (coarse_cluster.cu): arrays of levels 2^3 .. 64^3 (index 0 = 2^3);
// e and r of 64^3 in (its first red pass made by the restriction), e out.
// Needs nu1, nu2 >= 1.  coarse_cluster_ok: the device runs such a cluster
// (KPOISSON, KHELM).
bool coarse_cluster_ok(int kind);
void coarse_cluster(int kind, float *const *e, float *const *r, const float *const *m, const float *const *inv,
                    const double *h2, const double *ih2, int nu1, int nu2, cudaStream_t st);

// ---- mixed precision -------------------------------------------------------
// FP64 residual on the fine level; writes r32 = -eps (split), and for KPSI
// the Jacobian coefficient m32 = -dN/du > 0 and its inverse diagonal inv32.
int mixed_resid(int kind, int n, const double *u, const double *f, const double *c0, const double *c1, double ih2,
                double h2, double rho, float *r32, float *m32, float *inv32, double *partials, cudaStream_t st);
// u64 += e32 (split layout).
void mixed_update(int n, double *u, const float *e, cudaStream_t st);
// c32 = (float) c64.
void to_float(int64_t cnt, const double *a, float *b, cudaStream_t st);

// ---- double-float fine level (df_kernels.cu) -------------------------------
// hi/lo = a split into FP32 pairs; a = hi + lo.
// Fine residual in double-float: r32 = -eps, KPSI also m32/inv32 (Newton
// coefficient and FP32 inverse diagonal).  f, a = c0, b = c1 are pairs
// premultiplied by h^2 (KPOISSON, KHELM: h^2 f, h^2 m; KPSI: f' = h^2 f,
// a' = 2 pi h^2 s0, b' = h^2 AA / 8).  When e32 is not null it also writes the
// first red relaxation of the correction cycle from e = 0 (inv_in: the KHELM
// inverse diagonal).  Partials: block sums of (eps/ref)^2.  Returns the block
// count.
int df_resid(int kind, int n, const float *uh, const float *ul, const float *fh, const float *fl, const float *ah,
             const float *al, const float *bh, const float *bl, double h2, double rho, double ref, float *r32,
             float *m32, float *inv32, const float *inv_in, float *e32, double *partials, cudaStream_t st, int rev = 0,
             const double *fshift = nullptr);
void df_update(int n, float *uh, float *ul, const float *e, cudaStream_t st);
// last black pass of the FP32 correction cycle (KPOISSON or KHELM, n >= 8)
// fused with u += e on both colours; e's black half is left unwritten
void df_black_update(int kind, int n, const float *e, const float *r, const float *inv, double h2, float *uh,
                     float *ul, cudaStream_t st, int rev = 0);

// ---- double-float set-up and write-back (df_setup.cu) -----------------------
// Natural FP64 inputs -> split-layout hi/lo pairs, right-hand sides and
// coefficients premultiplied by h^2 as df_resid takes them (the callers pass
// the scales with h^2 folded in).  The int-returning ones
// leave block partials (sum, sum of squares of the high parts) of the
// quantity named and return the block count for finalize().
int dfs_sum(int64_t cnt, const double *a, double *partials, cudaStream_t st);                      // a
int dfs_pair_sum(int64_t cnt, const float *h, const float *l, double *partials, cudaStream_t st);  // h + l
// f = scale (s - sum[0]/n^3), u = fld; partials of f
int dfs_mean_rhs(int n, const double *s, const double *sum, double scale, const double *fld, float *uh, float *ul,
                 float *fh, float *fl, double *partials, cudaStream_t st);
// f = scale sum_l (F_l(+l) - F_l(-l)), u = fld; partials of f
int dfs_div_rhs(int n, double scale, const double *Fx, const double *Fy, const double *Fz, const double *fld,
                float *uh, float *ul, float *fh, float *fl, double *partials, cudaStream_t st);
// f = scale sum_l ((A^{comp l} w)(+l) - (A^{comp l} w)(-l)), u = fld; partials of f
int dfs_shift_rhs(int n, double scale, const float *A, const float *wh, const float *wl, int comp, const double *fld,
                  float *uh, float *ul, float *fh, float *fl, double *partials, cudaStream_t st);
// A_ij (12 n^3 floats: component c hi at A + 2c n^3, lo at A + (2c+1) n^3) and AA pairs, natural layout;
// scratch: four arrays of 2 n^3 floats for the pairs of V_x, V_y, V_z, U
void dfs_aij(int n, double inv2h, double ih2, const double *Vx, const double *Vy, const double *Vz, const double *U,
             float *const scratch[4], float *A, float *AAh, float *AAl, cudaStream_t st);
// psi: u = psi - 1, a = 2 pi h^2 s0, b = h^2 AA / 8, f = 0; partials of s0
int dfs_psi(int n, double h2, const double *psi, const double *s0, const float *AAh, const float *AAl, float *uh,
            float *ul, float *ah, float *al, float *bh, float *bl, float *fh, float *fl, double *partials,
            cudaStream_t st);
// alpha psi: u = alpha psi - 1, a = h^2 m, f = h^2 (m - psi^5 Kdot), m32, inv32; partials of psi^5 Kdot
int dfs_apsi(int n, double h2, const double *psi, const double *apsi, const double *s0, const double *sig,
             const float *AAh, const float *AAl, double K2, double Kdot, float *uh, float *ul, float *ah, float *al,
             float *fh, float *fl, float *m32, float *inv32, double *partials, cudaStream_t st);
// w = alpha psi psi^-7 pairs, natural layout
void dfs_weight(int n, const double *psi, const double *apsi, float *wh, float *wl, cudaStream_t st);
// out (natural) = hi + lo - sum[0]/n^3 (sum may be null) + (dev ? 1 : 0)
void dfs_store(int n, const float *uh, const float *ul, const double *sum, int dev, double *out, cudaStream_t st);

// ---- sources, coefficients, layouts (field_kernels.cu) ---------------------
void deposit(int n, double L, int64_t np, const double *x, const double *u, double mass, double *s0, double *sx,
             double *sy, double *sz, double *sig, cudaStream_t st);
// the deposit kernel alone, adding to the five arrays (no zeroing): for
// particles arriving in chunks
void deposit_add(int n, double L, int64_t np, const double *x, const double *u, double mass, double *s0, double *sx,
                 double *sy, double *sz, double *sig, cudaStream_t st);
// Partial sums of a and a^2 over cnt doubles; returns the block count.
int sum_sq(int64_t cnt, const double *a, double *partials, cudaStream_t st);
// a[i] = scale * (a[i] - s[0] / cnt_total), s a device scalar (a sum).
void scale_sub_mean(int64_t cnt, double *a, const double *sum, double inv_cnt, double scale, cudaStream_t st);
// natural -> split with a shift: split = nat + shift; split -> natural:
// nat = split + shift - sum[0] * inv_cnt (sum may be null).
void to_split(int n, const double *nat, double *split, double shift, cudaStream_t st);
void from_split(int n, const double *split, double *nat, double shift, const double *sum, double inv_cnt,
                cudaStream_t st);
// f (split) = scale * div3(F) from natural F (3-point central differences).
void div_to_split(int n, double inv2h, const double *Fx, const double *Fy, const double *Fz, double scale, double *f,
                  cudaStream_t st);
// A_ij (6 natural arrays: xx yy zz xy xz yz) and AA (natural) from V, U.
void aij_aa(int n, double inv2h, double ih2, const double *Vx, const double *Vy, const double *Vz, const double *U,
            double *A, double *AA, cudaStream_t st);
// psi equation: u = psi - 1, c0 = s0, c1 = AA, f = 0 (split).
void psi_setup(int n, const double *psi, const double *s0, const double *AA, double *u, double *c0, double *c1,
               double *f, cudaStream_t st);
// alpha psi equation: u = apsi - 1, c0 = m, c1 = 1/(6 + h^2 m), f = m - psi^5 Kdot (split);
// g = psi^5 Kdot (natural scratch) for the reference norm.
void apsi_setup(int n, double h2, const double *psi, const double *apsi, const double *s0, const double *sig,
                const double *AA, double K2, double Kdot, double *u, double *c0, double *c1, double *f, double *g,
                cudaStream_t st);
// B^i source: f (split) = 2 sum_j D_j (w A^ij), w = apsi psi^-7 (natural scratch).
void shift_weight(int n, const double *psi, const double *apsi, double *w, cudaStream_t st);
void shift_source(int n, double inv2h, const double *A, const double *w, int comp, double *f, cudaStream_t st);

// ---- particles (particle_kernels.cu) ----------------------------------------
// The per-cell records of the particle update: 20 FP32 quantities (alpha - 1,
// psi - 1, beta^j, D_i alpha, D_i psi, D_i beta^j at 11 + 3 j + i), 80 bytes
// per cell (rec: 20 n^3 floats, 16-byte aligned), from the natural FP64
// fields; dev is FP32 scratch of 5 n^3 floats.
void particle_fields(int n, double L, const double *psi, const double *apsi, const double *Bx, const double *By,
                     const double *Bz, const double *b, float *dev, float *rec, cudaStream_t st);
// Kicks and drift of np particles (x, u: [3][np] device SoA) with the flags
// GR_KICK_SYNC, GR_KICK_OPEN, GR_DRIFT.
void particle_update(int n, double L, int64_t np, double *x, double *u, const float *rec, double dt, int flags,
                     cudaStream_t st);
// The deposit with W = sqrt(1 + psi^-4 |u|^2), psi interpolated at the particle.
void deposit_metric(int n, double L, int64_t np, const double *x, const double *u, double mass, const double *psi,
                    double *s0, double *sx, double *sy, double *sz, double *sig, cudaStream_t st);

// ---- code units (codeunits.cu) ----------------------------------------------
struct CuPtrs {
    double *p[10];  // sources: s0 s_x s_y s_z sigma; fields: psi apsi V_x V_y V_z U B^x B^y B^z b
};
struct CuScale {
    double s[5];   // source scales (code units -> the a = 1 problem)
    double f[10];  // field scales of the potentials (entries 2..9)
};
// code-unit sources -> scaled copies; code-unit fields -> the a = 1 form, in place
void code_units_in(int64_t N, const CuPtrs &src_in, const CuPtrs &src_out, const CuScale &sc, const CuPtrs &fld,
                   double a2c2, cudaStream_t st);
// the a = 1 solution -> code-unit fields, in place
void code_units_out(int64_t N, const CuScale &sc, const CuPtrs &fld, double a2c2, cudaStream_t st);

// ---------------------------------------------------------------- nested patches
// Base level as the patch kernels see it: natural FP64 fields (PB_NAT, nat),
// the FP64 split-layout arrays of a solve (PB_SPLIT: u, f, c0, c1 as the
// FP64 relaxation uses them) or the double-float split-layout arrays
// (PB_DF: uh/ul, fh/fl = h^2 f, ah/al, bh/bl = the h^2-scaled coefficients).
enum PatchBaseFmt : int { PB_NAT = 0, PB_SPLIT = 1, PB_DF = 2 };
struct PBase {
    int lgn = 0;
    const double *nat = nullptr;
    double *u = nullptr, *f = nullptr;
    const double *c0 = nullptr, *c1 = nullptr;
    float *uh = nullptr, *ul = nullptr, *fh = nullptr, *fl = nullptr;
    const float *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    double h2 = 0, ih2 = 0, rho = 0;
};
// One patch level: ghosted (n + 4)^3 arrays; co/cnc the block its child
// covers (cnc = 0: none); lam the Poisson solvability constant (NULL: none).
// The working unknown is u (FP64) or the pair uh/ul (the double-float
// relaxation of the mixed modes, with the h^2-scaled pairs fh/fl, ah/al,
// bh/bl of the right-hand side and coefficients, cpr = 2 pi rho h^2 and
// c5 = 10 pi rho h^2); f, c0, c1 are the FP64 right-hand side and
// coefficients (Helmholtz c1: 1 / (6 + h^2 m)).
struct PPatch {
    int lgn = 0, m = 0;
    double *u = nullptr, *f = nullptr;
    const double *c0 = nullptr, *c1 = nullptr;
    float *uh = nullptr, *ul = nullptr, *fh = nullptr, *fl = nullptr;
    float *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    df cpr = {0.0f, 0.0f};
    float c5 = 0.0f;
    double h2 = 0, ih2 = 0, rho = 0;
    int co[3] = {0, 0, 0}, cnc = 0;
    const double *lam = nullptr;
};
struct PSetSrc {
    double *s[5];  // s0 s_x s_y s_z sigma, natural n^3
};
struct PSetFld {
    const double *g[10];  // ghosted fields, setup order V_x V_y V_z U psi apsi B^x B^y B^z b
};
void patch_deposit(int64_t np, const double *x, const double *u, double mass, double L, int N, const int O[3], int nw,
                   const PSetSrc &out, cudaStream_t st);
// indices of the particles in base cells [lo, lo + len) (mod n0) per axis -> list, their number -> count
void patch_select(int64_t np, const double *x, double L, int n0, const int lo[3], int len, int *list,
                  unsigned *count, cudaStream_t st);
// patch_deposit over the particles of such a list (np: the particle arrays' length)
void patch_deposit_list(int64_t np, const int *list, const unsigned *count, const double *x, const double *u,
                        double mass, double L, int N, const int O[3], int nw, const PSetSrc &out, cudaStream_t st);
// win = the parent's window; with dold, also dold := win - dold (and d32 its FP32 copy)
void patch_gather_base(int fmt, const PBase &B, const int o[3], int w, double *win, cudaStream_t st,
                       double *dold = nullptr, float *d32 = nullptr);
void patch_gather_patch(const PPatch &par, bool pdf, const int o[3], int w, double *win, cudaStream_t st,
                        double *dold = nullptr, float *d32 = nullptr);
// ghosts of the unknown = P(win); with d (or its FP32 copy d32 for pdf), the interior += P(d)
void patch_interp(const PPatch &P, bool pdf, const double *win, const double *d, const float *d32, cudaStream_t st);
void patch_gs(int kind, const PPatch &P, bool pdf, int color, cudaStream_t st);
int patch_resid(int kind, const PPatch &P, bool pdf, double *eps, double *partials, cudaStream_t st);
void patch_restrict(const PPatch &P, bool pdf, const double *eps, double *Ru, double *Re, cudaStream_t st);
void patch_inject_u_base(int fmt, const PBase &B, const int o[3], int nc, const double *Ru, cudaStream_t st);
int patch_inject_f_base(int fmt, int kind, const PBase &B, const int o[3], int nc, const double *Re, const double *lam,
                        double *partials, cudaStream_t st);
int patch_sum_f_base(int fmt, const PBase &B, const int o[3], int nc, double *partials, cudaStream_t st);
void patch_inject_u_patch(const PPatch &par, bool pdf, const int o[3], int nc, const double *Ru, cudaStream_t st);
void patch_inject_f_patch(int kind, const PPatch &par, bool pdf, const int o[3], int nc, const double *Re,
                          cudaStream_t st);
void patch_reflux(int parent_fmt, const PBase &B, const PPatch &par, const PPatch &ch, bool pdf, const int o[3],
                  double hc, double *flux, cudaStream_t st);
void patch_lambda(double *sc, const double *flux, int nq, double N, double Ncov, double *lam, cudaStream_t st);
void sub_scalar(int64_t cnt, double *a, const double *m, cudaStream_t st);
void patch_to_ghosted(int n, const double *in, double *out, double add, cudaStream_t st);
void patch_u_load(const PPatch &P, bool pdf, const double *in, double add, cudaStream_t st);
void patch_u_store(const PPatch &P, bool pdf, double *out, double *keep, double add, const double *usum, double scale,
                   cudaStream_t st);
void patch_coef_df(int kind, const PPatch &P, cudaStream_t st);
// A_ij of the ghosted V, U on the interior and first ghost layer (six ghosted arrays)
void patch_aij(int n, double nh, const PSetFld &G, double *A6, cudaStream_t st);
int patch_setup(int eq, int n, double nh, const PSetSrc &S, const PSetFld &G, const double *A6, double smean,
                double K2, double Kdot, double *f, double *c0, double *c1, double *partials, cudaStream_t st);

// Three FP32 colour passes of the correction equation (KPOISSON, KHELM) in
// one pass over memory: colour c1 from the other colour of ein, then the other
// colour, then c1 again; both colours of the result go to eout (smooth3.cu).
// inv: KHELM's 1/(6 + h^2 m).  rt: row tiles (smooth3_row_tiles).
bool smooth3_fits(int kind, int n);
int smooth3_row_tiles(int n, int sms);
void smooth3(int kind, int n, const float *ein, float *eout, const float *f, const float *inv, double h2, int c1,
             int rt, cudaStream_t st);

}  // namespace gr
