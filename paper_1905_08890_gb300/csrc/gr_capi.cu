// gr_capi.cu - host orchestration and the C ABI declared in include/gr.h.
//
// Each equation is solved on a hierarchy of levels n, n/2, ..., 2 (Sec. 4.3.1,
// last paragraph) held in red-black split layout.  FP64 path: V(nu1, nu2)
// cycles, correction form for the linear equations (Eq. GR-linear-coarse),
// full approximation scheme for psi (Sec. 4.3.2.1).  Mixed paths: a
// defect-correction loop whose correction equation lap e - m e = -eps is
// relaxed by one FP32 V-cycle per iteration (for psi, m is the Newton
// linearisation of the Hamiltonian-constraint operator; optionally a full
// multigrid cycle for the first iteration); the fine residual and update are
// FP64 (GR_PREC_MIXED) or double-float, with the finest level's set-up and
// write-back too (GR_PREC_MIXED_DF); the 2^3 level and all reductions' last
// stages stay FP64.  Host-buffer I/O runs on a copy stream of the context.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gr.h"
#include "gr_internal.cuh"

using namespace gr;

std::atomic<long long> gr::g_launches{0};

namespace {

thread_local std::string g_err;

gr_status fail(gr_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

struct Level {
    int n = 0;
    double h = 0, h2 = 0, ih2 = 0;
    double *u = nullptr, *f = nullptr, *c0 = nullptr, *c1 = nullptr, *ur = nullptr;  // FP64
    float *e = nullptr, *r = nullptr, *m = nullptr, *inv = nullptr;                 // FP32
    float *e2 = nullptr;  // finest level: second correction buffer of the fused colour passes
};

// one patch of a chain (gr_patch): ghosted (n + 4)^3 FP64 work arrays
struct PatchLevel {
    int n = 0, lgn = 0, m = 0, nc = 0, w = 0;
    int o[3] = {0, 0, 0};
    double h = 0;                                     // spacing
    double *u = nullptr, *f = nullptr, *c0 = nullptr, *c1 = nullptr, *eps = nullptr;
    double *G[GR_NEQ] = {};                           // the fields, interior = latest solution, ghosts on demand
    double *win = nullptr, *old = nullptr;            // parent windows, (n/2 + 4)^3
    double *Ru = nullptr, *Re = nullptr;              // restricted u and residual, (n/2)^3
    double *flux = nullptr;                           // flux corrections in force, 6 (n/2)^2
    double *A6 = nullptr;                             // A_ij of the solved V, U (6 ghosted arrays)
    // the double-float relaxation (mixed modes): unknown, h^2 f and h^2-scaled coefficients as FP32 pairs
    float *uh = nullptr, *ul = nullptr, *fh = nullptr, *fl = nullptr;
    float *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    float *d32 = nullptr;                             // the parent's change on the window, FP32
    double ref = 1;
};

struct EqInfo {
    int kind;      // operator on the FP64 fine level
    int kind32;    // operator of the FP32 correction equation
    int dev;       // unknown is field - 1
    int poisson;   // zero-mean solution
    double ref;    // reference norm of the relative residual
};

}  // namespace

struct gr_ctx {
    int n = 0, nlev = 0;
    double L = 1, h = 1;
    cudaStream_t st = nullptr;
    std::vector<Level> lev;  // lev[0] is 2^3, lev[nlev-1] the finest
    double *A6 = nullptr, *AA = nullptr, *tmp = nullptr;
    float *dfu = nullptr, *dff = nullptr, *dfa = nullptr, *dfb = nullptr;  // finest level hi|lo pairs
    double *partials = nullptr, *dscal = nullptr;
    double *hscal = nullptr, *hscal_dev = nullptr;  // mapped pinned host scalars and their device alias
    double rho_dep = NAN;
    // what A6/AA hold for the V, U in the fields, and tmp (alpha psi psi^-7) for
    // the psi, alpha psi in the fields: 0 nothing current, 1 FP64, 2 double-float pairs
    int a_fmt = 0;
    int w_fmt = 0;
    bool tail_on = true;   // FP32 cycles: levels <= 16^3 in one block (GR_COARSE_TAIL=0 turns it off)
    bool cluster_on = false;  // FP32 cycles under a 128^3 or finer top: levels <= 64^3 in one
                              // 16-CTA cluster (GR_COARSE_CLUSTER=1; measured slower)
    int s3_min = 1 << 30;  // finest grids from this size fuse three colour passes per smoothing: off unless
                           // GR_SMOOTH3=1 (from 512^3, or from GR_SMOOTH3_MIN)
    int s3_rt = 0;         // row tiles of the fused colour passes on the finest level
    int dir = 0;           // traversal direction of the next finest-level launch (alternates)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // host-buffer I/O: a copy stream, its events and two particle staging buffers
    cudaStream_t cs = nullptr;
    cudaEvent_t ready[2] = {}, used[2] = {}, xfer = nullptr;
    double *stage[2] = {};
    int64_t stage_cap = 0;            // particles per staging buffer
    int64_t host_chunk = 4 << 20;     // particles per host chunk (GR_HOST_CHUNK)
    std::vector<void *> allocs;
    // finest-level kernel timing (gr_opts.profile)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    int prof_launches[GR_NPROF] = {};
    double prof_ms[GR_NPROF] = {};
    // nested patches: work arrays of the current chain, device scalars (0: the
    // Poisson solvability constant, 1..8: its sums, 16..: set-up sums, 32..: norms)
    std::vector<PatchLevel> pl;
    std::vector<void *> palloc;
    double *pdev = nullptr, *phost = nullptr, *phost_dev = nullptr;  // phost: mapped pinned, phost_dev its alias
    bool pdf = false;  // the patches relax in double-float (mixed modes) rather than FP64
    // particle update: the per-cell records of 20 FP32 quantities (allocated on first use)
    float *pf = nullptr;
    // code units: the scaled sources of the a = 1 problem (allocated on first use)
    double *cu_src = nullptr;
    // patch deposits: indices of the particles near the first patch, and their number
    int *plist = nullptr;
    int64_t plist_cap = 0;
    unsigned *pcount = nullptr;
};

namespace {

}  // namespace

void gr::set_last_error(const char *msg) { g_err = msg; }

namespace {

gr_status cuda_check(const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GR_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    return GR_OK;
}

template <typename T>
gr_status dalloc(gr_ctx *c, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) < 256 ? 256 : count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GR_ERR_NOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *p = (T *)q;
    return GR_OK;
}

int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

bool valid_opts(const gr_opts *o)
{
    return o && !(o->tol < 0) && o->max_cycles >= 0 && o->nu1 >= 0 && o->nu1 <= 8 && o->nu2 >= 0 && o->nu2 <= 8 &&
           (o->prec == GR_PREC_FP64 || o->prec == GR_PREC_MIXED || o->prec == GR_PREC_MIXED_DF) &&
           o->npatch >= 0 && o->npatch <= GR_MAX_PATCHES && (o->npatch == 0 || o->patch);
}

// non-NULL and on a 16-byte boundary (the set-up and write-back kernels move
// the natural-layout arrays in 16-byte vectors)
bool a16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }

bool src_ok(const gr_sources *s)
{
    return s && a16(s->s0) && a16(s->s[0]) && a16(s->s[1]) && a16(s->s[2]) && a16(s->sigma);
}

bool fld_ok(const gr_fields *f)
{
    return f && a16(f->psi) && a16(f->apsi) && a16(f->V[0]) && a16(f->V[1]) && a16(f->V[2]) && a16(f->U) &&
           a16(f->B[0]) && a16(f->B[1]) && a16(f->B[2]) && a16(f->b);
}

double *field_ptr(const gr_fields *f, int eq)
{
    switch (eq) {
    case GR_VX: return f->V[0];
    case GR_VY: return f->V[1];
    case GR_VZ: return f->V[2];
    case GR_U: return f->U;
    case GR_PSI: return f->psi;
    case GR_APSI: return f->apsi;
    case GR_BX: return f->B[0];
    case GR_BY: return f->B[1];
    case GR_BZ: return f->B[2];
    default: return f->b;
    }
}

// device sums (sum, sum of squares) of cnt doubles into c->dscal[0..1]
void dsum(gr_ctx *c, int64_t cnt, const double *a)
{
    int g = gr::sum_sq(cnt, a, c->partials, c->st);
    gr::finalize(c->partials, g, c->dscal, c->st);
}

cudaEvent_t pool_event(gr_ctx *c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Run f (which queues finest-level kernels) and, when profiling, bracket it
// with a pair of events attributed to class cls.
template <class F>
void timed(gr_ctx *c, int cls, F &&f)
{
    if (!c->prof_on) {
        f();
        return;
    }
    const long long before = gr::g_launches.load(std::memory_order_relaxed);
    cudaEvent_t a = pool_event(c), b = pool_event(c);
    cudaEventRecord(a, c->st);
    f();
    cudaEventRecord(b, c->st);
    c->pending.push_back({cls, a, b});
    c->prof_launches[cls] += (int)(gr::g_launches.load(std::memory_order_relaxed) - before);
}

// after a stream synchronisation: accumulate the finished event pairs
void prof_collect(gr_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->prof_ms[p.cls] += ms;
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->pending.clear();
    cudaGetLastError();
}

gr_status read_scalars(gr_ctx *c, double *a, double *b)
{
    // a kernel store, not a copy: a device-to-host copy would wait for the
    // field copies that host_out keeps in flight on the copy stream
    gr::scalars_out(c->dscal, c->hscal_dev, 2, c->st);
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(GR_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    gr_status s = cuda_check("kernel");
    if (s != GR_OK) return s;
    if (c->prof_on) prof_collect(c);
    const volatile double *h = c->hscal;
    *a = h[0];
    if (b) *b = h[1];
    return GR_OK;
}

// mean-free Poisson right-hand side on the fine level (split layout);
// ref = RMS after the first mean removal, then the mean is removed again
gr_status poisson_rhs_finish(gr_ctx *c, Level &F, double *ref)
{
    const int64_t N = (int64_t)c->n * c->n * c->n;
    dsum(c, N, F.f);
    gr::scale_sub_mean(N, F.f, c->dscal, 1.0 / N, 1.0, c->st);
    dsum(c, N, F.f);
    double s, q;
    gr_status st = read_scalars(c, &s, &q);
    if (st != GR_OK) return st;
    *ref = std::sqrt(q / N);
    gr::scale_sub_mean(N, F.f, c->dscal, 1.0 / N, 1.0, c->st);
    return GR_OK;
}

void ensure_aij(gr_ctx *c, const gr_fields *fl)
{
    if (c->a_fmt == 1) return;
    gr::aij_aa(c->n, 0.5 / c->h, 1.0 / (c->h * c->h), fl->V[0], fl->V[1], fl->V[2], fl->U, c->A6, c->AA, c->st);
    c->a_fmt = 1;
}

// Build the fine-level unknown, right-hand side and coefficients of equation eq
// (split layout) from the sources and current fields; fills info.
gr_status setup_eq(gr_ctx *c, int eq, const gr_sources *s, const gr_fields *fl, double rho, double S_hat, EqInfo *info)
{
    const int n = c->n;
    const int64_t N = (int64_t)n * n * n;
    Level &F = c->lev[c->nlev - 1];
    const double K2 = 24.0 * kPi * rho, Kdot = 12.0 * kPi * rho + 4.0 * kPi * S_hat;
    info->dev = (eq == GR_PSI || eq == GR_APSI);
    info->poisson = !info->dev;
    info->kind = eq == GR_PSI ? KPSI : (eq == GR_APSI ? KHELM : KPOISSON);
    info->kind32 = info->kind == KPOISSON ? KPOISSON : KHELM;
    gr_status st = GR_OK;
    if (eq <= GR_VZ) {
        // lap V_i = 8 pi (s_i - <s_i>)  (Eq. MG-linear-1a; mean removal of Sec. 4.3.1)
        gr::to_split(n, s->s[eq], F.f, 0.0, c->st);
        dsum(c, N, F.f);
        gr::scale_sub_mean(N, F.f, c->dscal, 1.0 / N, 8.0 * kPi, c->st);
        st = poisson_rhs_finish(c, F, &info->ref);
    } else if (eq == GR_U || eq == GR_B_SCALAR) {
        // lap U = -1/4 div V ; lap b = -1/4 div B  (Eqs. MG-linear-1, MG-linear-2)
        double *const *Fv = eq == GR_U ? fl->V : fl->B;
        gr::div_to_split(n, 0.5 / c->h, Fv[0], Fv[1], Fv[2], -0.25, F.f, c->st);
        st = poisson_rhs_finish(c, F, &info->ref);
    } else if (eq == GR_PSI) {
        ensure_aij(c, fl);
        gr::psi_setup(n, fl->psi, s->s0, c->AA, F.u, F.c0, F.c1, F.f, c->st);
        dsum(c, N, s->s0);
        double a, q;
        st = read_scalars(c, &a, &q);
        info->ref = 2.0 * kPi * std::sqrt(q / N);
    } else if (eq == GR_APSI) {
        ensure_aij(c, fl);
        gr::apsi_setup(n, c->h * c->h, fl->psi, fl->apsi, s->s0, s->sigma, c->AA, K2, Kdot, F.u, F.c0, F.c1, F.f,
                       c->tmp, c->st);
        c->w_fmt = 0;  // tmp now holds psi^5 Kdot
        dsum(c, N, c->tmp);
        double a, q;
        st = read_scalars(c, &a, &q);
        info->ref = std::sqrt(q / N);
    } else {
        // lap B^i = 2 d_j (alpha psi^-6 A^ij)  (Eqs. MDC-CF, MG-linear-2a)
        ensure_aij(c, fl);
        if (c->w_fmt != 1) gr::shift_weight(n, fl->psi, fl->apsi, c->tmp, c->st);
        c->w_fmt = 1;
        gr::shift_source(n, 0.5 / c->h, c->A6, c->tmp, eq - GR_BX, F.f, c->st);
        st = poisson_rhs_finish(c, F, &info->ref);
    }
    if (st != GR_OK) return st;
    if (!info->dev) gr::to_split(n, field_ptr(fl, eq), F.u, 0.0, c->st);
    if (!(info->ref >= 1e-300)) info->ref = 1.0;
    return cuda_check("setup");
}

// Double-float set-up of equation eq: unknown, right-hand side and
// coefficients as split-layout pairs in dfu, dff, dfa, dfb (and, for alpha psi,
// lev[fine].m and .inv), from the natural FP64 sources and fields; the
// right-hand side and coefficients premultiplied by h^2 as df_resid takes them.  The same
// equations as setup_eq; the Poisson right-hand sides lose their mean once in
// double-float, which leaves it at the double-float rounding level.
gr_status setup_eq_df(gr_ctx *c, int eq, const gr_sources *s, const gr_fields *fl, double rho, double S_hat,
                      EqInfo *info)
{
    const int n = c->n;
    const int64_t N = (int64_t)n * n * n;
    Level &F = c->lev[c->nlev - 1];
    const double K2 = 24.0 * kPi * rho, Kdot = 12.0 * kPi * rho + 4.0 * kPi * S_hat;
    info->dev = (eq == GR_PSI || eq == GR_APSI);
    info->poisson = !info->dev;
    info->kind = eq == GR_PSI ? KPSI : (eq == GR_APSI ? KHELM : KPOISSON);
    info->kind32 = info->kind == KPOISSON ? KPOISSON : KHELM;
    float *uh = c->dfu, *ul = c->dfu + N, *fh = c->dff, *fl_ = c->dff + N;
    float *A = reinterpret_cast<float *>(c->A6), *AAh = reinterpret_cast<float *>(c->AA), *AAl = AAh + N;
    float *wh = reinterpret_cast<float *>(c->tmp), *wl = wh + N;
    double *fld = field_ptr(fl, eq);
    auto aij = [&] {
        if (c->a_fmt == 2) return;
        // the finest level's FP64 arrays are free in this mode: scratch for the pairs of V and U
        float *const scratch[4] = {reinterpret_cast<float *>(F.u), reinterpret_cast<float *>(F.f),
                                   reinterpret_cast<float *>(F.c0), reinterpret_cast<float *>(F.c1)};
        gr::dfs_aij(n, 0.5 / c->h, 1.0 / (c->h * c->h), fl->V[0], fl->V[1], fl->V[2], fl->U, scratch, A, AAh, AAl,
                    c->st);
        c->a_fmt = 2;
    };
    int g;
    if (eq <= GR_VZ) {
        // lap V_i = 8 pi (s_i - <s_i>)  (Eq. MG-linear-1a; mean removal of Sec. 4.3.1)
        g = gr::dfs_sum(N, s->s[eq], c->partials, c->st);
        gr::finalize(c->partials, g, c->dscal, c->st);
        g = gr::dfs_mean_rhs(n, s->s[eq], c->dscal, 8.0 * kPi * F.h2, fld, uh, ul, fh, fl_, c->partials, c->st);
    } else if (eq == GR_U || eq == GR_B_SCALAR) {
        // lap U = -1/4 div V ; lap b = -1/4 div B  (Eqs. MG-linear-1, MG-linear-2)
        double *const *Fv = eq == GR_U ? fl->V : fl->B;
        g = gr::dfs_div_rhs(n, -0.25 * (0.5 / c->h) * F.h2, Fv[0], Fv[1], Fv[2], fld, uh, ul, fh, fl_, c->partials,
                            c->st);
    } else if (eq == GR_PSI) {
        aij();
        g = gr::dfs_psi(n, F.h2, fl->psi, s->s0, AAh, AAl, uh, ul, c->dfa, c->dfa + N, c->dfb, c->dfb + N, fh, fl_,
                        c->partials, c->st);
    } else if (eq == GR_APSI) {
        aij();
        g = gr::dfs_apsi(n, F.h2, fl->psi, fl->apsi, s->s0, s->sigma, AAh, AAl, K2, Kdot, uh, ul, c->dfa, c->dfa + N,
                         fh, fl_, F.m, F.inv, c->partials, c->st);
    } else {
        // lap B^i = 2 d_j (alpha psi^-6 A^ij)  (Eqs. MDC-CF, MG-linear-2a)
        aij();
        if (c->w_fmt != 2) gr::dfs_weight(n, fl->psi, fl->apsi, wh, wl, c->st);
        c->w_fmt = 2;
        g = gr::dfs_shift_rhs(n, 2.0 * (0.5 / c->h) * F.h2, A, wh, wl, eq - GR_BX, fld, uh, ul, fh, fl_,
                              c->partials, c->st);
    }
    gr::finalize(c->partials, g, c->dscal, c->st);
    double a, q;
    gr_status st = read_scalars(c, &a, &q);
    if (st != GR_OK) return st;
    if (info->poisson) {  // the sums are of h^2 f
        const double mean = a / N;
        info->ref = std::sqrt(std::fmax(q / N - mean * mean, 0.0)) / F.h2;
    } else {
        info->ref = (eq == GR_PSI ? 2.0 * kPi : 1.0) * std::sqrt(q / N);
    }
    if (!(info->ref >= 1e-300)) info->ref = 1.0;
    return cuda_check("setup");
}

void restrict_coefs64(gr_ctx *c, int kind)
{
    if (kind == KPOISSON) return;
    for (int l = c->nlev - 1; l >= 1; l--) {
        Level &A = c->lev[l], &C = c->lev[l - 1];
        gr::restrict_coef<double>(kind, A.n, A.c0, A.c1, C.c0, C.c1, C.h2, c->st);
    }
}

void restrict_coefs32(gr_ctx *c)
{
    for (int l = c->nlev - 1; l >= 1; l--) {
        Level &A = c->lev[l], &C = c->lev[l - 1];
        gr::restrict_coef<float>(KHELM, A.n, A.m, A.inv, C.m, C.inv, C.h2, c->st);
    }
}

// cells relaxed by one V-cycle whose top is level top (default: the finest);
// coarsest: the cell updates of the 2^3 solve (8 for the exact solve of a
// linear level, 8 per sweep for the nonlinear one)
long long vcycle_cells(const gr_ctx *c, int nu1, int nu2, int top = -1, long long coarsest = 8)
{
    if (top < 0) top = c->nlev - 1;
    long long s = 0;
    for (int l = 1; l <= top; l++) s += (long long)(nu1 + nu2) * c->lev[l].n * c->lev[l].n * c->lev[l].n;
    return s + coarsest;
}

// cells relaxed by one full multigrid cycle (fmg32, linear correction levels)
long long fmg_cells(const gr_ctx *c, int nu1, int nu2)
{
    long long s = 2 * vcycle_cells(c, nu1, nu2, 3);
    for (int l = 4; l < c->nlev; l++) s += vcycle_cells(c, nu1, nu2, l);
    return s;
}

// Relaxation and transfers of one V-cycle.  With profiling, the finest
// level's launches are timed per class and everything below it (which runs
// as one contiguous stretch between the finest restriction and
// prolongation) as GR_PROF_COARSE.
void vcycle64(gr_ctx *c, int kind, double rho, int nu1, int nu2)
{
    const int fas = kind == KPSI;
    const int top = c->nlev - 1;
    auto smooth = [&](Level &A, int nu) {
        for (int s = 0; s < nu; s++)
            for (int col = 0; col < 2; col++)
                gr::sweep_colour<double>(kind, A.n, A.u, A.f, A.c0, A.c1, A.h2, A.ih2, rho, col, c->st);
    };
    auto down = [&](int l) {
        Level &A = c->lev[l], &C = c->lev[l - 1];
        gr::resid_restrict<double>(kind, A.n, A.u, A.f, A.c0, A.c1, A.ih2, rho, C.u, C.f, C.ur, fas, c->st);
        if (fas) gr::fas_rhs(C.n, C.u, C.f, C.c0, C.c1, C.ih2, rho, c->st);
    };
    auto up = [&](int l) {
        Level &A = c->lev[l], &C = c->lev[l - 1];
        if (fas) gr::fas_diff(C.n, C.u, C.ur, c->st);
        gr::prolong_add<double>(A.n, A.u, C.u, c->st);
    };
    Level &F = c->lev[top];
    timed(c, GR_PROF_SWEEP64, [&] { smooth(F, nu1); });
    timed(c, GR_PROF_RESTRICT, [&] { down(top); });
    timed(c, GR_PROF_COARSE, [&] {
        for (int l = top - 1; l >= 1; l--) {
            smooth(c->lev[l], nu1);
            down(l);
        }
        Level &Z = c->lev[0];
        gr::coarsest<double>(kind, Z.u, Z.f, Z.c0, Z.c1, Z.h2, Z.ih2, rho, c->st);
        for (int l = 1; l < top; l++) {
            up(l);
            smooth(c->lev[l], nu2);
        }
    });
    timed(c, GR_PROF_PROLONG, [&] { up(top); });
    timed(c, GR_PROF_SWEEP64, [&] { smooth(F, nu2); });
}

// direction for the next finest-level launch; consecutive launches alternate
// so that each starts on the data its predecessor touched last
int next_dir(gr_ctx *c)
{
    const int d = c->dir;
    c->dir ^= 1;
    return d;
}

// How a correction V-cycle finds its top level's e: zero (cleared here), the
// first red relaxation from zero already made (by the fine residual kernel;
// the black cells are then not read before they are written), or a given
// initial e (full multigrid).
enum Start { START_ZERO = 0, START_RED_DONE = 1, START_GIVEN = 2 };

// One FP32 correction V-cycle on lev[*].e with right-hand side lev[top].r,
// top = the finest level unless given (full multigrid's coarser cycles, all
// timed as GR_PROF_COARSE).  uh, ul not null (needs nu2 >= 1 and a top level
// of at least 8^3): the last black pass also adds e to the double-float
// unknown (uh, ul).
void vcycle32(gr_ctx *c, int kind32, int nu1, int nu2, Start start, float *uh = nullptr, float *ul = nullptr,
              int top = -1)
{
    if (top < 0) top = c->nlev - 1;
    const bool fine = top == c->nlev - 1;
    auto cls = [&](int k) { return fine ? k : (int)GR_PROF_COARSE; };
    Level &F = c->lev[top];
    // finest-level launches alternate their traversal direction
    auto dir_of = [&](const Level &A) { return (fine && &A == &F) ? next_dir(c) : 0; };
    auto smooth = [&](Level &A, int nu) {
        for (int s = 0; s < nu; s++)
            for (int col = 0; col < 2; col++)
                gr::sweep_colour<float>(kind32, A.n, A.e, A.r, A.m, A.inv, A.h2, A.ih2, 0.0, col, c->st, dir_of(A));
    };
    // levels up to 16^3 run in one block (coarse_tail) when the top is finer than that
    const int tail = (top > 3 && c->tail_on) ? 3 : 0;
    // after a black pre-smoothing pass only red residuals are restricted; a
    // coarse level relaxed by separate launches (above the tail, not the 2^3
    // solve) also gets its first red pass from the restriction
    auto first_red_from_restrict = [&](int lc) { return nu1 > 0 && lc >= 1 && lc > (tail ? tail : 0); };
    auto down = [&](int l) {
        Level &A = c->lev[l], &C = c->lev[l - 1];
        if (nu1 > 0) {
            const bool fr = first_red_from_restrict(l - 1);
            gr::resid_restrict_red(kind32, A.n, A.e, A.r, A.m, A.ih2, C.e, C.r, fr ? C.inv : nullptr, fr ? C.h2 : 0.0,
                                   c->st, dir_of(A));
        } else {
            gr::resid_restrict<float>(kind32, A.n, A.e, A.r, A.m, A.inv, A.ih2, 0.0, C.e, C.r, nullptr, 0, c->st);
        }
    };
    // pre-smoothing of a coarse level whose first red pass the restriction made
    auto smooth_after_restrict = [&](Level &A, int lc) {
        if (!first_red_from_restrict(lc)) {
            smooth(A, nu1);
            return;
        }
        gr::sweep_colour<float>(kind32, A.n, A.e, A.r, A.m, A.inv, A.h2, A.ih2, 0.0, 1, c->st, dir_of(A));
        smooth(A, nu1 - 1);
    };
    // a red pass follows each prolongation when nu2 > 0: only black cells need the correction
    auto up = [&](int l) {
        if (nu2 > 0) gr::prolong_add_black(c->lev[l].n, c->lev[l].e, c->lev[l - 1].e, c->st, dir_of(c->lev[l]));
        else gr::prolong_add<float>(c->lev[l].n, c->lev[l].e, c->lev[l - 1].e, c->st);
    };
    // finest level with two sweeps: three of the colour passes fused into one
    // pass over memory (smooth3.cu), colour `first` first; the result lands in
    // the second buffer, which becomes the level's correction
    auto fused3 = [&](int nu, int first) {
        if (!fine || nu != 2 || !F.e2 || !gr::smooth3_fits(kind32, F.n)) return false;
        timed(c, GR_PROF_SMOOTH3, [&] {
            gr::smooth3(kind32, F.n, F.e, F.e2, F.r, F.inv, F.h2, first, c->s3_rt, c->st);
        });
        std::swap(F.e, F.e2);
        return true;
    };
    // nu red + black sweeps of the finest level
    auto smooth_fine = [&](int nu) {
        if (fused3(nu, 0)) {
            timed(c, cls(GR_PROF_SWEEP32), [&] {
                gr::sweep_colour<float>(kind32, F.n, F.e, F.r, F.m, F.inv, F.h2, F.ih2, 0.0, 1, c->st, dir_of(F));
            });
        } else {
            timed(c, cls(GR_PROF_SWEEP32), [&] { smooth(F, nu); });
        }
    };
    if (start == START_RED_DONE && nu1 > 0) {
        if (!fused3(nu1, 1)) {
            timed(c, cls(GR_PROF_SWEEP32), [&] {
                gr::sweep_colour<float>(kind32, F.n, F.e, F.r, F.m, F.inv, F.h2, F.ih2, 0.0, 1, c->st, dir_of(F));
                smooth(F, nu1 - 1);
            });
        }
    } else {
        if (start != START_GIVEN) cudaMemsetAsync(F.e, 0, sizeof(float) * (size_t)F.n * F.n * F.n, c->st);
        smooth_fine(nu1);
    }
    timed(c, cls(GR_PROF_RESTRICT), [&] { down(top); });
    // levels 64^3 .. 2^3 in one cluster launch below a 128^3 or finer top
    const bool clus = tail && c->cluster_on && top >= 6 && nu1 > 0 && nu2 > 0 && gr::coarse_cluster_ok(kind32);
    const int low = clus ? 5 : tail;  // the levels up to `low` run inside one launch
    timed(c, GR_PROF_COARSE, [&] {
        for (int l = top - 1; l >= (low ? low + 1 : 1); l--) {
            smooth_after_restrict(c->lev[l], l);
            down(l);
        }
        if (clus) {
            float *e[6], *r[6];
            const float *m[6], *iv[6];
            double h2[6], ih2[6];
            for (int l = 0; l < 6; l++) {
                e[l] = c->lev[l].e;
                r[l] = c->lev[l].r;
                m[l] = c->lev[l].m;
                iv[l] = c->lev[l].inv;
                h2[l] = c->lev[l].h2;
                ih2[l] = c->lev[l].ih2;
            }
            gr::coarse_cluster(kind32, e, r, m, iv, h2, ih2, nu1, nu2, c->st);
        } else if (tail) {
            float *e[4], *r[4];
            const float *m[4], *iv[4];
            double h2[4];
            for (int l = 0; l < 4; l++) {
                e[l] = c->lev[l].e;
                r[l] = c->lev[l].r;
                m[l] = c->lev[l].m;
                iv[l] = c->lev[l].inv;
                h2[l] = c->lev[l].h2;
            }
            gr::coarse_tail(kind32, e, r, m, iv, h2, nu1, nu2, c->st);
        } else {
            Level &Z = c->lev[0];
            gr::coarsest<float>(kind32, Z.e, Z.r, Z.m, Z.inv, Z.h2, Z.ih2, 0.0, c->st);
        }
        for (int l = low ? low + 1 : 1; l < top; l++) {
            up(l);
            smooth(c->lev[l], nu2);
        }
    });
    timed(c, cls(GR_PROF_PROLONG), [&] { up(top); });
    if (!uh) {
        smooth_fine(nu2);
        return;
    }
    if (!fused3(nu2, 0)) {
        timed(c, GR_PROF_SWEEP32, [&] {
            smooth(F, nu2 - 1);
            gr::sweep_colour<float>(kind32, F.n, F.e, F.r, F.m, F.inv, F.h2, F.ih2, 0.0, 0, c->st, dir_of(F));
        });
    }
    timed(c, GR_PROF_MIXED_UPDATE,
          [&] { gr::df_black_update(kind32, F.n, F.e, F.r, F.inv, F.h2, uh, ul, c->st, dir_of(F)); });
}

// Full multigrid correction cycle (nested iteration) on the FP32 correction
// equation with fine right-hand side lev[fine].r: the right-hand side is
// averaged down to 16^3, solved there by two V-cycles from zero (the coarse
// tail), and every finer level starts from the trilinear prolongation of the
// coarser level's solution and takes one V-cycle; the finest cycle may add
// its result to (uh, ul) as vcycle32 does.  Needs the coarse tail (fine
// level of at least 32^3).
void fmg32(gr_ctx *c, int kind32, int nu1, int nu2, float *uh, float *ul)
{
    const int top = c->nlev - 1;
    timed(c, GR_PROF_COARSE, [&] {
        for (int l = top; l > 3; l--) gr::restrict_avg(c->lev[l].n, c->lev[l].r, c->lev[l - 1].r, c->st);
        float *e[4], *r[4];
        const float *m[4], *iv[4];
        double h2[4];
        for (int l = 0; l < 4; l++) {
            e[l] = c->lev[l].e;
            r[l] = c->lev[l].r;
            m[l] = c->lev[l].m;
            iv[l] = c->lev[l].inv;
            h2[l] = c->lev[l].h2;
        }
        cudaMemsetAsync(c->lev[3].e, 0, sizeof(float) * 16 * 16 * 16, c->st);
        gr::coarse_tail(kind32, e, r, m, iv, h2, nu1, nu2, c->st);
        gr::coarse_tail(kind32, e, r, m, iv, h2, nu1, nu2, c->st);
    });
    for (int l = 4; l <= top; l++) {
        Level &A = c->lev[l];
        timed(c, l == top ? (int)GR_PROF_PROLONG : (int)GR_PROF_COARSE, [&] {
            cudaMemsetAsync(A.e, 0, sizeof(float) * (size_t)A.n * A.n * A.n, c->st);
            gr::prolong_add<float>(A.n, A.e, c->lev[l - 1].e, c->st);
        });
        if (l < top) vcycle32(c, kind32, nu1, nu2, START_GIVEN, nullptr, nullptr, l);
        else vcycle32(c, kind32, nu1, nu2, START_GIVEN, uh, ul);
    }
}

gr_status norm64(gr_ctx *c, int kind, double rho, double ref, double *eps_nat, double *r)
{
    Level &F = c->lev[c->nlev - 1];
    const int64_t N = (int64_t)F.n * F.n * F.n;
    int g = 0;
    timed(c, GR_PROF_NORM64, [&] {
        g = gr::resid_norm<double>(kind, F.n, F.u, F.f, F.c0, F.c1, F.ih2, rho, c->partials, eps_nat, c->st);
    });
    gr::finalize(c->partials, g, c->dscal, c->st);
    double q;
    gr_status st = read_scalars(c, &q, nullptr);
    *r = std::sqrt(q / N) / ref;
    return st;
}

// fine residual norm in double-float; with red != 0 also the first red
// relaxation of the next correction cycle (into lev[fine].e)
gr_status df_norm(gr_ctx *c, const EqInfo &in, double rho, bool red, double *r, const double *fshift = nullptr)
{
    Level &F = c->lev[c->nlev - 1];
    const int64_t N = (int64_t)F.n * F.n * F.n;
    int g = 0;
    timed(c, GR_PROF_MIXED_RESID, [&] {
        g = gr::df_resid(in.kind, F.n, c->dfu, c->dfu + N, c->dff, c->dff + N, c->dfa, c->dfa + N, c->dfb,
                         c->dfb + N, F.h2, rho, in.ref, F.r, F.m, F.inv, F.inv, red ? F.e : nullptr, c->partials,
                         c->st, next_dir(c), fshift);
    });
    gr::finalize(c->partials, g, c->dscal, c->st);
    double q;
    gr_status st = read_scalars(c, &q, nullptr);
    *r = std::sqrt(q / N);
    return st;
}

gr_status mixed_norm(gr_ctx *c, const EqInfo &in, double rho, double *r)
{
    Level &F = c->lev[c->nlev - 1];
    const int64_t N = (int64_t)F.n * F.n * F.n;
    int g = 0;
    timed(c, GR_PROF_MIXED_RESID, [&] {
        g = gr::mixed_resid(in.kind, F.n, F.u, F.f, F.c0, F.c1, F.ih2, F.h2, rho, F.r, F.m, F.inv, c->partials,
                            c->st);
    });
    gr::finalize(c->partials, g, c->dscal, c->st);
    double q;
    gr_status st = read_scalars(c, &q, nullptr);
    *r = std::sqrt(q / N) / in.ref;
    return st;
}

// ---------------------------------------------------------------- nested patches
// A chain of static patches (gr_patch): composite-grid FAS with flux matching,
// the multilevel reading of the paper's adaptive-grid solve (Sec. 3,
// Sec. 4.3).  Per equation: set-up on every patch, then per cycle the base's
// correction cycle, the patches' corrections and post-smoothing (coarse to
// fine), their pre-smoothing, residuals and injections into their parents
// (fine to coarse), and the base residual.

bool chain_valid(const gr_ctx *c, int np, const gr_patch *P)
{
    if (np < 0 || np > GR_MAX_PATCHES || (np > 0 && !P)) return false;
    int npar = c->n;
    for (int p = 0; p < np; p++) {
        const int n = P[p].n;
        if (n < 8 || n > 512 || (n & (n - 1))) return false;
        for (int d = 0; d < 3; d++) {
            const int o = P[p].origin[d];
            if (p == 0 ? (o < 0 || o >= c->n || n / 2 + 4 > c->n) : (o < 2 || o + n / 2 + 2 > npar)) return false;
        }
        npar = n;
    }
    return true;
}

void free_patches(gr_ctx *c)
{
    for (void *q : c->palloc) cudaFree(q);
    c->palloc.clear();
    c->pl.clear();
}

template <typename T>
gr_status palloc(gr_ctx *c, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(GR_ERR_NOMEM, "cudaMalloc(%zu bytes) for a patch", count * sizeof(T));
    }
    c->palloc.push_back(q);
    *p = (T *)q;
    return GR_OK;
}

// work arrays for the chain (kept while the chain's sizes stay the same)
gr_status ensure_patches(gr_ctx *c, int np, const gr_patch *P)
{
    if (!c->pdev) {
        gr_status st = dalloc(c, &c->pdev, 64);
        if (st != GR_OK) return st;
        if (cudaHostAlloc((void **)&c->phost, 64 * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&c->phost_dev, c->phost, 0) != cudaSuccess) {
            cudaGetLastError();
            if (c->phost) cudaFreeHost(c->phost);
            c->phost = c->phost_dev = nullptr;
            return fail(GR_ERR_NOMEM, "cudaHostAlloc (mapped patch scalars)");
        }
    }
    bool same = (int)c->pl.size() == np;
    for (int p = 0; same && p < np; p++) same = c->pl[p].n == P[p].n;
    if (!same) {
        cudaStreamSynchronize(c->st);
        free_patches(c);
        c->pl.resize(np);
        for (int p = 0; p < np; p++) {
            PatchLevel &L = c->pl[p];
            L.n = P[p].n;
            L.lgn = log2i(L.n);
            L.m = L.n + 4;
            L.nc = L.n / 2;
            L.w = L.nc + 4;
            const size_t M = (size_t)L.m * L.m * L.m, W = (size_t)L.w * L.w * L.w, Nc = (size_t)L.nc * L.nc * L.nc;
            gr_status st = GR_OK;
            double **arr[5] = {&L.u, &L.f, &L.c0, &L.c1, &L.eps};
            for (int q = 0; q < 5 && st == GR_OK; q++) st = palloc(c, arr[q], M);
            for (int q = 0; q < GR_NEQ && st == GR_OK; q++) st = palloc(c, &L.G[q], M);
            if (st == GR_OK) st = palloc(c, &L.win, W);
            if (st == GR_OK) st = palloc(c, &L.old, W);
            if (st == GR_OK) st = palloc(c, &L.Ru, Nc);
            if (st == GR_OK) st = palloc(c, &L.Re, Nc);
            if (st == GR_OK) st = palloc(c, &L.flux, 6 * (size_t)L.nc * L.nc);
            if (st == GR_OK) st = palloc(c, &L.A6, 6 * M);
            float **fa[8] = {&L.uh, &L.ul, &L.fh, &L.fl, &L.ah, &L.al, &L.bh, &L.bl};
            for (int q = 0; q < 8 && st == GR_OK; q++) st = palloc(c, fa[q], M);
            if (st == GR_OK) st = palloc(c, &L.d32, W);
            if (st != GR_OK) {
                free_patches(c);
                return st;
            }
            // ghost cells never written keep defined values
            for (int q = 0; q < 5; q++) cudaMemsetAsync(*arr[q], 0, M * sizeof(double), c->st);
            for (int q = 0; q < 8; q++) cudaMemsetAsync(*fa[q], 0, M * sizeof(float), c->st);
            for (int q = 0; q < GR_NEQ; q++) cudaMemsetAsync(L.G[q], 0, M * sizeof(double), c->st);
        }
    }
    for (int p = 0; p < np; p++) {
        PatchLevel &L = c->pl[p];
        for (int d = 0; d < 3; d++) L.o[d] = P[p].origin[d];
        L.h = c->h / (double)(2 << p);
    }
    return cuda_check("patch arrays");
}

gr::PBase base_view(gr_ctx *c, int fmt, double rho)
{
    Level &F = c->lev[c->nlev - 1];
    const int64_t N = (int64_t)F.n * F.n * F.n;
    gr::PBase B;
    B.lgn = log2i(F.n);
    B.h2 = F.h2;
    B.ih2 = F.ih2;
    B.rho = rho;
    if (fmt == gr::PB_SPLIT) {
        B.u = F.u, B.f = F.f, B.c0 = F.c0, B.c1 = F.c1;
    } else {
        B.uh = c->dfu, B.ul = c->dfu + N, B.fh = c->dff, B.fl = c->dff + N;
        B.ah = c->dfa, B.al = c->dfa + N, B.bh = c->dfb, B.bl = c->dfb + N;
    }
    return B;
}

gr::PPatch patch_view(gr_ctx *c, int p, const EqInfo &in, double rho)
{
    PatchLevel &L = c->pl[p];
    gr::PPatch V;
    V.lgn = L.lgn;
    V.m = L.m;
    V.u = L.u;
    V.f = L.f;
    V.c0 = in.kind != KPOISSON ? L.c0 : nullptr;
    V.c1 = in.kind != KPOISSON ? L.c1 : nullptr;  // psi: AA; Helmholtz: the inverse diagonal
    V.uh = L.uh, V.ul = L.ul, V.fh = L.fh, V.fl = L.fl;
    V.ah = L.ah, V.al = L.al, V.bh = L.bh, V.bl = L.bl;
    V.h2 = L.h * L.h;
    V.ih2 = 1.0 / V.h2;
    V.rho = rho;
    V.cpr = gr::df_from_double_host(2.0 * kPi * rho * V.h2);
    V.c5 = (float)(10.0 * kPi * rho * V.h2);
    if (p + 1 < (int)c->pl.size()) {
        for (int d = 0; d < 3; d++) V.co[d] = c->pl[p + 1].o[d];
        V.cnc = c->pl[p + 1].nc;
    }
    V.lam = in.poisson ? c->pdev : nullptr;
    return V;
}

// an FP64 ghosted array of patch p seen as a level (for windows of the fields)
gr::PPatch field_view(gr_ctx *c, int p, double *a)
{
    gr::PPatch V;
    V.lgn = c->pl[p].lgn;
    V.m = c->pl[p].m;
    V.u = a;
    return V;
}

// parent window of patch p: from the base (format fmt; PB_NAT reads the
// natural field nat), else from patch p - 1's working unknown (a == NULL) or
// its FP64 ghosted array a
void parent_window(gr_ctx *c, int p, int fmt, double rho, const double *nat, double *a, const EqInfo *in,
                   double *win, double *dold = nullptr, float *d32 = nullptr)
{
    PatchLevel &L = c->pl[p];
    if (p == 0) {
        gr::PBase B = base_view(c, fmt, rho);
        if (fmt == gr::PB_NAT) B.nat = nat;
        gr::patch_gather_base(fmt, B, L.o, L.w, win, c->st, dold, d32);
    } else if (a) {
        gr::patch_gather_patch(field_view(c, p - 1, a), false, L.o, L.w, win, c->st, dold, d32);
    } else {
        gr::patch_gather_patch(patch_view(c, p - 1, *in, rho), c->pdf, L.o, L.w, win, c->st, dold, d32);
    }
}

// Set-up of equation eq on every patch: ghosts of the solved fields it reads,
// right-hand side, coefficients and reference, the working unknown with
// ghosts from the parent's, and the Poisson bookkeeping.
gr_status patch_setup_eq(gr_ctx *c, int eq, const gr_opts *o, const EqInfo &in, const gr_sources *s,
                         const gr_fields *fl, double rho, double S_hat, int fmt)
{
    const int np = (int)c->pl.size();
    const int64_t N0 = (int64_t)c->n * c->n * c->n;
    const double K2 = 24.0 * kPi * rho, Kdot = 12.0 * kPi * rho + 4.0 * kPi * S_hat;
    bool need[GR_NEQ] = {};
    if (eq == GR_U) need[GR_VX] = need[GR_VY] = need[GR_VZ] = true;
    if (eq == GR_PSI || eq == GR_APSI || (eq >= GR_BX && eq <= GR_BZ))
        need[GR_VX] = need[GR_VY] = need[GR_VZ] = need[GR_U] = true;
    if (eq == GR_APSI || (eq >= GR_BX && eq <= GR_BZ)) need[GR_PSI] = true;
    if (eq >= GR_BX && eq <= GR_BZ) need[GR_APSI] = true;
    if (eq == GR_B_SCALAR) need[GR_BX] = need[GR_BY] = need[GR_BZ] = true;
    for (int q = 0; q < GR_NEQ; q++) {
        if (!need[q]) continue;
        for (int p = 0; p < np; p++) {
            PatchLevel &L = c->pl[p];
            parent_window(c, p, gr::PB_NAT, rho, field_ptr(fl, q), p ? c->pl[p - 1].G[q] : nullptr, &in, L.win);
            gr::patch_interp(field_view(c, p, L.G[q]), false, L.win, nullptr, nullptr, c->st);
        }
    }
    double smean = 0.0;
    if (eq <= GR_VZ) {  // the base mean of s_i (the homogeneous background)
        dsum(c, N0, s->s[eq]);
        double a, q2;
        gr_status st = read_scalars(c, &a, &q2);
        if (st != GR_OK) return st;
        smean = a / N0;
    }
    for (int p = 0; p < np; p++) {
        PatchLevel &L = c->pl[p];
        const gr_sources &ps = o->patch[p].src;
        gr::PSetSrc S = {{ps.s0, ps.s[0], ps.s[1], ps.s[2], ps.sigma}};
        gr::PSetFld G;
        for (int q = 0; q < GR_NEQ; q++) G.g[q] = L.G[q];
        if (eq == GR_PSI) gr::patch_aij(L.n, 1.0 / L.h, G, L.A6, c->st);  // V and U are final from here on
        const int g = gr::patch_setup(eq, L.n, 1.0 / L.h, S, G, L.A6, smean, K2, Kdot, L.f, L.c0, L.c1, c->partials,
                                      c->st);
        if (c->pdf) gr::patch_coef_df(in.kind, patch_view(c, p, in, rho), c->st);
        gr::finalize(c->partials, g, c->pdev + 16 + 2 * p, c->st);
    }
    gr::scalars_out(c->pdev + 16, c->phost_dev + 16, 2 * np, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check("patch set-up");
    for (int p = 0; p < np; p++) {
        PatchLevel &L = c->pl[p];
        L.ref = (eq == GR_PSI ? 2.0 * kPi : 1.0) * std::sqrt(c->phost[16 + 2 * p] / ((double)L.n * L.n * L.n));
        if (!(L.ref >= 1e-300)) L.ref = 1.0;
        gr::patch_u_load(patch_view(c, p, in, rho), c->pdf, field_ptr(&o->patch[p].fld, eq), in.dev ? -1.0 : 0.0,
                         c->st);
    }
    for (int p = 0; p < np; p++) {
        PatchLevel &L = c->pl[p];
        parent_window(c, p, fmt, rho, nullptr, nullptr, &in, L.win);
        gr::patch_interp(patch_view(c, p, in, rho), c->pdf, L.win, nullptr, nullptr, c->st);
        cudaMemsetAsync(L.flux, 0, 6 * (size_t)L.nc * L.nc * sizeof(double), c->st);
    }
    cudaMemsetAsync(c->pdev, 0, sizeof(double), c->st);  // lambda = 0
    if (in.poisson) {
        const gr::PBase B = base_view(c, fmt, rho);
        const int g = gr::patch_sum_f_base(fmt, B, c->pl[0].o, c->pl[0].nc, c->partials, c->st);
        gr::finalize(c->partials, g, c->pdev + 1, c->st);  // the original right-hand side over the covered cells
    }
    return cuda_check("patch set-up");
}

// patches fine to coarse: nu sweeps, residual (norm into pdev[32 + 2p]),
// restriction, injection into the parent with flux matching; for Poisson the
// solvability constant after the base injection.  Queues the norms' store
// to the mapped phost (the caller's next synchronisation covers it).
void patch_down(gr_ctx *c, const EqInfo &in, int fmt, int nu, double rho)
{
    const int np = (int)c->pl.size();
    Level &F = c->lev[c->nlev - 1];
    const int64_t N0 = (int64_t)F.n * F.n * F.n;
    for (int p = np - 1; p >= 0; p--) {
        PatchLevel &L = c->pl[p];
        const gr::PPatch V = patch_view(c, p, in, rho);
        for (int sw = 0; sw < nu; sw++) {
            gr::patch_gs(in.kind, V, c->pdf, 0, c->st);
            gr::patch_gs(in.kind, V, c->pdf, 1, c->st);
        }
        int g = gr::patch_resid(in.kind, V, c->pdf, L.eps, c->partials, c->st);
        gr::finalize(c->partials, g, c->pdev + 32 + 2 * p, c->st);
        gr::patch_restrict(V, c->pdf, L.eps, L.Ru, L.Re, c->st);
        if (p == 0) {
            const gr::PBase B = base_view(c, fmt, rho);
            gr::patch_inject_u_base(fmt, B, L.o, L.nc, L.Ru, c->st);
            gr::patch_gather_base(fmt, B, L.o, L.w, L.old, c->st);
            g = gr::patch_inject_f_base(fmt, in.kind, B, L.o, L.nc, L.Re,
                                        (fmt == gr::PB_DF && in.poisson) ? c->pdev : nullptr, c->partials, c->st);
            gr::finalize(c->partials, g, c->pdev + 3, c->st);
            gr::patch_reflux(fmt, B, gr::PPatch{}, V, c->pdf, L.o, c->h, L.flux, c->st);
            if (in.poisson) {
                gr::patch_lambda(c->pdev + 1, L.flux, 6 * L.nc * L.nc, (double)N0, (double)L.nc * L.nc * L.nc,
                                 c->pdev, c->st);
                if (fmt == gr::PB_SPLIT) gr::sub_scalar(N0, F.f, c->pdev + 5, c->st);
            }
        } else {
            PatchLevel &Q = c->pl[p - 1];
            const gr::PPatch par = patch_view(c, p - 1, in, rho);
            gr::patch_inject_u_patch(par, c->pdf, L.o, L.nc, L.Ru, c->st);
            gr::patch_gather_patch(par, c->pdf, L.o, L.w, L.old, c->st);
            gr::patch_inject_f_patch(in.kind, par, c->pdf, L.o, L.nc, L.Re, c->st);
            gr::patch_reflux(-1, gr::PBase{}, par, V, c->pdf, L.o, Q.h, L.flux, c->st);
        }
    }
    gr::scalars_out(c->pdev + 32, c->phost_dev + 32, 2 * np, c->st);
}

// patches coarse to fine: the parent's correction P(u_new - u_old), fresh ghosts, nu sweeps
void patch_up(gr_ctx *c, const EqInfo &in, int fmt, int nu, double rho)
{
    const int np = (int)c->pl.size();
    for (int p = 0; p < np; p++) {
        PatchLevel &L = c->pl[p];
        // L.old becomes the parent's change since the injection
        parent_window(c, p, fmt, rho, nullptr, nullptr, &in, L.win, L.old, c->pdf ? L.d32 : nullptr);
        const gr::PPatch V = patch_view(c, p, in, rho);
        gr::patch_interp(V, c->pdf, L.win, L.old, L.d32, c->st);
        for (int sw = 0; sw < nu; sw++) {
            gr::patch_gs(in.kind, V, c->pdf, 0, c->st);
            gr::patch_gs(in.kind, V, c->pdf, 1, c->st);
        }
    }
}

// relative residuals of the patches from the last patch_down (after a synchronisation)
void patch_norms(const gr_ctx *c, double *r)
{
    for (size_t p = 0; p < c->pl.size(); p++) {
        const PatchLevel &L = c->pl[p];
        r[p] = std::sqrt(c->phost[32 + 2 * p] / ((double)L.n * L.n * L.n)) / L.ref;
    }
}

long long patch_cells(const gr_ctx *c, int nu)
{
    long long s = 0;
    for (const PatchLevel &L : c->pl) s += (long long)nu * L.n * L.n * L.n;
    return s;
}

// Solve (or cycle) one equation; writes the field back.  tol < 0 with
// max_cycles = 1 performs exactly one cycle and reports OK.
gr_status solve_eq(gr_ctx *c, int eq, const gr_sources *s, gr_fields *fl, const gr_opts *o, double rho,
                   double S_hat, double tol, int max_cycles, int *cycles, double *res0, double *res,
                   long long *cells, int *rejected = nullptr, double *res_level = nullptr)
{
    EqInfo in;
    gr_status st = GR_OK;
    const bool dfm = o->prec == GR_PREC_MIXED_DF;
    timed(c, GR_PROF_SETUP, [&] {
        st = dfm ? setup_eq_df(c, eq, s, fl, rho, S_hat, &in) : setup_eq(c, eq, s, fl, rho, S_hat, &in);
    });
    if (st != GR_OK) return st;
    Level &F = c->lev[c->nlev - 1];
    const int64_t N = (int64_t)F.n * F.n * F.n;
    // the double-float residual also makes the first red pass of the next
    // cycle, and the last black pass adds the correction to u
    const bool red = dfm && o->nu1 > 0;
    const bool fuse_update = dfm && o->nu2 > 0 && F.n >= 8;
    // full multigrid start: the first correction of the equation (mixed modes, coarse tail present)
    const bool fmg = o->fmg != 0 && (o->prec == GR_PREC_MIXED || dfm) && c->nlev - 1 > 3 && c->tail_on;
    // residual of the plain guess (unknown 0: psi = alpha psi = 1, vectors 0),
    // the bar a given guess must beat after its first cycle
    double r_plain = NAN;
    const bool patches = o->npatch > 0;
    const int pfmt = dfm ? gr::PB_DF : gr::PB_SPLIT;
    const bool check = o->check_guess != 0 && rejected != nullptr && !patches;
    if (check) {
        *rejected = 0;
        if (in.kind == KPOISSON) {
            // u = 0 leaves eps = -f, and ref is RMS(f): the plain guess's relative residual is 1
            r_plain = 1.0;
        } else if (dfm) {
            // the pair array (2N floats) fits the FP64 scratch level array
            cudaMemcpyAsync(F.ur, c->dfu, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
            cudaMemsetAsync(c->dfu, 0, N * sizeof(double), c->st);
            st = df_norm(c, in, rho, false, &r_plain);
            if (st != GR_OK) return st;
            cudaMemcpyAsync(c->dfu, F.ur, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
        } else {
            cudaMemcpyAsync(F.ur, F.u, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
            cudaMemsetAsync(F.u, 0, N * sizeof(double), c->st);
            st = norm64(c, in.kind, rho, in.ref, nullptr, &r_plain);
            if (st != GR_OK) return st;
            cudaMemcpyAsync(F.u, F.ur, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
        }
    }
    const bool mixed = o->prec == GR_PREC_MIXED || dfm;
    const long long per_cycle =
        vcycle_cells(c, o->nu1, o->nu2, -1, (!mixed && in.kind == KPSI) ? 8LL * kCoarsestSweeps : 8LL);
    if (mixed) {
        if (in.kind == KHELM) {
            if (!dfm) {  // the double-float set-up wrote m and its inverse diagonal
                gr::to_float(N, F.c0, F.m, c->st);
                gr::helm_invdiag<float>(F.n, F.m, F.inv, F.h2, c->st);
            }
            restrict_coefs32(c);
        }
    } else {
        restrict_coefs64(c, in.kind);
    }
    double rlev[GR_MAX_PATCHES + 1] = {};
    // the base residual and, with patches, the largest of all levels' (rlev: each level's)
    auto fine_norm = [&](double *r) {
        gr_status q;
        if (dfm) q = df_norm(c, in, rho, red, r, (patches && in.poisson) ? c->pdev : nullptr);
        else if (mixed) q = mixed_norm(c, in, rho, r);
        else q = norm64(c, in.kind, rho, in.ref, nullptr, r);
        rlev[0] = *r;
        if (q == GR_OK && patches) {
            patch_norms(c, rlev + 1);
            for (int p = 1; p <= o->npatch; p++) *r = std::isfinite(rlev[p]) && rlev[p] <= *r ? *r : rlev[p];
        }
        return q;
    };
    if (patches) {
        timed(c, GR_PROF_PATCH, [&] { st = patch_setup_eq(c, eq, o, in, s, fl, rho, S_hat, pfmt); });
        if (st != GR_OK) return st;
        timed(c, GR_PROF_PATCH, [&] { patch_down(c, in, pfmt, 0, rho); });
    }
    auto use_plain_guess = [&]() {
        cudaMemsetAsync(F.u, 0, N * sizeof(double), c->st);
        if (dfm) cudaMemsetAsync(c->dfu, 0, 2 * N * sizeof(float), c->st);
        *rejected = 1;
    };
    double r = 0;
    st = fine_norm(&r);
    if (st != GR_OK) return st;
    if (check && !std::isfinite(r)) {
        use_plain_guess();
        st = fine_norm(&r);
        if (st != GR_OK) return st;
    }
    if (res0) *res0 = r;
    int cyc = 0;
    if (!std::isfinite(r)) st = fail(GR_ERR_NONFINITE, "equation %d: initial residual is not finite", eq);
    while (st == GR_OK && r > tol && cyc < max_cycles) {
        if (mixed) {
            if (in.kind == KPSI) restrict_coefs32(c);
            const bool full = fmg && cyc == 0;
            const Start start = red ? START_RED_DONE : START_ZERO;
            if (fuse_update) {
                if (full) fmg32(c, in.kind32, o->nu1, o->nu2, c->dfu, c->dfu + N);
                else vcycle32(c, in.kind32, o->nu1, o->nu2, start, c->dfu, c->dfu + N);
            } else {
                if (full) fmg32(c, in.kind32, o->nu1, o->nu2, nullptr, nullptr);
                else vcycle32(c, in.kind32, o->nu1, o->nu2, start);
                timed(c, GR_PROF_MIXED_UPDATE, [&] {
                    if (dfm) gr::df_update(F.n, c->dfu, c->dfu + N, F.e, c->st);
                    else gr::mixed_update(F.n, F.u, F.e, c->st);
                });
            }
            if (cells && full) *cells += fmg_cells(c, o->nu1, o->nu2) - per_cycle;
        } else {
            vcycle64(c, in.kind, rho, o->nu1, o->nu2);
        }
        if (patches) {
            timed(c, GR_PROF_PATCH, [&] {
                patch_up(c, in, pfmt, o->nu2, rho);
                patch_down(c, in, pfmt, o->nu1, rho);
            });
            if (cells) *cells += patch_cells(c, o->nu1 + o->nu2);
        }
        st = fine_norm(&r);
        cyc++;
        if (cells) *cells += per_cycle;
        if (st == GR_OK && check && cyc == 1 && !*rejected && !(r <= r_plain)) {
            use_plain_guess();
            st = fine_norm(&r);
        }
        if (st == GR_OK && !std::isfinite(r)) st = fail(GR_ERR_NONFINITE, "equation %d: residual not finite", eq);
    }
    if (cycles) *cycles = cyc;
    if (res) *res = r;
    // write back: +1 for the deviation unknowns, zero mean for Poisson-type
    // (the FP64 norm kernels leave the sum of u in dscal[1])
    if (dfm) {
        if (in.poisson) {
            const int g = gr::dfs_pair_sum(N, c->dfu, c->dfu + N, c->partials, c->st);
            gr::finalize(c->partials, g, c->dscal, c->st);
        }
        gr::dfs_store(F.n, c->dfu, c->dfu + N, in.poisson ? c->dscal : nullptr, in.dev, field_ptr(fl, eq), c->st);
    } else {
        const double *usum = in.poisson ? c->dscal + 1 : nullptr;
        gr::from_split(F.n, F.u, field_ptr(fl, eq), in.dev ? 1.0 : 0.0, usum, 1.0 / N, c->st);
    }
    if (patches) {  // the same mean off every patch; the patch's copy of the field for later set-ups
        const double *usum = in.poisson ? (dfm ? c->dscal : c->dscal + 1) : nullptr;
        for (int p = 0; p < o->npatch; p++)
            gr::patch_u_store(patch_view(c, p, in, rho), c->pdf, field_ptr(&o->patch[p].fld, eq), c->pl[p].G[eq],
                              in.dev ? 1.0 : 0.0, usum, 1.0 / N, c->st);
        if (res_level)
            for (int p = 0; p <= o->npatch; p++) res_level[p] = rlev[p];
    }
    gr_status cs = cuda_check("write back");
    if (cs != GR_OK) return cs;
    if (st == GR_OK && tol >= 0 && r > tol)
        st = fail(GR_ERR_NOCONV, "equation %d: %d cycles, relative residual %.3e > tol %.3e", eq, cyc, r, tol);
    return st;
}

gr_status resolve_bg(gr_ctx *c, const gr_opts *o, double *rho, double *S_hat)
{
    *rho = (o->rho_hat > 0) ? o->rho_hat : c->rho_dep;
    *S_hat = std::isnan(o->S_hat) ? 0.0 : o->S_hat;
    if (!(*rho > 0)) return fail(GR_ERR_ARG, "rho_hat not given and no gr_deposit on this context");
    return GR_OK;
}

// true for memory the host addresses directly (pinned or pageable), false
// for device (or managed) memory
bool host_memory(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// the copy stream and events of host-buffer I/O, created at first use
gr_status ensure_copy_stream(gr_ctx *c)
{
    if (c->cs) return GR_OK;
    if (cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cs = nullptr;
        return fail(GR_ERR_CUDA, "cudaStreamCreate");
    }
    bool ok = cudaEventCreateWithFlags(&c->xfer, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; b++)
        ok = cudaEventCreateWithFlags(&c->ready[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->used[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(GR_ERR_CUDA, "cudaEventCreate");
    }
    return GR_OK;
}

// Deposit from host arrays: chunks of particles go through two staging
// buffers; chunk i's six copies (x and u, three components each) run on the
// copy stream while chunk i-1 deposits on the context's stream.
gr_status deposit_from_host(gr_ctx *c, int64_t np, const double *x, const double *u, double mass,
                            const gr_sources *out)
{
    gr_status st = ensure_copy_stream(c);
    if (st != GR_OK) return st;
    const int64_t chunk = np < c->host_chunk ? np : c->host_chunk;
    if (c->stage_cap < chunk) {
        for (int b = 0; b < 2; b++) {
            st = dalloc(c, &c->stage[b], (size_t)6 * chunk);  // kept until gr_destroy
            if (st != GR_OK) return st;
        }
        c->stage_cap = chunk;
    }
    const size_t bytes = (size_t)c->n * c->n * c->n * sizeof(double);
    double *f[5] = {out->s0, out->s[0], out->s[1], out->s[2], out->sigma};
    for (int k = 0; k < 5; k++) cudaMemsetAsync(f[k], 0, bytes, c->st);
    // the staging buffers may still be read by the previous call's last chunks
    for (int b = 0; b < 2; b++) cudaEventRecord(c->used[b], c->st);
    int b = 0;
    for (int64_t p0 = 0; p0 < np; p0 += chunk, b ^= 1) {
        const int64_t m = np - p0 < chunk ? np - p0 : chunk;
        double *xs = c->stage[b], *us = c->stage[b] + 3 * m;
        cudaStreamWaitEvent(c->cs, c->used[b], 0);
        for (int d = 0; d < 3; d++) {
            cudaMemcpyAsync(xs + d * m, x + d * np + p0, m * sizeof(double), cudaMemcpyDefault, c->cs);
            cudaMemcpyAsync(us + d * m, u + d * np + p0, m * sizeof(double), cudaMemcpyDefault, c->cs);
        }
        cudaEventRecord(c->ready[b], c->cs);
        cudaStreamWaitEvent(c->st, c->ready[b], 0);
        gr::deposit_add(c->n, c->L, m, xs, us, mass, out->s0, out->s[0], out->s[1], out->s[2], out->sigma, c->st);
        cudaEventRecord(c->used[b], c->st);
    }
    return GR_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

void gr_default_opts(gr_opts *o)
{
    if (!o) return;
    o->tol = 1e-10;
    o->max_cycles = 50;
    o->nu1 = 2;
    o->nu2 = 2;
    o->prec = GR_PREC_FP64;
    o->rho_hat = 0.0;
    o->S_hat = 0.0;
    o->verbose = 0;
    o->profile = 0;
    o->check_guess = 0;
    o->fmg = 0;
    o->host_out = nullptr;
    o->npatch = 0;
    o->patch = nullptr;
}

const char *gr_last_error(void) { return g_err.c_str(); }

long long gr_kernel_launches(void) { return gr::g_launches.load(); }

void gr_destroy(gr_ctx *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    for (void *p : c->allocs) cudaFree(p);
    free_patches(c);
    if (c->hscal) cudaFreeHost(c->hscal);
    if (c->phost) cudaFreeHost(c->phost);
    if (c->cs) cudaStreamSynchronize(c->cs);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (int b = 0; b < 2; b++) {
        if (c->ready[b]) cudaEventDestroy(c->ready[b]);
        if (c->used[b]) cudaEventDestroy(c->used[b]);
    }
    if (c->xfer) cudaEventDestroy(c->xfer);
    if (c->cs) cudaStreamDestroy(c->cs);
    for (auto &p : c->pending) {
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

gr_status gr_create(int n, double L, void *stream, gr_ctx **out)
{
    g_err.clear();
    if (!out) return fail(GR_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 4 || n > 1024 || (n & (n - 1))) return fail(GR_ERR_ARG, "n = %d: must be a power of two in [4, 1024]", n);
    if (!(L > 0) || !std::isfinite(L)) return fail(GR_ERR_ARG, "L must be finite and > 0");
    gr_ctx *c = new (std::nothrow) gr_ctx();
    if (!c) return fail(GR_ERR_NOMEM, "host allocation");
    c->n = n;
    c->L = L;
    if (const char *env = getenv("GR_COARSE_TAIL")) c->tail_on = env[0] != '0';
    if (const char *env = getenv("GR_COARSE_CLUSTER")) c->cluster_on = env[0] == '1';
    if (const char *env = getenv("GR_SMOOTH3")) {
        if (env[0] == '1') {
            c->s3_min = 512;
            if (const char *m = getenv("GR_SMOOTH3_MIN")) c->s3_min = atoi(m);
        }
    }
    if (const char *env = getenv("GR_HOST_CHUNK")) {
        const long long v = atoll(env);
        if (v > 0) c->host_chunk = v;
    }
    c->h = L / n;
    c->st = (cudaStream_t)stream;
    c->nlev = log2i(n);
    c->lev.resize(c->nlev);
    gr_status st = GR_OK;
    for (int l = 0; l < c->nlev && st == GR_OK; l++) {
        Level &A = c->lev[l];
        A.n = 2 << l;
        A.h = L / A.n;
        A.h2 = A.h * A.h;
        A.ih2 = 1.0 / A.h2;
        const size_t N = (size_t)A.n * A.n * A.n;
        if (st == GR_OK) st = dalloc(c, &A.u, N);
        if (st == GR_OK) st = dalloc(c, &A.f, N);
        if (st == GR_OK) st = dalloc(c, &A.c0, N);
        if (st == GR_OK) st = dalloc(c, &A.c1, N);
        if (st == GR_OK) st = dalloc(c, &A.ur, N);
        if (st == GR_OK) st = dalloc(c, &A.e, N);
        if (st == GR_OK) st = dalloc(c, &A.r, N);
        if (st == GR_OK) st = dalloc(c, &A.m, N);
        if (st == GR_OK) st = dalloc(c, &A.inv, N);
    }
    const size_t N = (size_t)n * n * n;
    if (st == GR_OK && n >= c->s3_min && gr::smooth3_fits(KPOISSON, n)) {
        Level &F = c->lev[c->nlev - 1];
        st = dalloc(c, &F.e2, N);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c->s3_rt = gr::smooth3_row_tiles(n, sms > 0 ? sms : 1);
        // GR_SMOOTH3_RT: another row-tile count (tiles of at most 14 rows)
        if (const char *env = getenv("GR_SMOOTH3_RT")) {
            const int rt = atoi(env);
            if (rt >= (n + 13) / 14 && rt <= n) c->s3_rt = rt;
        }
    }
    if (st == GR_OK) st = dalloc(c, &c->A6, 6 * N);
    if (st == GR_OK) st = dalloc(c, &c->dfu, 2 * N);
    if (st == GR_OK) st = dalloc(c, &c->dff, 2 * N);
    if (st == GR_OK) st = dalloc(c, &c->dfa, 2 * N);
    if (st == GR_OK) st = dalloc(c, &c->dfb, 2 * N);
    if (st == GR_OK) st = dalloc(c, &c->AA, N);
    if (st == GR_OK) st = dalloc(c, &c->tmp, N);
    if (st == GR_OK) st = dalloc(c, &c->partials, 2 * kMaxRedBlocks);
    if (st == GR_OK) st = dalloc(c, &c->dscal, 16);
    if (st == GR_OK && (cudaHostAlloc((void **)&c->hscal, 16 * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
                        cudaHostGetDevicePointer((void **)&c->hscal_dev, c->hscal, 0) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(GR_ERR_NOMEM, "cudaHostAlloc (mapped scalars)");
    }
    if (st == GR_OK && (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(GR_ERR_CUDA, "cudaEventCreate");
    }
    if (st != GR_OK) {
        gr_destroy(c);
        return st;
    }
    *out = c;
    return GR_OK;
}

gr_status gr_deposit(gr_ctx *c, int64_t np, const double *x, const double *u, double mass, gr_sources *out)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if (np < 0) return fail(GR_ERR_ARG, "np < 0");
    if (np > 0 && (!x || !u)) return fail(GR_ERR_ARG, "x or u is NULL");
    if (!src_ok(out)) return fail(GR_ERR_ARG, "a source array is NULL or not 16-byte aligned");
    if (!(mass >= 0) || !std::isfinite(mass)) return fail(GR_ERR_ARG, "mass must be finite and >= 0");
    const bool hx = np > 0 && host_memory(x), hu = np > 0 && host_memory(u);
    if (hx != hu) return fail(GR_ERR_ARG, "x and u must both be device or both host memory");
    if (hx) {
        gr_status st = deposit_from_host(c, np, x, u, mass, out);
        if (st != GR_OK) return st;
    } else {
        gr::deposit(c->n, c->L, np, x, u, mass, out->s0, out->s[0], out->s[1], out->s[2], out->sigma, c->st);
    }
    c->rho_dep = mass * (double)np / (c->L * c->L * c->L);
    return cuda_check("gr_deposit");
}

gr_status gr_solve_constraints(gr_ctx *c, const gr_sources *s, gr_fields *fl, const gr_opts *o, gr_report *rep)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if (!src_ok(s) || !fld_ok(fl)) return fail(GR_ERR_ARG, "a source or field array is NULL or not 16-byte aligned");
    if (!valid_opts(o)) return fail(GR_ERR_ARG, "invalid gr_opts");
    if (o->npatch > 0) {
        if (!chain_valid(c, o->npatch, o->patch)) return fail(GR_ERR_ARG, "invalid patch chain");
        for (int p = 0; p < o->npatch; p++)
            if (!src_ok(&o->patch[p].src) || !fld_ok(&o->patch[p].fld))
                return fail(GR_ERR_ARG, "patch %d: a source or field array is NULL or not 16-byte aligned", p);
    }
    double rho, S_hat;
    gr_status st = resolve_bg(c, o, &rho, &S_hat);
    if (st != GR_OK) return st;
    if (o->npatch > 0) {
        st = ensure_patches(c, o->npatch, o->patch);
        if (st != GR_OK) return st;
        c->pdf = o->prec != GR_PREC_FP64;
        for (int p = 0; p < o->npatch; p++)  // every field's guess, for the set-ups of the equations before its own
            for (int q = 0; q < GR_NEQ; q++)
                gr::patch_to_ghosted(c->pl[p].n, field_ptr(&o->patch[p].fld, q), c->pl[p].G[q], 0.0, c->st);
    } else if (!c->pl.empty()) {
        free_patches(c);
    }
    gr_report R;
    memset(&R, 0, sizeof(R));
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = gr::g_launches.load();
    c->a_fmt = 0;
    c->w_fmt = 0;
    c->prof_on = o->profile != 0;
    memset(c->prof_launches, 0, sizeof(c->prof_launches));
    memset(c->prof_ms, 0, sizeof(c->prof_ms));
    gr_status worst = GR_OK;
    std::string first_err;
    if (o->host_out) {
        st = ensure_copy_stream(c);
        if (st != GR_OK) return st;
    }
    const size_t field_bytes = (size_t)c->n * c->n * c->n * sizeof(double);
    for (int eq = 0; eq < GR_NEQ; eq++) {
        if (eq == GR_PSI) c->a_fmt = 0;  // V and U are final now
        cudaEventRecord(c->ev0, c->st);
        st = solve_eq(c, eq, s, fl, o, rho, S_hat, o->tol, o->max_cycles, &R.cycles[eq], &R.res0[eq], &R.res[eq],
                      &R.cell_updates, &R.guess_rejected[eq], R.res_level[eq]);
        if (o->host_out && (st == GR_OK || st == GR_ERR_NOCONV)) {
            // this field is final: copy it out while the next equations solve
            cudaEventRecord(c->xfer, c->st);
            cudaStreamWaitEvent(c->cs, c->xfer, 0);
            cudaMemcpyAsync(field_ptr(o->host_out, eq), field_ptr(fl, eq), field_bytes, cudaMemcpyDefault, c->cs);
        }
        cudaEventRecord(c->ev1, c->st);
        cudaEventSynchronize(c->ev1);
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        R.eq_seconds[eq] = ms * 1e-3;
        R.eq_status[eq] = st;
        if (o->verbose)
            fprintf(stderr, "[gr] eq %d: %d cycles, res %.3e -> %.3e, %.3f ms, status %d\n", eq, R.cycles[eq],
                    R.res0[eq], R.res[eq], ms, (int)st);
        if (st != GR_OK && worst == GR_OK) {
            worst = st;
            first_err = g_err;
        }
        if (st != GR_OK && st != GR_ERR_NOCONV) break;
    }
    if (o->host_out) {  // the call's stream waits for the last copy
        cudaEventRecord(c->xfer, c->cs);
        cudaStreamWaitEvent(c->st, c->xfer, 0);
    }
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (c->prof_on) {
        cudaStreamSynchronize(c->st);
        prof_collect(c);
        for (int k = 0; k < GR_NPROF; k++) {
            R.prof_launches[k] = c->prof_launches[k];
            R.prof_ms[k] = c->prof_ms[k];
        }
        c->prof_on = false;
    }
    R.kernel_launches = gr::g_launches.load() - launches0;
    if (rep) *rep = R;
    if (worst != GR_OK) g_err = first_err;
    return worst;
}

gr_status gr_vcycle(gr_ctx *c, gr_eq eq, const gr_sources *s, gr_fields *fl, const gr_opts *o, double *res_after)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if ((int)eq < 0 || (int)eq >= GR_NEQ) return fail(GR_ERR_ARG, "bad equation %d", (int)eq);
    if (!src_ok(s) || !fld_ok(fl)) return fail(GR_ERR_ARG, "a source or field array is NULL or not 16-byte aligned");
    if (!valid_opts(o)) return fail(GR_ERR_ARG, "invalid gr_opts");
    double rho, S_hat;
    gr_status st = resolve_bg(c, o, &rho, &S_hat);
    if (st != GR_OK) return st;
    c->a_fmt = 0;
    c->w_fmt = 0;
    double r = NAN;
    gr_opts base_only = *o;  // one cycle of the periodic base: patches are gr_solve_constraints's
    base_only.npatch = 0;
    st = solve_eq(c, eq, s, fl, &base_only, rho, S_hat, -1.0, 1, nullptr, nullptr, &r, nullptr);
    if (res_after) *res_after = r;
    return st;
}

gr_status gr_residual(gr_ctx *c, gr_eq eq, const gr_sources *s, const gr_fields *fl, const gr_opts *o,
                      double *res_field, double *rel_norm)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if ((int)eq < 0 || (int)eq >= GR_NEQ) return fail(GR_ERR_ARG, "bad equation %d", (int)eq);
    if (!src_ok(s) || !fld_ok(fl)) return fail(GR_ERR_ARG, "a source or field array is NULL or not 16-byte aligned");
    if (!valid_opts(o)) return fail(GR_ERR_ARG, "invalid gr_opts");
    double rho, S_hat;
    gr_status st = resolve_bg(c, o, &rho, &S_hat);
    if (st != GR_OK) return st;
    c->a_fmt = 0;
    c->w_fmt = 0;
    EqInfo in;
    st = setup_eq(c, eq, s, fl, rho, S_hat, &in);
    if (st != GR_OK) return st;
    double r;
    st = norm64(c, in.kind, rho, in.ref, res_field, &r);
    if (rel_norm) *rel_norm = r;
    return st;
}

gr_status gr_deposit_patches(gr_ctx *c, int npatch, const gr_patch *patch, int64_t np, const double *x,
                             const double *u, double mass)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if (npatch < 1 || !chain_valid(c, npatch, patch)) return fail(GR_ERR_ARG, "invalid patch chain");
    if (np < 0 || (np > 0 && (!x || !u))) return fail(GR_ERR_ARG, "bad particle arrays");
    if (np > 0 && (host_memory(x) || host_memory(u)))
        return fail(GR_ERR_ARG, "gr_deposit_patches takes device particle arrays");
    for (int p = 0; p < npatch; p++)
        if (!src_ok(&patch[p].src)) return fail(GR_ERR_ARG, "patch %d: a source array is NULL or not 16-byte aligned", p);
    // one pass over the particles lists those near the first patch (every
    // later patch lies inside it); each patch then deposits from that list
    if (np > 0 && np <= INT32_MAX && c->plist_cap < np) {
        if (c->plist) {
            cudaFree(c->plist);
            c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), (void *)c->plist), c->allocs.end());
            c->plist = nullptr;
            c->plist_cap = 0;
        }
        gr_status st = dalloc(c, &c->plist, (size_t)np);
        if (st != GR_OK) return st;
        c->plist_cap = np;
    }
    if (!c->pcount) {
        gr_status st = dalloc(c, &c->pcount, 1);
        if (st != GR_OK) return st;
    }
    const bool listed = np > 0 && np <= INT32_MAX;
    if (listed) {
        int lo[3];
        for (int d = 0; d < 3; d++) lo[d] = patch[0].origin[d] - 1;
        gr::patch_select(np, x, c->L, c->n, lo, patch[0].n / 2 + 2, c->plist, c->pcount, c->st);
    }
    int O[3] = {0, 0, 0};
    for (int p = 0; p < npatch; p++) {
        const int N = c->n << (p + 1), n = patch[p].n;
        for (int d = 0; d < 3; d++) O[d] = (2 * (O[d] + patch[p].origin[d])) & (N - 1);
        const gr_sources &ps = patch[p].src;
        double *f[5] = {ps.s0, ps.s[0], ps.s[1], ps.s[2], ps.sigma};
        for (int k = 0; k < 5; k++) cudaMemsetAsync(f[k], 0, (size_t)n * n * n * sizeof(double), c->st);
        const gr::PSetSrc out{{f[0], f[1], f[2], f[3], f[4]}};
        if (listed) gr::patch_deposit_list(np, c->plist, c->pcount, x, u, mass, c->L, N, O, n, out, c->st);
        else gr::patch_deposit(np, x, u, mass, c->L, N, O, n, out, c->st);
    }
    return cuda_check("gr_deposit_patches");
}

gr_status gr_particle_update(gr_ctx *c, int64_t np, double *x, double *u, const gr_fields *fl, double dt, int flags)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if (np < 0 || (np > 0 && (!x || !u))) return fail(GR_ERR_ARG, "bad particle arrays");
    if (!fl || !fl->psi || !fl->apsi || !fl->B[0] || !fl->B[1] || !fl->B[2] || !fl->b)
        return fail(GR_ERR_ARG, "a field array is NULL");
    if (!std::isfinite(dt)) return fail(GR_ERR_ARG, "dt must be finite");
    if (flags & ~(GR_KICK_SYNC | GR_KICK_OPEN | GR_DRIFT)) return fail(GR_ERR_ARG, "flags = %d", flags);
    if (np > 0 && (host_memory(x) || host_memory(u)))
        return fail(GR_ERR_ARG, "gr_particle_update takes device particle arrays");
    if (np == 0 || flags == 0) return GR_OK;
    const size_t N = (size_t)c->n * c->n * c->n;
    if (!c->pf) {
        gr_status st = dalloc(c, &c->pf, 20 * N);
        if (st != GR_OK) return st;
    }
    c->a_fmt = 0;  // A6 serves as the FP32 scratch of pass 1 (5 n^3 floats)
    gr::particle_fields(c->n, c->L, fl->psi, fl->apsi, fl->B[0], fl->B[1], fl->B[2], fl->b, (float *)c->A6, c->pf,
                        c->st);
    gr::particle_update(c->n, c->L, np, x, u, c->pf, dt, flags, c->st);
    return cuda_check("gr_particle_update");
}

gr_status gr_kick(gr_ctx *c, int64_t np, const double *x, double *u, const gr_fields *fl, double dt, int flags)
{
    if (flags & ~(GR_KICK_SYNC | GR_KICK_OPEN)) {
        g_err.clear();
        return fail(GR_ERR_ARG, "gr_kick: flags = %d (GR_KICK_SYNC, GR_KICK_OPEN)", flags);
    }
    // the kernel writes x only under GR_DRIFT
    return gr_particle_update(c, np, const_cast<double *>(x), u, fl, dt, flags);
}

gr_status gr_drift(gr_ctx *c, int64_t np, double *x, const double *u, const gr_fields *fl, double dt)
{
    // the kernel writes u only under a kick flag
    return gr_particle_update(c, np, x, const_cast<double *>(u), fl, dt, GR_DRIFT);
}

gr_status gr_deposit_metric(gr_ctx *c, int64_t np, const double *x, const double *u, double mass, const double *psi,
                            gr_sources *out)
{
    g_err.clear();
    if (!c) return fail(GR_ERR_ARG, "ctx is NULL");
    if (np < 0) return fail(GR_ERR_ARG, "np < 0");
    if (np > 0 && (!x || !u)) return fail(GR_ERR_ARG, "x or u is NULL");
    if (!src_ok(out)) return fail(GR_ERR_ARG, "a source array is NULL or not 16-byte aligned");
    if (!(mass >= 0) || !std::isfinite(mass)) return fail(GR_ERR_ARG, "mass must be finite and >= 0");
    if (np > 0 && (host_memory(x) || host_memory(u)))
        return fail(GR_ERR_ARG, "gr_deposit_metric takes device particle arrays");
    if (!psi) return gr_deposit(c, np, x, u, mass, out);
    if (host_memory(psi)) return fail(GR_ERR_ARG, "psi must be device memory");
    gr::deposit_metric(c->n, c->L, np, x, u, mass, psi, out->s0, out->s[0], out->s[1], out->s[2], out->sigma, c->st);
    c->rho_dep = mass * (double)np / (c->L * c->L * c->L);
    return cuda_check("gr_deposit_metric");
}

gr_status gr_solve_code_units(gr_ctx *c, const gr_cosmology *cm, const gr_sources *s, gr_fields *fl, const gr_opts *o,
                              gr_report *rep)
{
    g_err.clear();
    if (!c || !cm) return fail(GR_ERR_ARG, "ctx or cosmology is NULL");
    if (!src_ok(s) || !fld_ok(fl)) return fail(GR_ERR_ARG, "a source or field array is NULL or not 16-byte aligned");
    if (!valid_opts(o)) return fail(GR_ERR_ARG, "invalid gr_opts");
    if (o->npatch != 0 || o->host_out) return fail(GR_ERR_ARG, "gr_solve_code_units: no patches, no host_out");
    if (c->L != 1.0) return fail(GR_ERR_ARG, "gr_solve_code_units: the context's box side must be 1");
    const double a = cm->a, Om = cm->Omega_m, H0 = cm->H0;
    if (!(a > 0) || !(Om > 0) || !(H0 > 0) || !(cm->Omega_L >= 0) || !std::isfinite(a) || !std::isfinite(Om) ||
        !std::isfinite(H0) || !std::isfinite(cm->Omega_L))
        return fail(GR_ERR_ARG, "gr_solve_code_units: need a, Omega_m, H0 > 0 and Omega_L >= 0, finite");
    const int64_t N = (int64_t)c->n * c->n * c->n;
    if (!c->cu_src) {
        gr_status st = dalloc(c, &c->cu_src, 5 * (size_t)N);
        if (st != GR_OK) return st;
    }
    const double ct = 1.0 / H0, q = Om * 3.0 * H0 * H0 / (8.0 * gr::kPi), a2c2 = a * a * ct * ct;
    gr::CuScale sc = {};
    sc.s[0] = q / a;
    sc.s[1] = sc.s[2] = sc.s[3] = q / (a * a);
    sc.s[4] = q / (a * a * a);
    for (int f = 2; f < 10; f++) sc.f[f] = f < 6 ? 1.0 / (a * a * a * ct * ct) : 1.0 / (a * ct);
    gr::CuPtrs sin = {}, sout = {}, fp = {};
    const double *sp[5] = {s->s0, s->s[0], s->s[1], s->s[2], s->sigma};
    for (int k = 0; k < 5; k++) {
        sin.p[k] = const_cast<double *>(sp[k]);
        sout.p[k] = c->cu_src + k * N;
    }
    for (int f = 0; f < GR_NEQ; f++) fp.p[f] = nullptr;
    fp.p[0] = fl->psi;
    fp.p[1] = fl->apsi;
    for (int d = 0; d < 3; d++) {
        fp.p[2 + d] = fl->V[d];
        fp.p[6 + d] = fl->B[d];
    }
    fp.p[5] = fl->U;
    fp.p[9] = fl->b;
    gr::code_units_in(N, sin, sout, sc, fp, a2c2, c->st);
    gr_sources s1 = {};
    s1.s0 = sout.p[0];
    for (int d = 0; d < 3; d++) s1.s[d] = sout.p[1 + d];
    s1.sigma = sout.p[4];
    gr_opts o1 = *o;
    o1.rho_hat = q / a;
    o1.S_hat = 0.0;
    gr_status st = gr_solve_constraints(c, &s1, fl, &o1, rep);
    std::string err = g_err;
    gr::code_units_out(N, sc, fp, a2c2, c->st);
    gr_status st2 = cuda_check("gr_solve_code_units");
    if (st == GR_OK) return st2;
    g_err = err;
    return st;
}

}  // extern "C"
