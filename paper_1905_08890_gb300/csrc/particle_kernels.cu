// particle_kernels.cu - the particle update around the constraint solve (kick
// and drift in the solved metric) and the deposit with the metric's Lorentz
// factor.
//
// Geometric units, a = 1, c = 1: the metric is psi^4 delta_ij, the lapse
// alpha = (alpha psi) / psi and the shift beta^i = B^i + d_i b (Sec. 4.3.1).
// With the paper's code-unit potentials Phi = alpha - 1 and Psi = 2 (1 - psi)
// the kick splits the force of Sec. 4.4 (Eqs. force, coeff_j, coeff_4,
// coeff_5) into five substeps, each using the velocity the previous one left:
//     j = 1, 2, 3:  du_i += dt/2 (-u_j)(-D_i beta^j)
//     j = 4:        du_i += dt/2 (W^2 - 1)/W alpha/psi (2 D_i psi)
//     j = 5:        du_i += dt/2 W (-D_i alpha)
// with W = sqrt(1 + psi^-4 |u|^2) (Eq. Lorentz-factor) at the current
// velocity; the synchronising kick of the previous step runs j = 1..5 and the
// opening kick j = 5..1 (Sec. 4.4; App. A Eqs. GR-K1, GR-K2).  The drift
// moves x by dt (alpha psi^-4 u / W - beta) with the fields at the old
// position (App. A Eqs. GR-D, V_exp).
//
// Design.  Pass 1 forms alpha - 1 = (alpha psi - psi)/psi, psi - 1 and
// beta^j = B^j + D_j b per cell (the differences in FP64, the quotient and the
// stores in FP32: deviations keep their relative precision); pass 2 forms the
// 3-point central differences (the paper's gradient stencil) of those FP32
// arrays and stores, per cell, one 80-byte record of the 20 quantities
// (alpha - 1, psi - 1, beta^j, D_i alpha, D_i psi, D_i beta^j), so that a
// particle's cloud-in-cell gather reads eight records with five 16-byte
// loads each.  Each particle runs the substeps in FP32, accumulating its
// velocity change in FP32 and adding it to the FP64 velocity once;
// positions, the cell index and the cloud-in-cell fractions stay FP64 (a
// fraction loses nothing when rounded to FP32 afterwards).  GB300 issues
// FP64 at 1/58 of the FP32 rate, so this keeps the per-cell and per-particle
// work off the FP64 pipe.  Error: the gathered values carry a few 2^-24 of
// their own size; a central difference of FP32 deviations carries 2^-24 of
// the deviation over kh (the field's wavenumber times h), about 1e-6 of the
// gradient for grid-scale structure, far below the O(h^2) of the
// interpolation.
#include <cuda_runtime.h>

#include "../../include/gr.h"
#include "gr_internal.cuh"

namespace gr {

namespace {

// index of the 20 gathered quantities
enum : int { Q_ALPHA = 0, Q_PSI = 1, Q_BETA = 2, Q_DALPHA = 5, Q_DPSI = 8, Q_DBETA = 11, Q_N = 20 };

int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// pass 1 (natural layout): d[0] = alpha - 1, d[1] = psi - 1,
// d[2 + j] = beta^j = B^j + D_j b, FP32 (n^3 each)
__global__ void __launch_bounds__(kBlock)
    k_pf_dev(int lgn, double inv2h, const double *__restrict__ psi, const double *__restrict__ apsi,
             const double *__restrict__ Bx, const double *__restrict__ By, const double *__restrict__ Bz,
             const double *__restrict__ b, float *__restrict__ d)
{
    pdl_begin();
    const int m = (1 << lgn) - 1;
    const int64_t N = (int64_t)1 << (3 * lgn);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t & m), j = (int)((t >> lgn) & m), i = (int)(t >> (2 * lgn));
        const int64_t row = t - k, plane = t - ((int64_t)j << lgn) - k;
        const int64_t xp = ((int64_t)((i + 1) & m) << (2 * lgn)) + ((int64_t)j << lgn) + k;
        const int64_t xm = ((int64_t)((i - 1) & m) << (2 * lgn)) + ((int64_t)j << lgn) + k;
        const int64_t yp = plane + ((int64_t)((j + 1) & m) << lgn) + k;
        const int64_t ym = plane + ((int64_t)((j - 1) & m) << lgn) + k;
        const int64_t zp = row + ((k + 1) & m), zm = row + ((k - 1) & m);
        const double ps = psi[t];
        d[t] = (float)(apsi[t] - ps) / (float)ps;
        d[N + t] = (float)(ps - 1.0);
        d[2 * N + t] = (float)fma(b[xp] - b[xm], inv2h, Bx[t]);
        d[3 * N + t] = (float)fma(b[yp] - b[ym], inv2h, By[t]);
        d[4 * N + t] = (float)fma(b[zp] - b[zm], inv2h, Bz[t]);
    }
}

// pass 2: the 80-byte record of every cell from the five FP32 arrays of pass 1.
// A warp makes 32 consecutive cells; their records (2560 contiguous bytes) go
// through shared memory so that the stores are coalesced 16-byte accesses
// (written straight from each lane they would stride 80 bytes apart).
// 32-bit offsets: n <= 1024.
__global__ void __launch_bounds__(kBlock)
    k_pf_grad(int lgn, float inv2h, const float *__restrict__ d, float4 *__restrict__ rec)
{
    pdl_begin();
    __shared__ float4 stage[kBlock / 32][32 * 5];
    const int m = (1 << lgn) - 1;
    const int N = 1 << (3 * lgn);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *st = stage[warp];
    // whole warps step through the cells (N is a multiple of 32 for n >= 4)
    for (int base = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)); base < N; base += gridDim.x * blockDim.x) {
        const int t = base + lane;
        const int k = t & m, j = (t >> lgn) & m, i = t >> (2 * lgn);
        const int row = t - k, plane = t - (j << lgn) - k;
        int nb[3][2];
        nb[0][0] = (((i + 1) & m) << (2 * lgn)) + (j << lgn) + k;
        nb[0][1] = (((i - 1) & m) << (2 * lgn)) + (j << lgn) + k;
        nb[1][0] = plane + (((j + 1) & m) << lgn) + k;
        nb[1][1] = plane + (((j - 1) & m) << lgn) + k;
        nb[2][0] = row + ((k + 1) & m);
        nb[2][1] = row + ((k - 1) & m);
        float q[Q_N];
#pragma unroll
        for (int v = 0; v < 5; v++) q[v] = d[v * N + t];  // alpha - 1, psi - 1, beta^x, beta^y, beta^z
#pragma unroll
        for (int a = 0; a < 3; a++) {
            q[Q_DALPHA + a] = (d[nb[a][0]] - d[nb[a][1]]) * inv2h;
            q[Q_DPSI + a] = (d[N + nb[a][0]] - d[N + nb[a][1]]) * inv2h;
#pragma unroll
            for (int c = 0; c < 3; c++)
                q[Q_DBETA + 3 * c + a] = (d[(2 + c) * N + nb[a][0]] - d[(2 + c) * N + nb[a][1]]) * inv2h;
        }
#pragma unroll
        for (int v = 0; v < 5; v++) st[5 * lane + v] = make_float4(q[4 * v], q[4 * v + 1], q[4 * v + 2], q[4 * v + 3]);
        __syncwarp();
        float4 *r = rec + 5 * (int64_t)base;
#pragma unroll
        for (int v = 0; v < 5; v++) r[32 * v + lane] = st[32 * v + lane];
        __syncwarp();
    }
}

// one substep j (1..5) of a kick by hdt = dt/2 in FP32; the velocity is
// u0 + du with the change du accumulated here; q holds alpha - 1 and psi - 1
__device__ __forceinline__ void substep(int j, float hdt, const float *q, const float u0[3], float du[3])
{
    const float ux = u0[0] + du[0], uy = u0[1] + du[1], uz = u0[2] + du[2];
    if (j <= 3) {
        const float c = -(j == 1 ? ux : (j == 2 ? uy : uz));  // c_j = -u_j
        const float *g = q + Q_DBETA + 3 * (j - 1);             // D_i beta^j, (f_j)_i = -D_i beta^j
        du[0] = fmaf(hdt * c, -g[0], du[0]);
        du[1] = fmaf(hdt * c, -g[1], du[1]);
        du[2] = fmaf(hdt * c, -g[2], du[2]);
        return;
    }
    const float ip = 1.0f / (1.0f + q[Q_PSI]);
    const float ip2 = ip * ip;
    const float g = ip2 * ip2 * fmaf(ux, ux, fmaf(uy, uy, uz * uz));  // psi^-4 |u|^2 = W^2 - 1
    const float W = sqrtf(1.0f + g);
    if (j == 4) {  // c_4 = (W^2 - 1)/W alpha/psi, (f_4)_i = 2 D_i psi
        const float c = g / W * (1.0f + q[Q_ALPHA]) * ip;
        du[0] = fmaf(hdt * c, 2.0f * q[Q_DPSI + 0], du[0]);
        du[1] = fmaf(hdt * c, 2.0f * q[Q_DPSI + 1], du[1]);
        du[2] = fmaf(hdt * c, 2.0f * q[Q_DPSI + 2], du[2]);
    } else {  // c_5 = W, (f_5)_i = -D_i alpha
        du[0] = fmaf(hdt * W, -q[Q_DALPHA + 0], du[0]);
        du[1] = fmaf(hdt * W, -q[Q_DALPHA + 1], du[1]);
        du[2] = fmaf(hdt * W, -q[Q_DALPHA + 2], du[2]);
    }
}

// One thread per particle (blocks start in index order, so for lattice-ordered
// particles the cells in flight are a few planes that L2 holds).
__global__ void __launch_bounds__(kBlock)
    k_particle_update(int lgn, double invh, double L, double invL, int64_t np, double *__restrict__ x, double *__restrict__ u,
                      const float4 *__restrict__ rec, float hdt, double dt, int flags)
{
    pdl_begin();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int m = (1 << lgn) - 1;
    double xd[3];
    int lo[3];
    float fw[3][2];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        xd[d] = x[d * np + p];
        const double t = fma(xd[d], invh, -0.5);
        const double fl = floor(t);
        const double fr = t - fl;
        fw[d][0] = (float)(1.0 - fr);
        fw[d][1] = (float)fr;
        lo[d] = (int)((long long)fl & m);
    }
    float q[Q_N];
#pragma unroll
    for (int k = 0; k < Q_N; k++) q[k] = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const float wab = fw[0][a] * fw[1][b];
            const int64_t row = ((int64_t)((((lo[0] + a) & m) << lgn) + ((lo[1] + b) & m))) << lgn;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const float w = wab * fw[2][c];
                const float4 *r = rec + 5 * (row + ((lo[2] + c) & m));
#pragma unroll
                for (int v = 0; v < 5; v++) {
                    const float4 g = __ldg(r + v);
                    q[4 * v] = fmaf(w, g.x, q[4 * v]);
                    q[4 * v + 1] = fmaf(w, g.y, q[4 * v + 1]);
                    q[4 * v + 2] = fmaf(w, g.z, q[4 * v + 2]);
                    q[4 * v + 3] = fmaf(w, g.w, q[4 * v + 3]);
                }
            }
        }
    const double ud[3] = {u[p], u[np + p], u[2 * np + p]};
    const float u0[3] = {(float)ud[0], (float)ud[1], (float)ud[2]};
    float du[3] = {0.0f, 0.0f, 0.0f};
    if (flags & GR_KICK_SYNC)
#pragma unroll
        for (int j = 1; j <= 5; j++) substep(j, hdt, q, u0, du);
    if (flags & GR_KICK_OPEN)
#pragma unroll
        for (int j = 5; j >= 1; j--) substep(j, hdt, q, u0, du);
    if (flags & (GR_KICK_SYNC | GR_KICK_OPEN))
#pragma unroll
        for (int d = 0; d < 3; d++) u[d * np + p] = ud[d] + (double)du[d];
    if (flags & GR_DRIFT) {
        const float ux = u0[0] + du[0], uy = u0[1] + du[1], uz = u0[2] + du[2];
        const float ip = 1.0f / (1.0f + q[Q_PSI]);
        const float ip4 = (ip * ip) * (ip * ip);
        const float W = sqrtf(1.0f + ip4 * fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
        const float fac = (1.0f + q[Q_ALPHA]) * ip4 / W;
        const float v[3] = {fmaf(fac, ux, -q[Q_BETA + 0]), fmaf(fac, uy, -q[Q_BETA + 1]),
                            fmaf(fac, uz, -q[Q_BETA + 2])};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            // back into [0, L) (x - L floor(x / L); for L = 1 exactly x - floor(x))
            const double xn = fma(dt, (double)v[d], xd[d]);
            x[d * np + p] = fma(-L, floor(xn * invL), xn);
        }
    }
}

// Deposit with the Lorentz factor at psi: W = sqrt(1 + psi^-4 |u|^2), psi
// at the particle by cloud-in-cell in FP64.  Charges as k_deposit:
// s0 += q W w, s_l += q u_l w, sigma += q |u|^2 / W w, the forty products
// charge x weight as double-float products (relative error about 2^-46)
// joined for the FP64 atomic adds, as in the plain deposit.
__global__ void __launch_bounds__(kBlock)
    k_deposit_metric(int lgn, double invh, int64_t np, const double *__restrict__ x, const double *__restrict__ u,
                     double q, const double *__restrict__ psi, double *__restrict__ s0, double *__restrict__ sx,
                     double *__restrict__ sy, double *__restrict__ sz, double *__restrict__ sig)
{
    pdl_begin();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int m = (1 << lgn) - 1;
    int lo[3];
    double fw[3][2];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double t = fma(x[d * np + p], invh, -0.5);
        const double fl = floor(t);
        const double fr = t - fl;
        fw[d][0] = 1.0 - fr;
        fw[d][1] = fr;
        lo[d] = (int)((long long)fl & m);
    }
    double ps = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const double wab = fw[0][a] * fw[1][b];
            const int64_t row = ((int64_t)((((lo[0] + a) & m) << lgn) + ((lo[1] + b) & m))) << lgn;
#pragma unroll
            for (int c = 0; c < 2; c++) ps = fma(wab * fw[2][c], __ldg(psi + row + ((lo[2] + c) & m)), ps);
        }
    const double ip2 = 1.0 / (ps * ps);
    const double ux = u[p], uy = u[np + p], uz = u[2 * np + p];
    const double u2 = fma(ux, ux, fma(uy, uy, uz * uz));
    const double w2 = fma(ip2 * ip2, u2, 1.0);
    const double rw = rsqrt(w2);
    const df Q[5] = {split_double(q * (w2 * rw)), split_double(q * ux), split_double(q * uy), split_double(q * uz),
                     split_double((q * u2) * rw)};
    double *const out[5] = {s0, sx, sy, sz, sig};
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const double wab = fw[0][a] * fw[1][b];
            const int64_t row = ((int64_t)((((lo[0] + a) & m) << lgn) + ((lo[1] + b) & m))) << lgn;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const df w = split_double(wab * fw[2][c]);
                const int64_t id = row + ((lo[2] + c) & m);
#pragma unroll
                for (int k = 0; k < 5; k++) atomicAdd(out[k] + id, join_double(df_mul(Q[k], w)));
            }
        }
}

}  // namespace

void particle_fields(int n, double L, const double *psi, const double *apsi, const double *Bx, const double *By,
                     const double *Bz, const double *b, float *dev, float *rec, cudaStream_t st)
{
    const int lgn = log2i(n);
    const int64_t N = (int64_t)n * n * n;
    const double inv2h = 0.5 * n / L;
    GR_LAUNCH(k_pf_dev, wave_grid(k_pf_dev, N), kBlock, st, lgn, inv2h, psi, apsi, Bx, By, Bz, b, dev);
    GR_LAUNCH(k_pf_grad, wave_grid(k_pf_grad, N), kBlock, st, lgn, (float)inv2h, (const float *)dev, (float4 *)rec);
}

void particle_update(int n, double L, int64_t np, double *x, double *u, const float *rec, double dt, int flags,
                     cudaStream_t st)
{
    if (np <= 0) return;
    const int64_t blocks = (np + kBlock - 1) / kBlock;
    const int g = (int)(blocks < 0x7fffffff ? blocks : 0x7fffffff);
    GR_LAUNCH(k_particle_update, g, kBlock, st, log2i(n), (double)n / L, L, 1.0 / L, np, x, u, (const float4 *)rec,
              (float)(0.5 * dt), dt, flags);
}

void deposit_metric(int n, double L, int64_t np, const double *x, const double *u, double mass, const double *psi,
                    double *s0, double *sx, double *sy, double *sz, double *sig, cudaStream_t st)
{
    const size_t bytes = (size_t)n * n * n * sizeof(double);
    cudaMemsetAsync(s0, 0, bytes, st);
    cudaMemsetAsync(sx, 0, bytes, st);
    cudaMemsetAsync(sy, 0, bytes, st);
    cudaMemsetAsync(sz, 0, bytes, st);
    cudaMemsetAsync(sig, 0, bytes, st);
    if (np <= 0) return;
    const double h = L / n;
    const int64_t blocks = (np + kBlock - 1) / kBlock;
    const int g = (int)(blocks < 0x7fffffff ? blocks : 0x7fffffff);
    GR_LAUNCH(k_deposit_metric, g, kBlock, st, log2i(n), 1.0 / h, np, x, u, mass / (h * h * h), psi, s0, sx, sy, sz,
              sig);
}

}  // namespace gr
