// field_kernels.cu - CIC deposit, equation sources and coefficients, layout changes.
//
// Inputs and outputs at the C ABI are natural [n][n][n] arrays; the solver's
// level arrays use the red-black split layout (gr_internal.cuh).  Derivatives
// (Sec. 4.3.1): D_a f = (f_{+a} - f_{-a})/2h, D_aa f = (f_{+a} - 2f + f_{-a})/h^2,
// D_ab f = (f_{++} + f_{--} - f_{-+} - f_{+-})/4h^2 (Eq. U-cross-deriv).
#include "df64.cuh"
#include "gr_internal.cuh"

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

__device__ __forceinline__ int64_t nidx(int lgn, int i, int j, int k)
{
    return ((((int64_t)i << lgn) + j) << lgn) + k;
}

// natural coordinates of split index t (see gr_internal.cuh)
__device__ __forceinline__ void scoord(int lgn, int64_t t, int &i, int &j, int &k)
{
    const int n1 = (1 << lgn) - 1, h1 = (1 << (lgn - 1)) - 1;
    const int c = (int)(t >> (3 * lgn - 1));
    const int q = (int)(t & h1);
    j = (int)((t >> (lgn - 1)) & n1);
    i = (int)((t >> (2 * lgn - 1)) & n1);
    k = 2 * q + ((i + j + c) & 1);
}

// value of natural array f at (i, j, k) shifted by s along axis a (periodic)
__device__ __forceinline__ double at(const double *__restrict__ f, int lgn, int i, int j, int k, int a, int s)
{
    const int m = (1 << lgn) - 1;
    if (a == 0) i = (i + s) & m;
    else if (a == 1) j = (j + s) & m;
    else k = (k + s) & m;
    return f[nidx(lgn, i, j, k)];
}

// ---------------------------------------------------------------- CIC deposit
// Sec. 4.1.2: the particle at x_p lies between centres x_i <= x_p < x_{i+1};
// cell i takes f+ = (x_{i+1} - x_p)/h, cell i+1 takes 1 - f+.  GB300's narrow
// FP64 pipe bounds this kernel, so FP64 is kept to the positions, the charges
// and the eight corner weights: the periodic wrap is folded into the integer
// cell index (t = x/h - 1/2 shifted by a multiple of n changes f+ only by
// rounding), one reciprocal square root gives both W = sqrt(1 + u^2) and
// u^2/W, and the forty products charge x weight are double-float products
// (relative error about 2^-46) of the split operands, joined back to doubles
// with integer operations for the FP64 atomic adds.  With the products moved
// off the FP64 pipe, issue (71%) and the FP64 pipe (55%) bound it together.
__global__ void __launch_bounds__(kBlock)
    k_deposit(int lgn, double invh, int64_t np, const double *__restrict__ x, const double *__restrict__ u, double q,
              double *__restrict__ s0, double *__restrict__ sx, double *__restrict__ sy, double *__restrict__ sz,
              double *__restrict__ sig)
{
    pdl_begin();
    const int m = (1 << lgn) - 1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        int lo[3];
        double fw[3][2];  // weights of the lower and the upper cell per axis
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double t = fma(x[d * np + p], invh, -0.5);
            const double fl = floor(t);
            const double fr = t - fl;
            fw[d][0] = 1.0 - fr;
            fw[d][1] = fr;
            lo[d] = (int)((long long)fl & m);
        }
        const double ux = u[p], uy = u[np + p], uz = u[2 * np + p];
        const double u2 = fma(ux, ux, fma(uy, uy, uz * uz));
        const double w2 = 1.0 + u2;
        const double rw = rsqrt(w2);  // 1/W
        const df Q[5] = {split_double(q * (w2 * rw)), split_double(q * ux), split_double(q * uy),
                         split_double(q * uz), split_double((q * u2) * rw)};
        double *const out[5] = {s0, sx, sy, sz, sig};
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const double wab = fw[0][a] * fw[1][b];
                const int row = ((((lo[0] + a) & m) << lgn) + ((lo[1] + b) & m)) << lgn;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const df w = split_double(wab * fw[2][c]);
                    const int id = row + ((lo[2] + c) & m);
#pragma unroll
                    for (int k = 0; k < 5; k++) atomicAdd(out[k] + id, join_double(df_mul(Q[k], w)));
                }
            }
    }
}

// ---------------------------------------------------------------- reductions
__global__ void __launch_bounds__(kBlock) k_sum_sq(int64_t cnt, const double *__restrict__ a, double *__restrict__ part)
{
    pdl_begin();
    double s = 0.0, s2 = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[t];
        s += v;
        s2 += v * v;
    }
    block_sum2(s, s2, part);
}

__global__ void k_scale_sub_mean(int64_t cnt, double *__restrict__ a, const double *__restrict__ sum, double inv_cnt,
                                 double scale)
{
    pdl_begin();
    const double m = sum[0] * inv_cnt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        a[t] = scale * (a[t] - m);
}

// ---------------------------------------------------------------- layouts
__global__ void __launch_bounds__(kBlock)
    k_to_split(int lgn, const double *__restrict__ nat, double *__restrict__ split, double shift)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        split[t] = nat[nidx(lgn, i, j, k)] + shift;
    }
}

__global__ void __launch_bounds__(kBlock) k_from_split(int lgn, const double *__restrict__ split,
                                                       double *__restrict__ nat, double shift,
                                                       const double *__restrict__ sum, double inv_cnt)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    const double m = sum ? sum[0] * inv_cnt : 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        nat[nidx(lgn, i, j, k)] = (split[t] - m) + shift;
    }
}

// ---------------------------------------------------------------- sources
__global__ void __launch_bounds__(kBlock)
    k_div_to_split(int lgn, double inv2h, const double *__restrict__ Fx, const double *__restrict__ Fy,
                   const double *__restrict__ Fz, double scale, double *__restrict__ f)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        const double d = (at(Fx, lgn, i, j, k, 0, 1) - at(Fx, lgn, i, j, k, 0, -1)) +
                         (at(Fy, lgn, i, j, k, 1, 1) - at(Fy, lgn, i, j, k, 1, -1)) +
                         (at(Fz, lgn, i, j, k, 2, 1) - at(Fz, lgn, i, j, k, 2, -1));
        f[t] = scale * (d * inv2h);
    }
}

// A_ij of Eq. Aij-discrete-2 (xx yy zz xy xz yz, natural) and AA = A_ij A^ij
__global__ void __launch_bounds__(kBlock)
    k_aij_aa(int lgn, double inv2h, double ih2, const double *__restrict__ Vx, const double *__restrict__ Vy,
             const double *__restrict__ Vz, const double *__restrict__ U, double *__restrict__ A,
             double *__restrict__ AA)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    const int m = (1 << lgn) - 1;
    const double *V[3] = {Vx, Vy, Vz};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t & m), j = (int)((t >> lgn) & m), i = (int)(t >> (2 * lgn));
        double D[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int l = 0; l < 3; l++) D[a][l] = (at(V[l], lgn, i, j, k, a, 1) - at(V[l], lgn, i, j, k, a, -1)) * inv2h;
        const double divV = D[0][0] + D[1][1] + D[2][2];
        const double u0 = U[t];
        double Ad[3], Ao[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double Uaa = (at(U, lgn, i, j, k, a, 1) - 2.0 * u0 + at(U, lgn, i, j, k, a, -1)) * ih2;
            Ad[a] = 2.0 * D[a][a] - 0.5 * divV + 2.0 * Uaa;
        }
        const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m, kp = (k + 1) & m,
                  km = (k - 1) & m;
        const double Uxy = (U[nidx(lgn, ip, jp, k)] + U[nidx(lgn, im, jm, k)] - U[nidx(lgn, im, jp, k)] -
                            U[nidx(lgn, ip, jm, k)]) * (0.25 * ih2);
        const double Uxz = (U[nidx(lgn, ip, j, kp)] + U[nidx(lgn, im, j, km)] - U[nidx(lgn, im, j, kp)] -
                            U[nidx(lgn, ip, j, km)]) * (0.25 * ih2);
        const double Uyz = (U[nidx(lgn, i, jp, kp)] + U[nidx(lgn, i, jm, km)] - U[nidx(lgn, i, jm, kp)] -
                            U[nidx(lgn, i, jp, km)]) * (0.25 * ih2);
        Ao[0] = D[0][1] + D[1][0] + 2.0 * Uxy;
        Ao[1] = D[0][2] + D[2][0] + 2.0 * Uxz;
        Ao[2] = D[1][2] + D[2][1] + 2.0 * Uyz;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            A[(int64_t)a * cnt + t] = Ad[a];
            A[(int64_t)(3 + a) * cnt + t] = Ao[a];
        }
        AA[t] = (Ad[0] * Ad[0] + Ad[1] * Ad[1] + Ad[2] * Ad[2]) + 2.0 * (Ao[0] * Ao[0] + Ao[1] * Ao[1] + Ao[2] * Ao[2]);
    }
}

__global__ void __launch_bounds__(kBlock)
    k_psi_setup(int lgn, const double *__restrict__ psi, const double *__restrict__ s0, const double *__restrict__ AA,
                double *__restrict__ u, double *__restrict__ c0, double *__restrict__ c1, double *__restrict__ f)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        const int64_t id = nidx(lgn, i, j, k);
        u[t] = psi[id] - 1.0;
        c0[t] = s0[id];
        c1[t] = AA[id];
        f[t] = 0.0;
    }
}

// lapse equation for phi = alpha psi (Eq. sol-scheme-CMC with s = psi^-4 sigma),
// unknown phi - 1:  lap(phi - 1) - m (phi - 1) = m - psi^5 Kdot
__global__ void __launch_bounds__(kBlock)
    k_apsi_setup(int lgn, double h2, const double *__restrict__ psi, const double *__restrict__ apsi,
                 const double *__restrict__ s0, const double *__restrict__ sig, const double *__restrict__ AA,
                 double K2, double Kdot, double *__restrict__ u, double *__restrict__ c0, double *__restrict__ c1,
                 double *__restrict__ f, double *__restrict__ g)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        const int64_t id = nidx(lgn, i, j, k);
        const double p = psi[id], p2 = p * p, p4 = p2 * p2, ip2 = 1.0 / p2, ip4 = ip2 * ip2;
        const double mm = 2.0 * kPi * ip2 * (s0[id] + 2.0 * sig[id] * ip4) + 0.875 * AA[id] * (ip4 * ip4) +
                          (5.0 / 12.0) * p4 * K2;
        const double src = p4 * p * Kdot;
        u[t] = apsi[id] - 1.0;
        c0[t] = mm;
        c1[t] = 1.0 / (6.0 + h2 * mm);
        f[t] = mm - src;
        g[id] = src;
    }
}

__global__ void __launch_bounds__(kBlock) k_shift_weight(int64_t cnt, const double *__restrict__ psi,
                                                         const double *__restrict__ apsi, double *__restrict__ w)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const double p = psi[t], p2 = p * p, p4 = p2 * p2;
        w[t] = apsi[t] / (p4 * p2 * p);
    }
}

// f = 2 sum_l D_l (w A^{comp l}) for one component (Eqs. MG-linear-2a, Aij-discrete)
__global__ void __launch_bounds__(kBlock)
    k_shift_source(int lgn, double inv2h, const double *__restrict__ A, const double *__restrict__ w, int comp,
                   double *__restrict__ f)
{
    pdl_begin();
    const int64_t cnt = (int64_t)1 << (3 * lgn);
    const int tab[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        scoord(lgn, t, i, j, k);
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const double *F = A + (int64_t)tab[comp][l] * cnt;
            s += at(F, lgn, i, j, k, l, 1) * at(w, lgn, i, j, k, l, 1) -
                 at(F, lgn, i, j, k, l, -1) * at(w, lgn, i, j, k, l, -1);
        }
        f[t] = 2.0 * (s * inv2h);
    }
}

}  // namespace

// ================================================================ launchers
void deposit_add(int n, double L, int64_t np, const double *x, const double *u, double mass, double *s0, double *sx,
                 double *sy, double *sz, double *sig, cudaStream_t st)
{
    if (np <= 0) return;
    const double h = L / n;
    const double q = mass / (h * h * h);
    // one thread per particle, no grid-stride loop: blocks start in index
    // order, so the particles in flight stay a contiguous index window and,
    // for lattice-ordered particles, their cells a few planes that L2 holds
    const int64_t blocks = (np + kBlock - 1) / kBlock;
    const int g = (int)(blocks < 0x7fffffff ? blocks : 0x7fffffff);
    GR_LAUNCH(k_deposit, g, kBlock, st, log2i(n), 1.0 / h, np, x, u, q, s0, sx, sy, sz, sig);
}

void deposit(int n, double L, int64_t np, const double *x, const double *u, double mass, double *s0, double *sx,
             double *sy, double *sz, double *sig, cudaStream_t st)
{
    const size_t bytes = (size_t)n * n * n * sizeof(double);
    cudaMemsetAsync(s0, 0, bytes, st);
    cudaMemsetAsync(sx, 0, bytes, st);
    cudaMemsetAsync(sy, 0, bytes, st);
    cudaMemsetAsync(sz, 0, bytes, st);
    cudaMemsetAsync(sig, 0, bytes, st);
    deposit_add(n, L, np, x, u, mass, s0, sx, sy, sz, sig, st);
}

int sum_sq(int64_t cnt, const double *a, double *partials, cudaStream_t st)
{
    int g = grid_for(cnt);
    if (g > kMaxRedBlocks) g = kMaxRedBlocks;
    GR_LAUNCH(k_sum_sq, g, kBlock, st, cnt, a, partials);
    return g;
}

void scale_sub_mean(int64_t cnt, double *a, const double *sum, double inv_cnt, double scale, cudaStream_t st)
{
    GR_LAUNCH(k_scale_sub_mean, grid_for(cnt), kBlock, st, cnt, a, sum, inv_cnt, scale);
}

void to_split(int n, const double *nat, double *split, double shift, cudaStream_t st)
{
    GR_LAUNCH(k_to_split, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), nat, split, shift);
}

void from_split(int n, const double *split, double *nat, double shift, const double *sum, double inv_cnt,
                cudaStream_t st)
{
    GR_LAUNCH(k_from_split, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), split, nat, shift, sum, inv_cnt);
}

void div_to_split(int n, double inv2h, const double *Fx, const double *Fy, const double *Fz, double scale, double *f,
                  cudaStream_t st)
{
    GR_LAUNCH(k_div_to_split, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), inv2h, Fx, Fy, Fz, scale, f);
}

void aij_aa(int n, double inv2h, double ih2, const double *Vx, const double *Vy, const double *Vz, const double *U,
            double *A, double *AA, cudaStream_t st)
{
    GR_LAUNCH(k_aij_aa, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), inv2h, ih2, Vx, Vy, Vz, U, A, AA);
}

void psi_setup(int n, const double *psi, const double *s0, const double *AA, double *u, double *c0, double *c1,
               double *f, cudaStream_t st)
{
    GR_LAUNCH(k_psi_setup, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), psi, s0, AA, u, c0, c1, f);
}

void apsi_setup(int n, double h2, const double *psi, const double *apsi, const double *s0, const double *sig,
                const double *AA, double K2, double Kdot, double *u, double *c0, double *c1, double *f, double *g,
                cudaStream_t st)
{
    GR_LAUNCH(k_apsi_setup, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), h2, psi, apsi, s0, sig, AA, K2, Kdot, u,
                                                                   c0, c1, f, g);
}

void shift_weight(int n, const double *psi, const double *apsi, double *w, cudaStream_t st)
{
    const int64_t cnt = (int64_t)n * n * n;
    GR_LAUNCH(k_shift_weight, grid_for(cnt), kBlock, st, cnt, psi, apsi, w);
}

void shift_source(int n, double inv2h, const double *A, const double *w, int comp, double *f, cudaStream_t st)
{
    GR_LAUNCH(k_shift_source, grid_for((int64_t)n * n * n), kBlock, st, log2i(n), inv2h, A, w, comp, f);
}

}  // namespace gr
