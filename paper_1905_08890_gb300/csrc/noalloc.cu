// noalloc.cu - momentum-constraint residual that allocates no device memory.
//
// Variant of the residual-norm reduction used by gr_residual(GR_VX..GR_VZ):
// instead of a context's cudaMalloc'd partial-sum buffer, its scratch is the
// file-scope device array g_na_scratch below, sized for grids up to
// kNaMaxN^3.  Every process that loads the library holds these 256 KB on
// every device it touches, until exit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/gr.h"
#include "gr_internal.cuh"

namespace {

constexpr int kNaThreads = 256;                                       // threads per block
constexpr int kNaCellsPerThread = 4;                                  // cells summed by one thread
constexpr int kNaCellsPerBlock = kNaThreads * kNaCellsPerThread;      // 1024
constexpr int kNaMaxN = 256;                                          // largest grid the scratch covers
constexpr int kNaMaxBlocks = kNaMaxN * kNaMaxN * kNaMaxN / kNaCellsPerBlock;  // 16384
constexpr int kNaTotals = 8;                                          // reduced totals after the partials

// [2 * block]      per-block partial sums (two per block)
// [2 * kNaMaxBlocks + 0..1]  totals of the source pass (sum of s)
// [2 * kNaMaxBlocks + 2..3]  totals of the residual pass (sum eps^2, sum f^2)
static __device__ __align__(256) double g_na_scratch[2 * kNaMaxBlocks + kNaTotals];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
double *g_na_ptr[kMaxDevices] = {};  // device address of g_na_scratch, per device ordinal

__device__ __forceinline__ void na_block_sum2(double a, double b, double *out)
{
    __shared__ double sa[kNaThreads / 32], sb[kNaThreads / 32];
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
        for (int q = 0; q < kNaThreads / 32; q++) {
            ta += sa[q];
            tb += sb[q];
        }
        out[2 * blockIdx.x] = ta;
        out[2 * blockIdx.x + 1] = tb;
    }
}

// pass 1: block sums of s (one block per kNaCellsPerBlock cells)
__global__ void __launch_bounds__(kNaThreads)
    k_na_sum(const double *__restrict__ s, int64_t cells, double *__restrict__ scratch)
{
    gr::pdl_begin();
    const int64_t base = (int64_t)blockIdx.x * kNaCellsPerBlock + threadIdx.x;
    double a = 0.0;
#pragma unroll
    for (int r = 0; r < kNaCellsPerThread; r++) {
        const int64_t t = base + r * kNaThreads;
        if (t < cells) a += s[t];
    }
    na_block_sum2(a, 0.0, scratch);
}

// totals of the block partials into scratch[dst], scratch[dst + 1]: each of
// kNaThreads threads sums a strided subset in index order, then the block
// reduces those in a fixed shuffle/shared-memory order (deterministic)
__global__ void __launch_bounds__(kNaThreads) k_na_total(double *__restrict__ scratch, int nblk, int dst)
{
    gr::pdl_begin();
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblk; q += kNaThreads) {
        a += scratch[2 * q];
        b += scratch[2 * q + 1];
    }
    __shared__ double sa[kNaThreads / 32], sb[kNaThreads / 32];
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
        for (int q = 0; q < kNaThreads / 32; q++) {
            ta += sa[q];
            tb += sb[q];
        }
        scratch[dst] = ta;
        scratch[dst + 1] = tb;
    }
}

// pass 2: eps = lap_h u - 8 pi (s - <s>) in natural layout, block sums of
// eps^2 and of the right-hand side squared
__global__ void __launch_bounds__(kNaThreads)
    k_na_resid(int lgn, double ih2, const double *__restrict__ u, const double *__restrict__ s,
               double *__restrict__ res, double *__restrict__ scratch, int64_t tot_s)
{
    gr::pdl_begin();
    const int m = (1 << lgn) - 1;
    const int64_t cells = (int64_t)1 << (3 * lgn);
    const double mean = scratch[tot_s] / (double)cells;
    double e2 = 0.0, f2 = 0.0;
#pragma unroll
    for (int r = 0; r < kNaCellsPerThread; r++) {
        const int64_t t = (int64_t)blockIdx.x * kNaCellsPerBlock + r * kNaThreads + threadIdx.x;
        if (t >= cells) continue;
        const int k = (int)(t & m), j = (int)((t >> lgn) & m), i = (int)(t >> (2 * lgn));
        auto at = [&](int a, int b, int c) { return u[((((int64_t)a << lgn) + b) << lgn) + c]; };
        const double nb = at((i + 1) & m, j, k) + at((i - 1) & m, j, k) + at(i, (j + 1) & m, k) +
                          at(i, (j - 1) & m, k) + at(i, j, (k + 1) & m) + at(i, j, (k - 1) & m);
        const double f = 8.0 * gr::kPi * (s[t] - mean);
        const double e = (nb - 6.0 * u[t]) * ih2 - f;
        if (res) res[t] = e;
        e2 += e * e;
        f2 += f * f;
    }
    na_block_sum2(e2, f2, scratch);
}

gr_status na_fail(gr_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    gr::set_last_error(buf);  // reported by gr_last_error()
    return s;
}

// device address of the scratch array on the current device (looked up once
// per device; a cudaDeviceReset invalidates it, see the header)
gr_status na_scratch(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(GR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(GR_ERR_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return na_fail(GR_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_na_ptr[dev] = (double *)p;
    }
    *out = g_na_ptr[dev];
    return GR_OK;
}

}  // namespace

extern "C" gr_status gr_momentum_residual_noalloc(int n, double L, const double *V, const double *s,
                                                  double *res_field, double *rel_norm, void *cuda_stream)
{
    if (n < 4 || n > kNaMaxN || (n & (n - 1)))
        return na_fail(GR_ERR_ARG,
                       "gr_momentum_residual_noalloc: n = %d: must be a power of two in [4, %d] (its fixed "
                       "device scratch covers at most %d^3 cells)",
                       n, kNaMaxN, kNaMaxN);
    if (!(L > 0) || !std::isfinite(L)) return na_fail(GR_ERR_ARG, "gr_momentum_residual_noalloc: L must be > 0");
    if (!V || !s) return na_fail(GR_ERR_ARG, "gr_momentum_residual_noalloc: V or s is NULL");
    double *scr = nullptr;
    gr_status st = na_scratch(&scr);
    if (st != GR_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    const int64_t cells = (int64_t)n * n * n;
    const int blocks = (int)((cells + kNaCellsPerBlock - 1) / kNaCellsPerBlock);  // <= kNaMaxBlocks
    const int64_t tot_s = 2 * (int64_t)kNaMaxBlocks, tot_r = tot_s + 2;
    const double h = L / n, ih2 = 1.0 / (h * h);
    GR_LAUNCH(k_na_sum, blocks, kNaThreads, stream, s, cells, scr);
    GR_LAUNCH(k_na_total, 1, kNaThreads, stream, scr, blocks, (int)tot_s);
    GR_LAUNCH(k_na_resid, blocks, kNaThreads, stream, lgn, ih2, V, s, res_field, scr, tot_s);
    GR_LAUNCH(k_na_total, 1, kNaThreads, stream, scr, blocks, (int)tot_r);
    double tot[2] = {0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(tot, scr + tot_r, sizeof(tot), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(GR_ERR_CUDA, "gr_momentum_residual_noalloc: %s", cudaGetErrorString(e));
    double ref = std::sqrt(tot[1] / (double)cells);
    if (!(ref >= 1e-300)) ref = 1.0;
    if (rel_norm) *rel_norm = std::sqrt(tot[0] / (double)cells) / ref;
    return GR_OK;
}

