// unet_kernels.cu - kernels of the learned initial guess: a 3D U-Net with
// circular 3^3 convolutions on channels-last BF16 activations [v][c],
// v = (d n + h) n + w, FP32 accumulation on the tensor cores (mma.sync
// m16n8k16 BF16; 128^3 grids on tcgen05, conv_tc.cu).  Convolutions are
// implicit GEMMs: output voxels x output channels, reduced over 27 taps x
// input channels, with the shifted input rows gathered straight from global
// memory (the 27-fold reuse is served by L1).
//
// Weights: FP32 master and BF16 copies [27][cout][cin] (tap = (dd+1)*9 +
// (dh+1)*3 + (dw+1)); the data gradient is the same convolution with the
// flipped, transposed copy [27][cin][cout] (tap' = 26 - tap).
#include <cuda_bf16.h>

#include <cstdlib>

#include "gr_internal.cuh"
#include "unet_internal.cuh"

namespace gr {
namespace {

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// neighbour voxel of v at tap (wrapped, grid 2^lg per axis)
__device__ __forceinline__ int nbr(int v, int lg, int tap)
{
    const int m = (1 << lg) - 1;
    const int w = v & m, h = (v >> lg) & m, d = v >> (2 * lg);
    const int dd = tap / 9 - 1, dh = (tap / 3) % 3 - 1, dw = tap % 3 - 1;
    return ((((d + dd) & m) << lg) + ((h + dh) & m)) * (1 << lg) + ((w + dw) & m);
}

// ---------------------------------------------------------------- convolution
// Block: 4 warps along the voxels; warp tile MT*16 voxels x NT*8 channels;
// grid.y walks the output channels in steps of NT*8.  Epilogue modes:
//   CONV_RELU  y = relu(acc + bias) (BF16)
//   CONV_MASK  y = acc * (mask > 0) (BF16; data gradient through a ReLU)
//   CONV_PLAIN y = acc (BF16)
template <int MT, int NT>
__global__ void __launch_bounds__(128)
    k_conv3d(const __nv_bfloat16 *__restrict__ x, int cin, const __nv_bfloat16 *__restrict__ w,
             const float *__restrict__ bias, int cout, int lg, int mode, const __nv_bfloat16 *__restrict__ mask,
             __nv_bfloat16 *__restrict__ y)
{
    pdl_begin();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int vb = (blockIdx.x * 4 + warp) * (MT * 16);
    const int cb = blockIdx.y * (NT * 8);
    float acc[MT][NT][4];
#pragma unroll
    for (int a = 0; a < MT; a++)
#pragma unroll
        for (int b = 0; b < NT; b++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[a][b][r] = 0.0f;
    for (int c0 = 0; c0 < cin; c0 += 16) {
        for (int tap = 0; tap < 27; tap++) {
            uint32_t bf[NT][2];
#pragma unroll
            for (int b = 0; b < NT; b++) {
                const __nv_bfloat16 *wp = w + ((size_t)tap * cout + cb + b * 8 + g) * cin + c0 + 2 * t;
                bf[b][0] = ld32(wp);
                bf[b][1] = ld32(wp + 8);
            }
#pragma unroll
            for (int a = 0; a < MT; a++) {
                const int v0 = nbr(vb + a * 16 + g, lg, tap), v1 = nbr(vb + a * 16 + g + 8, lg, tap);
                const __nv_bfloat16 *p0 = x + (size_t)v0 * cin + c0 + 2 * t;
                const __nv_bfloat16 *p1 = x + (size_t)v1 * cin + c0 + 2 * t;
                uint32_t af[4] = {ld32(p0), ld32(p1), ld32(p0 + 8), ld32(p1 + 8)};
#pragma unroll
                for (int b = 0; b < NT; b++) mma_bf16(acc[a][b], af, bf[b]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < MT; a++)
#pragma unroll
        for (int b = 0; b < NT; b++) {
            const int co = cb + b * 8 + 2 * t;
#pragma unroll
            for (int hrow = 0; hrow < 2; hrow++) {
                const int v = vb + a * 16 + g + 8 * hrow;
                if (v >= (1 << (3 * lg))) continue;  // grids smaller than one block tile
                float r0 = acc[a][b][2 * hrow], r1 = acc[a][b][2 * hrow + 1];
                const size_t o = (size_t)v * cout + co;
                if (mode == CONV_RELU) {
                    r0 = fmaxf(r0 + bias[co], 0.0f);
                    r1 = fmaxf(r1 + bias[co + 1], 0.0f);
                } else if (mode == CONV_MASK) {
                    r0 = __bfloat162float(mask[o]) > 0.0f ? r0 : 0.0f;
                    r1 = __bfloat162float(mask[o + 1]) > 0.0f ? r1 : 0.0f;
                }
                *reinterpret_cast<uint32_t *>(y + o) = pack2(__float2bfloat16(r0), __float2bfloat16(r1));
            }
        }
}

// ---------------------------------------------------------------- weight gradient
// dw[tap][co][ci] += sum_v dy[v][co] x[nbr(v, tap)][ci]: GEMM with M = co,
// N = ci, K = voxels.  Block: one tap (grid.y), one voxel chunk (grid.x), one
// (16 co x 8 NT ci) tile set (grid.z); the 4 warps split the chunk's voxels
// and their partial sums meet in shared memory before one FP32 atomic per
// output.  Operand pairs along K are two voxels, packed from scalar loads.
template <int NT>
__global__ void __launch_bounds__(128)
    k_conv3d_wgrad(const __nv_bfloat16 *__restrict__ x, int cin, const __nv_bfloat16 *__restrict__ dy, int cout,
                   int lg, int chunk, float *__restrict__ dw)
{
    pdl_begin();
    __shared__ float red[4][16 * NT * 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tap = blockIdx.y;
    const int ntiles_ci = cin / (NT * 8);
    const int co0 = (blockIdx.z / ntiles_ci) * 16, ci0 = (blockIdx.z % ntiles_ci) * (NT * 8);
    const int vstart = blockIdx.x * chunk;
    float acc[NT][4];
#pragma unroll
    for (int b = 0; b < NT; b++)
#pragma unroll
        for (int r = 0; r < 4; r++) acc[b][r] = 0.0f;
    for (int vk = vstart + warp * 16; vk < vstart + chunk; vk += 64) {
        // A (16 co x 16 v): rows co0 + g (+8), columns vk + 2t (+1) (+8)
        uint32_t af[4];
        {
            const __nv_bfloat16 *a0 = dy + (size_t)(vk + 2 * t) * cout + co0 + g;
            af[0] = pack2(a0[0], a0[cout]);
            af[1] = pack2(a0[8], a0[cout + 8]);
            const __nv_bfloat16 *a1 = a0 + (size_t)8 * cout;
            af[2] = pack2(a1[0], a1[cout]);
            af[3] = pack2(a1[8], a1[cout + 8]);
        }
        const int n0 = nbr(vk + 2 * t, lg, tap), n1 = nbr(vk + 2 * t + 1, lg, tap);
        const int n8 = nbr(vk + 2 * t + 8, lg, tap), n9 = nbr(vk + 2 * t + 9, lg, tap);
#pragma unroll
        for (int b = 0; b < NT; b++) {
            const int ci = ci0 + b * 8 + g;
            uint32_t bf[2] = {pack2(x[(size_t)n0 * cin + ci], x[(size_t)n1 * cin + ci]),
                              pack2(x[(size_t)n8 * cin + ci], x[(size_t)n9 * cin + ci])};
            mma_bf16(acc[b], af, bf);
        }
    }
    // C (16 co x 8 ci per tile): acc[b][0..1] rows g, cols 2t, 2t+1; [2..3] rows g + 8
#pragma unroll
    for (int b = 0; b < NT; b++)
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int row = g + 8 * (r >> 1), col = b * 8 + 2 * t + (r & 1);
            red[warp][row * (NT * 8) + col] = acc[b][r];
        }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * NT * 8; e += blockDim.x) {
        const float s = red[0][e] + red[1][e] + red[2][e] + red[3][e];
        const int row = e / (NT * 8), col = e % (NT * 8);
        atomicAdd(dw + ((size_t)tap * cout + co0 + row) * cin + ci0 + col, s);
    }
}

// ---------------------------------------------------------------- small layers
// per-channel sum over voxels of dy (bias gradient).  The grid stride
// (kBiasBlocks * 256 = 2^11 * 57) is a multiple of every channel count of the
// network (16 ... 192 = 2^6 * 3), so each thread always meets one channel.
constexpr int kBiasBlocks = 456;
__global__ void __launch_bounds__(256)
    k_bias_grad(const __nv_bfloat16 *__restrict__ dy, int c, int64_t nv, float *__restrict__ db)
{
    pdl_begin();
    extern __shared__ float sbuf[];
    for (int k = threadIdx.x; k < c; k += blockDim.x) sbuf[k] = 0.0f;
    __syncthreads();
    const int64_t total = nv * c;
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float s = 0.0f;
    for (int64_t e = first; e < total; e += (int64_t)gridDim.x * blockDim.x) s += __bfloat162float(dy[e]);
    atomicAdd(&sbuf[first % c], s);
    __syncthreads();
    for (int k = threadIdx.x; k < c; k += blockDim.x) atomicAdd(db + k, sbuf[k]);
}

// 2^3 average pooling, channels-last; fine extent 2^lgf
__global__ void k_pool(const __nv_bfloat16 *__restrict__ x, int c, int cstride, int lgf, __nv_bfloat16 *__restrict__ y)
{
    pdl_begin();
    const int lgc = lgf - 1, mc = (1 << lgc) - 1;
    const int64_t total = ((int64_t)1 << (3 * lgc)) * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int V = (int)(e / c);
        const int K = V & mc, J = (V >> lgc) & mc, I = V >> (2 * lgc);
        float s = 0.0f;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int k = 0; k < 2; k++) {
                    const int v = ((((2 * I + a) << lgf) + 2 * J + b) << lgf) + 2 * K + k;
                    s += __bfloat162float(x[(size_t)v * cstride + ch]);
                }
        y[e] = __float2bfloat16(0.125f * s);
    }
}

// adjoint of k_pool: dx[v][ch] (+)= dy[parent][ch] / 8 (into a strided slice)
__global__ void k_pool_back(const __nv_bfloat16 *__restrict__ dy, int c, int lgf, __nv_bfloat16 *__restrict__ dx,
                            int cstride, int accumulate)
{
    pdl_begin();
    const int mf = (1 << lgf) - 1, lgc = lgf - 1;
    const int64_t total = ((int64_t)1 << (3 * lgf)) * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int v = (int)(e / c);
        const int k = v & mf, j = (v >> lgf) & mf, i = v >> (2 * lgf);
        const int V = ((((i >> 1) << lgc) + (j >> 1)) << lgc) + (k >> 1);
        float g = 0.125f * __bfloat162float(dy[(size_t)V * c + ch]);
        __nv_bfloat16 *o = dx + (size_t)v * cstride + ch;
        if (accumulate) g += __bfloat162float(*o);
        *o = __float2bfloat16(g);
    }
}

// cell-centred trilinear x2 upsampling (weights 3/4, 1/4 per axis) into
// channels [0, c) of a buffer with channel stride cstride
__global__ void k_upsample(const __nv_bfloat16 *__restrict__ x, int c, int lgc, __nv_bfloat16 *__restrict__ y,
                           int cstride)
{
    pdl_begin();
    const int lgf = lgc + 1, mf = (1 << lgf) - 1, mc = (1 << lgc) - 1;
    const int64_t total = ((int64_t)1 << (3 * lgf)) * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int v = (int)(e / c);
        const int k = v & mf, j = (v >> lgf) & mf, i = v >> (2 * lgf);
        int I[2], J[2], K[2];
        I[0] = i >> 1;
        I[1] = (i & 1) ? ((I[0] + 1) & mc) : ((I[0] - 1) & mc);
        J[0] = j >> 1;
        J[1] = (j & 1) ? ((J[0] + 1) & mc) : ((J[0] - 1) & mc);
        K[0] = k >> 1;
        K[1] = (k & 1) ? ((K[0] + 1) & mc) : ((K[0] - 1) & mc);
        const float wt[2] = {0.75f, 0.25f};
        float s = 0.0f;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int q = 0; q < 2; q++)
                    s += wt[a] * wt[b] * wt[q] *
                         __bfloat162float(x[(size_t)((((I[a] << lgc) + J[b]) << lgc) + K[q]) * c + ch]);
        y[(size_t)v * cstride + ch] = __float2bfloat16(s);
    }
}

// adjoint of k_upsample: per axis coarse J gathers fine 2J-1 (1/4), 2J (3/4),
// 2J+1 (3/4), 2J+2 (1/4); dy read from channels [0, c) of stride cstride
__global__ void k_upsample_back(const __nv_bfloat16 *__restrict__ dy, int c, int cstride, int lgc,
                                __nv_bfloat16 *__restrict__ dx)
{
    pdl_begin();
    const int lgf = lgc + 1, mf = (1 << lgf) - 1, mc = (1 << lgc) - 1;
    const int64_t total = ((int64_t)1 << (3 * lgc)) * c;
    const float wt[4] = {0.25f, 0.75f, 0.75f, 0.25f};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int V = (int)(e / c);
        const int K = V & mc, J = (V >> lgc) & mc, I = V >> (2 * lgc);
        float s = 0.0f;
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++)
                for (int q = 0; q < 4; q++) {
                    const int i = (2 * I - 1 + a) & mf, j = (2 * J - 1 + b) & mf, k = (2 * K - 1 + q) & mf;
                    s += wt[a] * wt[b] * wt[q] * __bfloat162float(dy[(size_t)((((i << lgf) + j) << lgf) + k) * cstride + ch]);
                }
        dx[e] = __float2bfloat16(s);
    }
}

// y[v][off + ch] = x[v][ch] (copy into a channel slice); back: the reverse
__global__ void k_copy_slice(const __nv_bfloat16 *__restrict__ x, int c, int xs, int xoff, __nv_bfloat16 *__restrict__ y,
                             int ys, int yoff, int64_t nv, int accumulate)
{
    pdl_begin();
    const int64_t total = nv * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int64_t v = e / c;
        float val = __bfloat162float(x[v * xs + xoff + ch]);
        __nv_bfloat16 *o = y + v * ys + yoff + ch;
        if (accumulate) val += __bfloat162float(*o);
        *o = __float2bfloat16(val);
    }
}

// g *= (a > 0) elementwise (ReLU backward where the gradient was summed first)
__global__ void k_relu_mask(__nv_bfloat16 *__restrict__ gbuf, const __nv_bfloat16 *__restrict__ a, int64_t total)
{
    pdl_begin();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(a[e]) > 0.0f)) gbuf[e] = __float2bfloat16(0.0f);
}

// Eight channels per thread (c and the channel strides and offsets multiples
// of 8, 16-byte aligned rows): the same per-channel arithmetic as k_upsample
// and k_copy_slice with 16-byte loads and stores and the weights and indices
// formed once per eight channels.
__device__ __forceinline__ void bf8_unpack(uint4 r, float f[8])
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&r);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const float2 t = __bfloat1622float2(h[m]);
        f[2 * m] = t.x, f[2 * m + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 bf8_pack(const float f[8])
{
    uint4 r;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&r);
#pragma unroll
    for (int m = 0; m < 4; m++) h[m] = __floats2bfloat162_rn(f[2 * m], f[2 * m + 1]);
    return r;
}

__global__ void k_upsample8(const __nv_bfloat16 *__restrict__ x, int lgc8, int lgc, __nv_bfloat16 *__restrict__ y,
                            int cstride)
{
    pdl_begin();
    const int lgf = lgc + 1, mf = (1 << lgf) - 1, mc = (1 << lgc) - 1, c = 8 << lgc8;
    const int total = 1 << (3 * lgf + lgc8);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int ch = (e & ((1 << lgc8) - 1)) << 3;
        const int v = e >> lgc8;
        const int k = v & mf, j = (v >> lgf) & mf, i = v >> (2 * lgf);
        int I[2], J[2], K[2];
        I[0] = i >> 1;
        I[1] = (i & 1) ? ((I[0] + 1) & mc) : ((I[0] - 1) & mc);
        J[0] = j >> 1;
        J[1] = (j & 1) ? ((J[0] + 1) & mc) : ((J[0] - 1) & mc);
        K[0] = k >> 1;
        K[1] = (k & 1) ? ((K[0] + 1) & mc) : ((K[0] - 1) & mc);
        const float wt[2] = {0.75f, 0.25f};
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++)
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const float w = wt[a] * wt[b] * wt[q];
                    float xv[8];
                    bf8_unpack(*reinterpret_cast<const uint4 *>(x + (size_t)((((I[a] << lgc) + J[b]) << lgc) + K[q]) * c + ch), xv);
#pragma unroll
                    for (int m = 0; m < 8; m++) s[m] += w * xv[m];
                }
        *reinterpret_cast<uint4 *>(y + (size_t)v * cstride + ch) = bf8_pack(s);
    }
}

__global__ void k_copy_slice8(const __nv_bfloat16 *__restrict__ x, int lgc8, int xs, int xoff,
                              __nv_bfloat16 *__restrict__ y, int ys, int yoff, int nv, int accumulate)
{
    pdl_begin();
    const int total = nv << lgc8;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int ch = (e & ((1 << lgc8) - 1)) << 3;
        const int v = e >> lgc8;
        float val[8];
        bf8_unpack(*reinterpret_cast<const uint4 *>(x + (size_t)v * xs + xoff + ch), val);
        uint4 *o = reinterpret_cast<uint4 *>(y + (size_t)v * ys + yoff + ch);
        if (accumulate) {
            float prev[8];
            bf8_unpack(*o, prev);
#pragma unroll
            for (int m = 0; m < 8; m++) val[m] += prev[m];
        }
        *o = bf8_pack(val);
    }
}

// ---------------------------------------------------------------- input, head, loss
// x[v][0..15]: standardised log(eps + s0/rho), s_i/(rho v_rms), zeros; from natural-layout sources
__global__ void k_net_input(const double *__restrict__ s0, const double *__restrict__ sx, const double *__restrict__ sy,
                            const double *__restrict__ sz, int64_t nv, float inv_rho, float inv_rv,
                            const float *__restrict__ in_mean, const float *__restrict__ in_std,
                            __nv_bfloat16 *__restrict__ x)
{
    pdl_begin();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        float f[4];
        f[0] = logf(kNetLogEps + (float)s0[v] * inv_rho);
        f[1] = (float)sx[v] * inv_rv;
        f[2] = (float)sy[v] * inv_rv;
        f[3] = (float)sz[v] * inv_rv;
        // the voxel's 16 channels (4 used, 12 zero) as two 16-byte stores
        float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < 4; c++) g[c] = (f[c] - in_mean[c]) / in_std[c];
        static_assert(kNetCin == 16, "two 8-channel vectors per voxel");
        uint4 *o = reinterpret_cast<uint4 *>(x + v * kNetCin);
        o[0] = bf8_pack(g);
        o[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// 1x1 head (FP32): out[v][o] = b[o] + sum_c W[o][c] a[v][c], a with 16 channels
__global__ void k_head(const __nv_bfloat16 *__restrict__ a, const float *__restrict__ W, const float *__restrict__ b,
                       int64_t nv, float *__restrict__ out)
{
    pdl_begin();
    __shared__ float sw[kNetOut * 16 + kNetOut];
    for (int k = threadIdx.x; k < kNetOut * 16; k += blockDim.x) sw[k] = W[k];
    for (int k = threadIdx.x; k < kNetOut; k += blockDim.x) sw[kNetOut * 16 + k] = b[k];
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        float av[16];
        for (int c = 0; c < 16; c++) av[c] = __bfloat162float(a[v * 16 + c]);
        for (int o = 0; o < kNetOut; o++) {
            float s = sw[kNetOut * 16 + o];
            for (int c = 0; c < 16; c++) s += sw[o * 16 + c] * av[c];
            out[v * kNetOut + o] = s;
        }
    }
}

// loss and head backward: standardised target t[v][o]; dout = 2 (out - t) / (nv * 10);
// da[v][c] = (a > 0) sum_o W[o][c] dout[v][o]; dW, db accumulated; loss partial per block
__global__ void k_head_back(const __nv_bfloat16 *__restrict__ a, const float *__restrict__ W,
                            const float *__restrict__ out, const float *__restrict__ tgt, int64_t nv,
                            __nv_bfloat16 *__restrict__ da, float *__restrict__ dW, float *__restrict__ db,
                            float *__restrict__ loss)
{
    pdl_begin();
    __shared__ float sw[kNetOut * 16], sdw[kNetOut * 16], sdb[kNetOut], sl[1];
    for (int k = threadIdx.x; k < kNetOut * 16; k += blockDim.x) {
        sw[k] = W[k];
        sdw[k] = 0.0f;
    }
    for (int k = threadIdx.x; k < kNetOut; k += blockDim.x) sdb[k] = 0.0f;
    if (threadIdx.x == 0) sl[0] = 0.0f;
    __syncthreads();
    const float scale = 2.0f / ((float)nv * kNetOut);
    float lsum = 0.0f;
    float ldw[kNetOut * 16];
    float ldb[kNetOut];
    for (int k = 0; k < kNetOut * 16; k++) ldw[k] = 0.0f;
    for (int k = 0; k < kNetOut; k++) ldb[k] = 0.0f;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        float av[16], g[16], d[kNetOut];
        for (int c = 0; c < 16; c++) {
            av[c] = __bfloat162float(a[v * 16 + c]);
            g[c] = 0.0f;
        }
        for (int o = 0; o < kNetOut; o++) {
            const float r = out[v * kNetOut + o] - tgt[v * kNetOut + o];
            lsum += r * r;
            d[o] = scale * r;
            ldb[o] += d[o];
            for (int c = 0; c < 16; c++) {
                ldw[o * 16 + c] += d[o] * av[c];
                g[c] += sw[o * 16 + c] * d[o];
            }
        }
        for (int c = 0; c < 16; c++) da[v * 16 + c] = __float2bfloat16(av[c] > 0.0f ? g[c] : 0.0f);
    }
    for (int k = 0; k < kNetOut * 16; k++) atomicAdd(&sdw[k], ldw[k]);
    for (int k = 0; k < kNetOut; k++) atomicAdd(&sdb[k], ldb[k]);
    atomicAdd(&sl[0], lsum);
    __syncthreads();
    for (int k = threadIdx.x; k < kNetOut * 16; k += blockDim.x) atomicAdd(dW + k, sdw[k]);
    for (int k = threadIdx.x; k < kNetOut; k += blockDim.x) atomicAdd(db + k, sdb[k]);
    if (threadIdx.x == 0) atomicAdd(loss, sl[0] / ((float)nv * kNetOut));
}

// standardised target from natural-layout fields (psi, apsi as deviations)
__global__ void k_net_target(FieldPtrs fields, int64_t nv, const float *__restrict__ mean,
                             const float *__restrict__ stdv, float *__restrict__ tgt)
{
    pdl_begin();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x)
        for (int o = 0; o < kNetOut; o++) {
            double val = fields.p[o][v];
            if (o < 2) val -= 1.0;
            tgt[v * kNetOut + o] = (float)((val - mean[o]) / stdv[o]);
        }
}

// de-standardised output into the fields (psi, apsi get + 1)
__global__ void k_net_output(const float *__restrict__ out, int64_t nv, const float *__restrict__ mean,
                             const float *__restrict__ stdv, FieldPtrs fields)
{
    pdl_begin();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x)
        {
            const float2 *o2 = reinterpret_cast<const float2 *>(out + v * kNetOut);
            float ov[kNetOut];
#pragma unroll
            for (int o = 0; o < kNetOut / 2; o++) {
                const float2 t2 = o2[o];
                ov[2 * o] = t2.x, ov[2 * o + 1] = t2.y;
            }
#pragma unroll
            for (int o = 0; o < kNetOut; o++) {
                // FP32 de-standardisation as in k_net_output_fine (the guess carries BF16 accuracy),
                // so only the conversion and psi's and alpha psi's + 1 use the narrow FP64 pipe
                const double val = (double)(ov[o] * stdv[o] + mean[o]);
                fields.p[o][v] = o < 2 ? val + 1.0 : val;
            }
        }
}

// ---------------------------------------------------------------- guesses on finer grids
// Sources of a fine grid (extent nc << lr) averaged over the r^3 cells each
// coarse cell covers (r = 2^lr), FP64; one thread per coarse cell and array.
__global__ void __launch_bounds__(256)
    k_avg_down(FieldPtrs in, FieldPtrs out, int narr, int lgc, int lr)
{
    pdl_begin();
    const int64_t nvc = (int64_t)1 << (3 * lgc);
    const int lgf = lgc + lr, r = 1 << lr;
    const double inv = 1.0 / (double)((int64_t)1 << (3 * lr));
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nvc * narr;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t >> (3 * lgc));
        const int64_t v = t & (nvc - 1);
        const int64_t mc = ((int64_t)1 << lgc) - 1;
        const int64_t K = v & mc, J = (v >> lgc) & mc, I = v >> (2 * lgc);
        const double *f = in.p[a];
        double acc = 0.0;
        for (int di = 0; di < r; di++)
            for (int dj = 0; dj < r; dj++) {
                const int64_t row = ((((I << lr) + di) << lgf) + ((J << lr) + dj)) << lgf;
                for (int dk = 0; dk < r; dk++) acc += f[row + (K << lr) + dk];
            }
        out.p[a][v] = acc * inv;
    }
}

// The network's standardised output [vc][10] on the coarse grid, interpolated
// trilinearly between periodic coarse cell centres to every cell of the fine
// grid (extent nc << lr) and de-standardised (psi and alpha psi get their 1
// back): FP32 arithmetic, FP64 stores.  One thread per fine cell.
__global__ void __launch_bounds__(256)
    k_net_output_fine(const float *__restrict__ out, int lgc, int lr, const float *__restrict__ mean,
                      const float *__restrict__ stdv, FieldPtrs fields)
{
    pdl_begin();
    const int lgf = lgc + lr;
    const int64_t nvf = (int64_t)1 << (3 * lgf);
    const int mc = (1 << lgc) - 1, mf = (1 << lgf) - 1;
    const float r = (float)(1 << lr);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nvf; t += (int64_t)gridDim.x * blockDim.x) {
        const int idx[3] = {(int)(t >> (2 * lgf)), (int)((t >> lgf) & mf), (int)(t & mf)};
        int lo[3];
        float w1[3];
        for (int d = 0; d < 3; d++) {  // coarse position of the fine cell centre, in coarse cells
            const float c = ((float)idx[d] + 0.5f) / r - 0.5f;
            const float fl = floorf(c);
            w1[d] = c - fl;
            lo[d] = ((int)fl) & mc;
        }
        float acc[kNetOut];
        for (int o = 0; o < kNetOut; o++) acc[o] = 0.0f;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int c = 0; c < 2; c++) {
                    const float w = (a ? w1[0] : 1.0f - w1[0]) * (b ? w1[1] : 1.0f - w1[1]) *
                                    (c ? w1[2] : 1.0f - w1[2]);
                    const int64_t v = ((((int64_t)((lo[0] + a) & mc) << lgc) + ((lo[1] + b) & mc)) << lgc) +
                                      ((lo[2] + c) & mc);
                    const float *rec = out + v * kNetOut;
                    for (int o = 0; o < kNetOut; o++) acc[o] = fmaf(w, rec[o], acc[o]);
                }
        for (int o = 0; o < kNetOut; o++) {
            const double val = (double)(acc[o] * stdv[o] + mean[o]);
            fields.p[o][t] = o < 2 ? val + 1.0 : val;
        }
    }
}

// ---------------------------------------------------------------- optimiser
// Adam (Kingma & Ba 2015) on FP32 master weights; bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ gr, int64_t cnt, float lr, float b1, float b2, float eps, float bc1,
                       float bc2)
{
    pdl_begin();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        const float g = gr[e];
        const float mm = b1 * m[e] + (1.0f - b1) * g;
        const float vv = b2 * v[e] + (1.0f - b2) * g * g;
        m[e] = mm;
        v[e] = vv;
        w[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

// BF16 copies of one conv's FP32 weights: wb[tap][co][ci] and the data-gradient
// copy wt[26 - tap][ci][co]
__global__ void k_conv_weights_bf16(const float *__restrict__ w, int cout, int cin, __nv_bfloat16 *__restrict__ wb,
                                    __nv_bfloat16 *__restrict__ wt)
{
    pdl_begin();
    const int64_t total = (int64_t)27 * cout * cin;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(e % cin);
        const int co = (int)((e / cin) % cout);
        const int tap = (int)(e / ((int64_t)cin * cout));
        const __nv_bfloat16 b = __float2bfloat16(w[e]);
        wb[e] = b;
        wt[((int64_t)(26 - tap) * cin + ci) * cout + co] = b;
    }
}

}  // namespace

// ================================================================ launchers
void conv3d(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *w, const float *bias, int cout, int lg, int mode,
            const __nv_bfloat16 *mask, __nv_bfloat16 *y, cudaStream_t st)
{
    // 128^3 grids on the 5th-generation tensor cores (conv_tc.cu) unless GR_CONV_TC=0
    const char *env = getenv("GR_CONV_TC");
    if ((!env || env[0] != '0') && conv3d_tc_fits(cin, cout, lg)) {
        conv3d_tc(x, cin, w, bias, cout, mode, mask, y, st);
        return;
    }
    const int64_t nv = (int64_t)1 << (3 * lg);
    if (cout % 32 == 0) {
        // 4 warps x 32 voxels, 32 channels per block
        dim3 grid(cdiv(nv, 4 * 32), cout / 32);
        GR_LAUNCH((k_conv3d<2, 4>), grid, 128, st, x, cin, w, bias, cout, lg, mode, mask, y);
    } else {
        dim3 grid(cdiv(nv, 4 * 64), cout / 16);
        GR_LAUNCH((k_conv3d<4, 2>), grid, 128, st, x, cin, w, bias, cout, lg, mode, mask, y);
    }
}

void conv3d_wgrad(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *dy, int cout, int lg, float *dw,
                  cudaStream_t st)
{
    const int64_t nv = (int64_t)1 << (3 * lg);
    int chunk = 2048;
    while (chunk > 64 && nv / chunk < 64) chunk >>= 1;
    if (nv < chunk) chunk = (int)nv;
    if (cin % 32 == 0) {
        dim3 grid((unsigned)(nv / chunk), 27, (cout / 16) * (cin / 32));
        GR_LAUNCH((k_conv3d_wgrad<4>), grid, 128, st, x, cin, dy, cout, lg, chunk, dw);
    } else {
        dim3 grid((unsigned)(nv / chunk), 27, (cout / 16) * (cin / 16));
        GR_LAUNCH((k_conv3d_wgrad<2>), grid, 128, st, x, cin, dy, cout, lg, chunk, dw);
    }
}

void bias_grad(const __nv_bfloat16 *dy, int c, int64_t nv, float *db, cudaStream_t st)
{
    GR_LAUNCH_SMEM(k_bias_grad, kBiasBlocks, 256, c * sizeof(float), st, dy, c, nv, db);
}

void pool(const __nv_bfloat16 *x, int c, int cstride, int lgf, __nv_bfloat16 *y, cudaStream_t st)
{
    GR_LAUNCH(k_pool, cdiv(((int64_t)1 << (3 * lgf - 3)) * c, 256), 256, st, x, c, cstride, lgf, y);
}

void pool_back(const __nv_bfloat16 *dy, int c, int lgf, __nv_bfloat16 *dx, int cstride, int accumulate, cudaStream_t st)
{
    GR_LAUNCH(k_pool_back, cdiv(((int64_t)1 << (3 * lgf)) * c, 256), 256, st, dy, c, lgf, dx, cstride, accumulate);
}

// exponent of a power of two, -1 otherwise
static int pow2_log(int c)
{
    if (c <= 0 || (c & (c - 1))) return -1;
    int l = 0;
    while ((1 << l) < c) ++l;
    return l;
}

void upsample(const __nv_bfloat16 *x, int c, int lgc, __nv_bfloat16 *y, int cstride, cudaStream_t st)
{
    const int l8 = pow2_log(c) - 3;
    if (l8 >= 0 && cstride % 8 == 0 && 3 * lgc + 3 + l8 < 31) {
        GR_LAUNCH(k_upsample8, cdiv((int64_t)1 << (3 * lgc + 3 + l8), 256), 256, st, x, l8, lgc, y, cstride);
        return;
    }
    GR_LAUNCH(k_upsample, cdiv(((int64_t)1 << (3 * lgc + 3)) * c, 256), 256, st, x, c, lgc, y, cstride);
}

void upsample_back(const __nv_bfloat16 *dy, int c, int cstride, int lgc, __nv_bfloat16 *dx, cudaStream_t st)
{
    GR_LAUNCH(k_upsample_back, cdiv(((int64_t)1 << (3 * lgc)) * c, 256), 256, st, dy, c, cstride, lgc, dx);
}

void copy_slice(const __nv_bfloat16 *x, int c, int xs, int xoff, __nv_bfloat16 *y, int ys, int yoff, int64_t nv,
                int accumulate, cudaStream_t st)
{
    const int l8 = pow2_log(c) - 3;
    if (l8 >= 0 && xs % 8 == 0 && ys % 8 == 0 && xoff % 8 == 0 && yoff % 8 == 0 && (nv << l8) < (1LL << 31)) {
        GR_LAUNCH(k_copy_slice8, cdiv(nv << l8, 256), 256, st, x, l8, xs, xoff, y, ys, yoff, (int)nv, accumulate);
        return;
    }
    GR_LAUNCH(k_copy_slice, cdiv(nv * c, 256), 256, st, x, c, xs, xoff, y, ys, yoff, nv, accumulate);
}

void relu_mask(__nv_bfloat16 *g, const __nv_bfloat16 *a, int64_t total, cudaStream_t st)
{
    GR_LAUNCH(k_relu_mask, cdiv(total, 256), 256, st, g, a, total);
}

void net_input(const double *s0, const double *sx, const double *sy, const double *sz, int64_t nv, float inv_rho,
               float inv_rv, const float *in_mean, const float *in_std, __nv_bfloat16 *x, cudaStream_t st)
{
    GR_LAUNCH(k_net_input, cdiv(nv, 256), 256, st, s0, sx, sy, sz, nv, inv_rho, inv_rv, in_mean, in_std, x);
}

void avg_down(FieldPtrs in, FieldPtrs out, int narr, int lgc, int lr, cudaStream_t st)
{
    const int64_t tot = ((int64_t)narr) << (3 * lgc);
    GR_LAUNCH(k_avg_down, cdiv(tot, 256), 256, st, in, out, narr, lgc, lr);
}

void net_output_fine(const float *out, int lgc, int lr, const float *mean, const float *stdv, FieldPtrs fields,
                     cudaStream_t st)
{
    const int64_t nvf = (int64_t)1 << (3 * (lgc + lr));
    GR_LAUNCH(k_net_output_fine, wave_grid(k_net_output_fine, nvf), 256, st, out, lgc, lr, mean, stdv, fields);
}

void head(const __nv_bfloat16 *a, const float *W, const float *b, int64_t nv, float *out, cudaStream_t st)
{
    GR_LAUNCH(k_head, cdiv(nv, 256), 256, st, a, W, b, nv, out);
}

void head_back(const __nv_bfloat16 *a, const float *W, const float *out, const float *tgt, int64_t nv,
               __nv_bfloat16 *da, float *dW, float *db, float *loss, cudaStream_t st)
{
    GR_LAUNCH(k_head_back, 152 * 4, 128, st, a, W, out, tgt, nv, da, dW, db, loss);
}

void net_target(FieldPtrs fields, int64_t nv, const float *mean, const float *stdv, float *tgt, cudaStream_t st)
{
    GR_LAUNCH(k_net_target, cdiv(nv, 256), 256, st, fields, nv, mean, stdv, tgt);
}

void net_output(const float *out, int64_t nv, const float *mean, const float *stdv, FieldPtrs fields,
                cudaStream_t st)
{
    GR_LAUNCH(k_net_output, cdiv(nv, 256), 256, st, out, nv, mean, stdv, fields);
}

void adam(float *w, float *m, float *v, const float *g, int64_t cnt, float lr, float b1, float b2, float eps,
          float bc1, float bc2, cudaStream_t st)
{
    GR_LAUNCH(k_adam, cdiv(cnt, 256) > 4096 ? 4096 : cdiv(cnt, 256), 256, st, w, m, v, g, cnt, lr, b1, b2, eps, bc1,
              bc2);
}

void conv_weights_bf16(const float *w, int cout, int cin, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t st)
{
    const int64_t total = (int64_t)27 * cout * cin;
    GR_LAUNCH(k_conv_weights_bf16, cdiv(total, 256) > 4096 ? 4096 : cdiv(total, 256), 256, st, w, cout, cin, wb, wt);
}

}  // namespace gr
