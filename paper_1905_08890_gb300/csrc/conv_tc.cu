// conv_tc.cu - the U-Net's circular 3^3 convolution on the 5th-generation
// tensor cores (tcgen05.mma, FP32 accumulator in tensor memory), for grids of
// 128^3 voxels (rows of exactly 128 voxels: the network's finest level, where
// two thirds of its arithmetic sits) with 16 or 48 input channels.
//
// Implicit GEMM per output row (d, h): D[128 voxels w][N = cout] = sum over
// taps (dd, dh, dw) of A[w][k] = x[(d + dd, h + dh, w + dw)][k] times
// B[k][n] = W[tap][n][k] (input channels k, 16 per MMA).  The input rows
// (d + dd, h + dh) are staged in shared memory in the canonical no-swizzle
// K-major layout of the tensor core (core matrices of 8 voxels x 16 bytes;
// plane p holds channels 8p .. 8p + 7 of every voxel), with one wrapped halo
// voxel on each side, so the A operand of tap dw is the same row read from a
// start address 16 (dw + 1) bytes further on, and that of channel chunk c two
// planes further on: the 27 cin/16 MMAs of a row read their operands straight
// from shared memory, with no per-tap copy.  A block takes
// a contiguous range of output rows and rolls the staged rows along h (three
// new input rows per output row, copied asynchronously one row ahead).  The
// weights of all taps sit in shared memory for the whole (persistent) block.  One thread issues
// the MMAs; tcgen05.commit signals an mbarrier when they have finished, after
// which the block reads the accumulator back with tcgen05.ld (thread t of the
// four warps owns tensor-memory lane t = output voxel w) for the epilogue
// (bias and ReLU, or the ReLU mask of the data gradient), writing BF16.
//
// Every wait on the mbarrier is bounded; a wait that runs out sets g_conv_tc_err
// and the block goes on to release its tensor memory and return.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include <mutex>

#include "gr_internal.cuh"
#include "unet_internal.cuh"

namespace gr {

__device__ int g_conv_tc_err = 0;

namespace {

constexpr int kRowVox = 128;                 // voxels per output row (= MMA M)
constexpr int kHaloVox = kRowVox + 2;        // staged voxels per input row
constexpr int kPlaneB = kHaloVox * 16;       // bytes of one 8-channel plane of one staged row (2080)

// dynamic shared memory: mbarrier and tensor-memory slot, the weights of every
// tap and 16-channel chunk, and four rolling slots of the three rows d + dd
// (cin / 8 planes each)
constexpr size_t tc_smem(int cin, int cout)
{
    return 128 + (size_t)27 * (cin / 16) * cout * 32 + (size_t)12 * (cin / 8) * kPlaneB;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: no swizzle, K-major; start, leading
// (K-direction core-matrix) and stride (M/N-direction 8-row group) byte offsets
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
    return d;                // base offset 0, swizzle none
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRowVox >> 4) << 24);
}

__device__ __forceinline__ void mma_tc(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(id), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// bounded wait for the completion of phase `parity` of the mbarrier
__device__ __forceinline__ void mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return;
    }
    atomicExch(&g_conv_tc_err, 1);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(hi)) << 16);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// x: [128^3][cin] BF16, w: [27][N][cin] BF16, bias [N] (CONV_RELU), mask
// [128^3][N] (CONV_MASK), y: [128^3][N] BF16; N = cout (16..64, multiple of
// 16), cin a multiple of 16.  Dynamic shared memory: tc_smem(cin, N) bytes;
// several blocks per SM (where it fits) overlap one another's copies, MMAs
// and epilogues.
template <int N>
__global__ void __launch_bounds__(128, 1)
    k_conv3d_tc(const __nv_bfloat16 *__restrict__ x, int cin, const __nv_bfloat16 *__restrict__ w,
                const float *__restrict__ bias, int mode, const __nv_bfloat16 *__restrict__ mask,
                __nv_bfloat16 *__restrict__ y)
{
    pdl_begin();
    extern __shared__ __align__(128) uint8_t sm[];
    constexpr uint32_t NCOL = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
    const int nch = cin >> 4, planes = cin >> 3, rowB = planes * kPlaneB;
    uint8_t *Bs = sm + 128;
    uint8_t *As = Bs + 27 * nch * N * 32;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar = smem_u32(sm), slot = smem_u32(sm + 16);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const uint32_t as = smem_u32(As), bs = smem_u32(Bs), id = idesc_bf16(N);
    // all taps' and chunks' weights: 16-byte pieces, plane p of row co at
    // Bs + (c 27 + tap) N 32 + p N 16 + co 16
    for (int e = tid; e < 27 * nch * N * 2; e += 128) {
        const int p = e & 1, co = (e >> 1) % N, tc = (e >> 1) / N, tap = tc % 27, c = tc / 27;
        cp16(bs + tc * N * 32 + p * N * 16 + co * 16, w + ((size_t)tap * N + co) * cin + 16 * c + 8 * p);
    }
    cp_commit();
    // Rows of a contiguous range r = 128 d + h, in order: the staged input rows
    // of one d roll along h in four slots per dd (rows h - 1, h, h + 1 in use,
    // h + 2 arriving), so each new output row stages three input rows, not nine.
    const int r_begin = (int)((int64_t)blockIdx.x * kRowVox * kRowVox / gridDim.x);
    const int r_end = (int)((int64_t)(blockIdx.x + 1) * kRowVox * kRowVox / gridDim.x);
    // the three input rows (d + dd, hh) of all dd, with the wrapped halo voxel on each side
    auto issue_rows = [&](int d, int hh) {
        const int sl = (hh + 4) & 3;
        for (int e = tid; e < 3 * kHaloVox * planes; e += 128) {
            const int p = e % planes, hv = (e / planes) % kHaloVox, r = (e / planes) / kHaloVox;  // r = dd + 1
            const int v = (((((d + r - 1) & 127) << 7) + (hh & 127)) << 7) + ((hv - 1) & 127);
            cp16(as + (r * 4 + sl) * rowB + p * kPlaneB + 16 * hv, x + (size_t)v * cin + 8 * p);
        }
    };
    uint32_t phase = 0u;
    fence_before();
    __syncthreads();  // the tensor-memory address written by the allocation is visible
    fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(sm + 16);
    for (int row = r_begin; row < r_end; row++) {
        const int d = row >> 7, h = row & 127;
        if (row == r_begin || h == 0) {  // a new d: stage rows h - 1, h, h + 1
            issue_rows(d, h - 1);
            issue_rows(d, h);
            issue_rows(d, h + 1);
            cp_commit();
        }
        // row h + 2 for the next output row (its slot was last read by the MMAs of row h - 1)
        if (row + 1 < r_end && h + 1 < kRowVox) {
            issue_rows(d, h + 2);
            cp_commit();
            cp_wait<1>();  // everything but that row has landed (this thread's copies)
        } else {
            cp_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            for (int tap = 0; tap < 27; tap++) {
                const int dd = tap / 9, dh = (tap / 3) % 3 - 1, sl = (h + dh + 4) & 3;
                for (int c = 0; c < nch; c++) {
                    const uint64_t ad = sdesc(as + (dd * 4 + sl) * rowB + 16 * (tap % 3) + c * 2 * kPlaneB, kPlaneB, 128);
                    const uint64_t bd = sdesc(bs + (c * 27 + tap) * N * 32, N * 16, 128);
                    mma_tc(tmem, ad, bd, id, (tap > 0 || c > 0) ? 1u : 0u);
                }
            }
            mma_commit(mbar);
        }
        mbar_wait(mbar, phase);
        phase ^= 1u;
        fence_after();
        // epilogue: thread tid holds output voxel w = tid of this row
        const size_t v = ((size_t)row << 7) + tid;
#pragma unroll
        for (int cb = 0; cb < N; cb += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
            float o[16];
#pragma unroll
            for (int k = 0; k < 16; k++) o[k] = __uint_as_float(r[k]);
            if (mode == CONV_RELU) {
#pragma unroll
                for (int k = 0; k < 16; k++) o[k] = fmaxf(o[k] + bias[cb + k], 0.0f);
            } else if (mode == CONV_MASK) {
                const uint4 m0 = *reinterpret_cast<const uint4 *>(mask + v * N + cb);
                const uint4 m1 = *reinterpret_cast<const uint4 *>(mask + v * N + cb + 8);
                const __nv_bfloat16 *mb0 = reinterpret_cast<const __nv_bfloat16 *>(&m0);
                const __nv_bfloat16 *mb1 = reinterpret_cast<const __nv_bfloat16 *>(&m1);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    o[k] = __bfloat162float(mb0[k]) > 0.0f ? o[k] : 0.0f;
                    o[8 + k] = __bfloat162float(mb1[k]) > 0.0f ? o[8 + k] : 0.0f;
                }
            }
            uint4 s0, s1;
            s0.x = pack_bf16(o[0], o[1]);
            s0.y = pack_bf16(o[2], o[3]);
            s0.z = pack_bf16(o[4], o[5]);
            s0.w = pack_bf16(o[6], o[7]);
            s1.x = pack_bf16(o[8], o[9]);
            s1.y = pack_bf16(o[10], o[11]);
            s1.z = pack_bf16(o[12], o[13]);
            s1.w = pack_bf16(o[14], o[15]);
            *reinterpret_cast<uint4 *>(y + v * N + cb) = s0;
            *reinterpret_cast<uint4 *>(y + v * N + cb + 8) = s1;
        }
        // every accumulator read is done before the next row's MMAs overwrite it
        fence_before();
        __syncthreads();
        fence_after();
    }
    cp_wait<0>();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

template <int N>
void launch_tc(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *w, const float *bias, int mode,
               const __nv_bfloat16 *mask, __nv_bfloat16 *y, cudaStream_t st)
{
    const size_t smem = tc_smem(cin, N);
    static int grid_of[16] = {};  // per cin / 16
    static std::mutex mu;         // host threads may launch concurrently
    const int ci = cin / 16;
    std::lock_guard<std::mutex> lock(mu);
    if (!grid_of[ci]) {
        int dev = 0, optin = 0, per_sm = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // the largest request of any cin (conv3d_tc_fits bounds it below the opt-in maximum)
        cudaFuncSetAttribute(k_conv3d_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        // resident blocks: shared memory (1 KB reserved per block), at most 4, and the 512
        // tensor-memory columns (every block holds a power of two >= 32)
        const int ncol = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
        int b = per_sm / (int)(smem + 1024);
        if (b > 4) b = 4;
        if (b * ncol > 512) b = 512 / ncol;
        if (b < 1) b = 1;
        grid_of[ci] = b * (sms > 0 ? sms : 1);
    }
    const int rows = kRowVox * kRowVox;
    const int grid = grid_of[ci] < rows ? grid_of[ci] : rows;
    GR_LAUNCH_SMEM((k_conv3d_tc<N>), grid, 128, smem, st, x, cin, w, bias, mode, mask, y);
}

}  // namespace

bool conv3d_tc_fits(int cin, int cout, int lg)
{
    // 16 input channels, or the decoder's 48 -> 16: one block per SM (191 KB of shared memory), the
    // rolled input rows holding all 48 channels, so a row's three new input rows are staged once; it
    // measured at parity with the mma.sync kernel (701 against 699 us, cold launch list), its 81
    // dependent MMAs per row (N = 16) not overlapped by other blocks.  (An earlier version that staged
    // each 16-channel chunk's nine rows separately took 573 us against 390 us timed alone.)
    if (lg != 7) return false;
    if (cin == 16) return cout == 16 || cout == 32 || cout == 48 || cout == 64;
    return cin == 48 && cout == 16 && tc_smem(cin, cout) <= 227 * 1024;
}

void conv3d_tc(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *w, const float *bias, int cout, int mode,
               const __nv_bfloat16 *mask, __nv_bfloat16 *y, cudaStream_t st)
{
    switch (cout) {
    case 16: launch_tc<16>(x, cin, w, bias, mode, mask, y, st); break;
    case 32: launch_tc<32>(x, cin, w, bias, mode, mask, y, st); break;
    case 48: launch_tc<48>(x, cin, w, bias, mode, mask, y, st); break;
    default: launch_tc<64>(x, cin, w, bias, mode, mask, y, st); break;
    }
}

int conv3d_tc_error(cudaStream_t st)
{
    int e = 0;
    if (cudaMemcpyFromSymbolAsync(&e, g_conv_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -1;
    return e;
}

}  // namespace gr
