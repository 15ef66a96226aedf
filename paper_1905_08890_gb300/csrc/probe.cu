// probe.cu - FMA issue rate of the GPU in FP64 and FP32 (a diagnostic, not
// part of the method).  The ALU-bound rooflines of this library (the particle
// update, the FP64 colour passes, the double-float set-up) are stated against
// these measured rates beside the rates from unit counts and clock.
#include <cuda_runtime.h>

#include "gr.h"
#include "gr_internal.cuh"

namespace gr {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// kChains dependent chains of `iters` FMAs each per thread; the chains'
// values are written out so that no FMA is dead
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(long long iters, T a, T b, T *out)
{
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = T(threadIdx.x + c) * T(1e-3);
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) v[c] = v[c] * a + b;
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; c++) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
gr_status run(long long iters, cudaStream_t st, double *flops)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (sms > 0 ? sms : 1) * 8, threads = 256;
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) {
        cudaGetLastError();
        return GR_ERR_NOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a = 1 - 2^-20, b = 2^-20: the chains stay near 1, finite and normal
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0);
    k_fma_chains<T><<<blocks, threads, 0, st>>>(iters / 16 + 1, a, b, out);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, threads, 0, st>>>(iters, a, b, out);
    cudaEventRecord(e1, st);
    g_launches.fetch_add(2, std::memory_order_relaxed);
    const cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || !(ms > 0.f)) {
        cudaGetLastError();
        return GR_ERR_CUDA;
    }
    *flops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3);
    return GR_OK;
}

}  // namespace
}  // namespace gr

extern "C" gr_status gr_fma_rate(int fp64, long long iters, void *cuda_stream, double *flops_per_s)
{
    if (!flops_per_s || iters < 1 || iters > (1LL << 32)) return GR_ERR_ARG;
    *flops_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return fp64 ? gr::run<double>(iters, st, flops_per_s) : gr::run<float>(iters, st, flops_per_s);
}
