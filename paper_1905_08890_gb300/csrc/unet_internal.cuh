// unet_internal.cuh - shared definitions of the U-Net kernels (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace gr {

constexpr int kNetCin = 16;         // input channels after zero padding (4 used)
constexpr int kNetOut = 10;         // psi - 1, alpha psi - 1, V_x, V_y, V_z, U, B^x, B^y, B^z, b
constexpr float kNetLogEps = 0.01f; // input channel 0: log(eps + s0 / rho_hat)

enum ConvMode : int { CONV_RELU = 0, CONV_MASK = 1, CONV_PLAIN = 2 };

struct FieldPtrs {
    double *p[kNetOut];
};

void conv3d(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *w, const float *bias, int cout, int lg, int mode,
            const __nv_bfloat16 *mask, __nv_bfloat16 *y, cudaStream_t st);
// the same convolution on tcgen05 (conv_tc.cu) for the cases conv3d_tc_fits
// accepts (128^3 voxels, 16 input channels, cout 16, 32, 48 or 64);
// conv3d_tc_error: synchronises st; nonzero once a bounded wait of that kernel ran out
bool conv3d_tc_fits(int cin, int cout, int lg);
void conv3d_tc(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *w, const float *bias, int cout, int mode,
               const __nv_bfloat16 *mask, __nv_bfloat16 *y, cudaStream_t st);
int conv3d_tc_error(cudaStream_t st);
void conv3d_wgrad(const __nv_bfloat16 *x, int cin, const __nv_bfloat16 *dy, int cout, int lg, float *dw,
                  cudaStream_t st);
void bias_grad(const __nv_bfloat16 *dy, int c, int64_t nv, float *db, cudaStream_t st);
void pool(const __nv_bfloat16 *x, int c, int cstride, int lgf, __nv_bfloat16 *y, cudaStream_t st);
void pool_back(const __nv_bfloat16 *dy, int c, int lgf, __nv_bfloat16 *dx, int cstride, int accumulate,
               cudaStream_t st);
void upsample(const __nv_bfloat16 *x, int c, int lgc, __nv_bfloat16 *y, int cstride, cudaStream_t st);
void upsample_back(const __nv_bfloat16 *dy, int c, int cstride, int lgc, __nv_bfloat16 *dx, cudaStream_t st);
void copy_slice(const __nv_bfloat16 *x, int c, int xs, int xoff, __nv_bfloat16 *y, int ys, int yoff, int64_t nv,
                int accumulate, cudaStream_t st);
void relu_mask(__nv_bfloat16 *g, const __nv_bfloat16 *a, int64_t total, cudaStream_t st);
void net_input(const double *s0, const double *sx, const double *sy, const double *sz, int64_t nv, float inv_rho,
               float inv_rv, const float *in_mean, const float *in_std, __nv_bfloat16 *x, cudaStream_t st);
void head(const __nv_bfloat16 *a, const float *W, const float *b, int64_t nv, float *out, cudaStream_t st);
void head_back(const __nv_bfloat16 *a, const float *W, const float *out, const float *tgt, int64_t nv,
               __nv_bfloat16 *da, float *dW, float *db, float *loss, cudaStream_t st);
void net_target(FieldPtrs fields, int64_t nv, const float *mean, const float *stdv, float *tgt, cudaStream_t st);
void net_output(const float *out, int64_t nv, const float *mean, const float *stdv, FieldPtrs fields,
                cudaStream_t st);
// the first narr arrays of in (fine, extent 2^(lgc + lr)) averaged over r^3 blocks into out (extent 2^lgc)
void avg_down(FieldPtrs in, FieldPtrs out, int narr, int lgc, int lr, cudaStream_t st);
// the network output on the 2^lgc grid interpolated to the 2^(lgc + lr) grid as the ten fields
void net_output_fine(const float *out, int lgc, int lr, const float *mean, const float *stdv, FieldPtrs fields,
                     cudaStream_t st);
void adam(float *w, float *m, float *v, const float *g, int64_t cnt, float lr, float b1, float b2, float eps,
          float bc1, float bc2, cudaStream_t st);
void conv_weights_bf16(const float *w, int cout, int cin, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t st);

}  // namespace gr
