// codeunits.cu - the paper's code units (Sec. 4.1) at a fiducial scale
// factor a, mapped onto the a = 1 geometric problem the solver works on.
//
// Code units (box L = 1, c = G = 1, H0 in units of c/L): ct = 1/H0,
// rho_c = 3 H0^2 / (8 pi); sources st = s / (Omega_m rho_c); fields
//   alpha = 1 + Phi / (a^2 ct^2),   psi = a^(1/2) (1 - Psi / (2 a^2 ct^2)),
//   Vt = a ct^2 V,  Ut = a ct^2 U,  Bt = a^2 ct B,  bt = a^2 ct b.
// The geometric equations of Sec. 2.4 at scale factor a (homogeneous density
// rho_hat(a) = Omega_m rho_c a^-3, Kdot = 12 pi rho_hat(a)) are those at
// a = 1 for chi = psi / a^(1/2), phi = alpha chi, V' = V / a^2, U' = U / a^2,
// B' = a B, b' = a b with the sources s0 / a, s_i / a^2, sigma / a^3 and
// rho_hat' = a^2 rho_hat(a); so the code-unit problem becomes an a = 1
// problem whose unknowns chi - 1 and phi - 1 stay small, and the solver's
// deviation form and double-float arithmetic keep their precision at any a.
#include <cuda_runtime.h>

#include "gr_internal.cuh"

namespace gr {

namespace {

// sources: out[k] = scale[k] * in[k]; fields in place: Psi -> chi,
// Phi -> phi = (1 + Phi / a2c2) chi, the potentials scaled by fs[f]
__global__ void __launch_bounds__(kBlock)
    k_cu_in(int64_t N, CuPtrs src_in, CuPtrs src_out, CuScale sc, CuPtrs fld, double a2c2)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 5; k++) src_out.p[k][t] = sc.s[k] * src_in.p[k][t];
        const double chi = 1.0 - fld.p[0][t] / (2.0 * a2c2);
        fld.p[0][t] = chi;
        fld.p[1][t] = (1.0 + fld.p[1][t] / a2c2) * chi;
#pragma unroll
        for (int f = 2; f < 10; f++) fld.p[f][t] *= sc.f[f];
    }
}

// fields back: chi -> Psi = 2 a2c2 (1 - chi), phi -> Phi = a2c2 (phi - chi) / chi,
// the potentials divided by fs[f]
__global__ void __launch_bounds__(kBlock) k_cu_out(int64_t N, CuScale sc, CuPtrs fld, double a2c2)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const double chi = fld.p[0][t], phi = fld.p[1][t];
        fld.p[0][t] = 2.0 * a2c2 * (1.0 - chi);
        fld.p[1][t] = a2c2 * (phi - chi) / chi;
#pragma unroll
        for (int f = 2; f < 10; f++) fld.p[f][t] /= sc.f[f];
    }
}

}  // namespace

void code_units_in(int64_t N, const CuPtrs &src_in, const CuPtrs &src_out, const CuScale &sc, const CuPtrs &fld,
                   double a2c2, cudaStream_t st)
{
    GR_LAUNCH(k_cu_in, wave_grid(k_cu_in, N), kBlock, st, N, src_in, src_out, sc, fld, a2c2);
}

void code_units_out(int64_t N, const CuScale &sc, const CuPtrs &fld, double a2c2, cudaStream_t st)
{
    GR_LAUNCH(k_cu_out, wave_grid(k_cu_out, N), kBlock, st, N, sc, fld, a2c2);
}

}  // namespace gr
