// unet.cu - the learned initial guess: a 3D U-Net (4 levels, 16-32-64-128
// channels, two circular 3^3 convolutions per level and side, 2^3 average
// pooling, trilinear x2 upsampling, concatenated skips, 1x1 head) mapping the
// sources (s0, s_x, s_y, s_z) to the ten fields, trained on the GPU with its
// own forward and backward kernels (unet_kernels.cu) and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "../../include/gr.h"
#include "gr_internal.cuh"
#include "unet_internal.cuh"

using namespace gr;
using bf16 = __nv_bfloat16;

namespace {

struct Conv {
    int cin, cout, lev;   // level 0 = input grid
    size_t w, b;          // offsets of weights [27][cout][cin] and bias [cout] in the FP32 parameters
    size_t wb;            // offset of the BF16 copies (forward and data-gradient layouts)
};

// the 14 convolutions: encoder (0..7), decoder (8..13)
const int kConvSpec[14][3] = {
    {kNetCin, 16, 0}, {16, 16, 0},  {16, 32, 1},  {32, 32, 1}, {32, 64, 2},   {64, 64, 2},  {64, 128, 3},
    {128, 128, 3},    {192, 64, 2}, {64, 64, 2},  {96, 32, 1}, {32, 32, 1},   {48, 16, 0},  {16, 16, 0},
};

gr_status nfail(gr_status s, const char *msg)
{
    gr::set_last_error(msg);
    return s;
}

}  // namespace

struct gr_net {
    int n = 0, lg0 = 0;
    cudaStream_t st = nullptr;
    Conv conv[14];
    size_t nparams = 0, nbf = 0, head_w = 0, head_b = 0;
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    bf16 *wb = nullptr, *wt = nullptr;
    float *norm = nullptr;  // in_mean[4], in_std[4], out_mean[10], out_std[10]
    float hnorm[28];
    int step = 0;
    // activations [v][c] (index = tensor id) and their gradients
    std::vector<bf16 *> act, grad;
    float *out = nullptr, *tgt = nullptr, *loss = nullptr, *hloss = nullptr;
    double *coarse_src = nullptr;  // gr_net_guess: four averaged source arrays (allocated on first use)
    std::vector<void *> allocs;
};

namespace {

enum Tensor {
    T_X0, T_E0A, T_E0B, T_P1, T_E1A, T_E1B, T_P2, T_E2A, T_E2B, T_P3, T_E3A, T_E3B,
    T_CAT2, T_D2A, T_D2B, T_CAT1, T_D1A, T_D1B, T_CAT0, T_D0A, T_D0B, T_NT
};
// (level, channels) of every tensor
const int kTensor[T_NT][2] = {{0, kNetCin}, {0, 16}, {0, 16}, {1, 16}, {1, 32}, {1, 32}, {2, 32},
                              {2, 64},      {2, 64}, {3, 64}, {3, 128}, {3, 128}, {2, 192}, {2, 64},
                              {2, 64},      {1, 96}, {1, 32}, {1, 32},  {0, 48},  {0, 16},  {0, 16}};
// input and output tensor of every convolution
const int kConvIO[14][2] = {{T_X0, T_E0A},   {T_E0A, T_E0B}, {T_P1, T_E1A},  {T_E1A, T_E1B}, {T_P2, T_E2A},
                            {T_E2A, T_E2B},  {T_P3, T_E3A},  {T_E3A, T_E3B}, {T_CAT2, T_D2A}, {T_D2A, T_D2B},
                            {T_CAT1, T_D1A}, {T_D1A, T_D1B}, {T_CAT0, T_D0A}, {T_D0A, T_D0B}};

template <typename T>
bool nalloc(gr_net *net, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) < 256 ? 256 : count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    net->allocs.push_back(q);
    *p = (T *)q;
    return true;
}

int64_t nvox(const gr_net *net, int lev) { return (int64_t)1 << (3 * (net->lg0 - lev)); }

void refresh_bf16(gr_net *net)
{
    for (int k = 0; k < 14; k++) {
        const Conv &c = net->conv[k];
        gr::conv_weights_bf16(net->params + c.w, c.cout, c.cin, net->wb + c.wb, net->wt + c.wb, net->st);
    }
}

FieldPtrs field_ptrs(const gr_fields *f)
{
    FieldPtrs p;
    p.p[0] = f->psi;
    p.p[1] = f->apsi;
    for (int d = 0; d < 3; d++) p.p[2 + d] = f->V[d];
    p.p[5] = f->U;
    for (int d = 0; d < 3; d++) p.p[6 + d] = f->B[d];
    p.p[9] = f->b;
    return p;
}

void forward(gr_net *net, const gr_sources *s, double rho, double vrms)
{
    cudaStream_t st = net->st;
    const int64_t nv0 = nvox(net, 0);
    gr::net_input(s->s0, s->s[0], s->s[1], s->s[2], nv0, (float)(1.0 / rho), (float)(1.0 / (rho * vrms)),
                  net->norm, net->norm + 4, net->act[T_X0], st);
    auto cv = [&](int k) {
        const Conv &c = net->conv[k];
        gr::conv3d(net->act[kConvIO[k][0]], c.cin, net->wb + c.wb, net->params + c.b, c.cout, net->lg0 - c.lev,
                   CONV_RELU, nullptr, net->act[kConvIO[k][1]], st);
    };
    cv(0);
    cv(1);
    gr::pool(net->act[T_E0B], 16, 16, net->lg0, net->act[T_P1], st);
    cv(2);
    cv(3);
    gr::pool(net->act[T_E1B], 32, 32, net->lg0 - 1, net->act[T_P2], st);
    cv(4);
    cv(5);
    gr::pool(net->act[T_E2B], 64, 64, net->lg0 - 2, net->act[T_P3], st);
    cv(6);
    cv(7);
    gr::upsample(net->act[T_E3B], 128, net->lg0 - 3, net->act[T_CAT2], 192, st);
    gr::copy_slice(net->act[T_E2B], 64, 64, 0, net->act[T_CAT2], 192, 128, nvox(net, 2), 0, st);
    cv(8);
    cv(9);
    gr::upsample(net->act[T_D2B], 64, net->lg0 - 2, net->act[T_CAT1], 96, st);
    gr::copy_slice(net->act[T_E1B], 32, 32, 0, net->act[T_CAT1], 96, 64, nvox(net, 1), 0, st);
    cv(10);
    cv(11);
    gr::upsample(net->act[T_D1B], 32, net->lg0 - 1, net->act[T_CAT0], 48, st);
    gr::copy_slice(net->act[T_E0B], 16, 16, 0, net->act[T_CAT0], 48, 32, nv0, 0, st);
    cv(12);
    cv(13);
    gr::head(net->act[T_D0B], net->params + net->head_w, net->params + net->head_b, nv0, net->out, st);
}

// gradient of the loss with respect to every parameter (net->grads), given
// the forward activations and the standardised target in net->tgt
void backward(gr_net *net)
{
    cudaStream_t st = net->st;
    const int64_t nv0 = nvox(net, 0);
    cudaMemsetAsync(net->grads, 0, net->nparams * sizeof(float), st);
    cudaMemsetAsync(net->loss, 0, sizeof(float), st);
    gr::head_back(net->act[T_D0B], net->params + net->head_w, net->out, net->tgt, nv0, net->grad[T_D0B],
                  net->grads + net->head_w, net->grads + net->head_b, net->loss, st);
    // conv k: gradient at its output (already through that output's ReLU) ->
    // weight and bias gradients, and (dgrad_mode) the gradient at its input
    auto back = [&](int k, int dgrad_mode) {
        const Conv &c = net->conv[k];
        const int lg = net->lg0 - c.lev;
        const int in = kConvIO[k][0], outt = kConvIO[k][1];
        gr::conv3d_wgrad(net->act[in], c.cin, net->grad[outt], c.cout, lg, net->grads + c.w, st);
        gr::bias_grad(net->grad[outt], c.cout, nvox(net, c.lev), net->grads + c.b, st);
        if (dgrad_mode >= 0)
            gr::conv3d(net->grad[outt], c.cout, net->wt + c.wb, nullptr, c.cin, lg, dgrad_mode,
                       dgrad_mode == CONV_MASK ? net->act[in] : nullptr, net->grad[in], st);
    };
    back(13, CONV_MASK);   // -> grad d0a (through d0a's ReLU)
    back(12, CONV_PLAIN);  // -> grad cat0
    gr::upsample_back(net->grad[T_CAT0], 32, 48, net->lg0 - 1, net->grad[T_D1B], st);
    gr::relu_mask(net->grad[T_D1B], net->act[T_D1B], nvox(net, 1) * 32, st);
    gr::copy_slice(net->grad[T_CAT0], 16, 48, 32, net->grad[T_E0B], 16, 0, nv0, 0, st);
    back(11, CONV_MASK);
    back(10, CONV_PLAIN);
    gr::upsample_back(net->grad[T_CAT1], 64, 96, net->lg0 - 2, net->grad[T_D2B], st);
    gr::relu_mask(net->grad[T_D2B], net->act[T_D2B], nvox(net, 2) * 64, st);
    gr::copy_slice(net->grad[T_CAT1], 32, 96, 64, net->grad[T_E1B], 32, 0, nvox(net, 1), 0, st);
    back(9, CONV_MASK);
    back(8, CONV_PLAIN);
    gr::upsample_back(net->grad[T_CAT2], 128, 192, net->lg0 - 3, net->grad[T_E3B], st);
    gr::relu_mask(net->grad[T_E3B], net->act[T_E3B], nvox(net, 3) * 128, st);
    gr::copy_slice(net->grad[T_CAT2], 64, 192, 128, net->grad[T_E2B], 64, 0, nvox(net, 2), 0, st);
    back(7, CONV_MASK);
    back(6, CONV_PLAIN);  // -> grad p3
    gr::pool_back(net->grad[T_P3], 64, net->lg0 - 2, net->grad[T_E2B], 64, 1, st);
    gr::relu_mask(net->grad[T_E2B], net->act[T_E2B], nvox(net, 2) * 64, st);
    back(5, CONV_MASK);
    back(4, CONV_PLAIN);
    gr::pool_back(net->grad[T_P2], 32, net->lg0 - 1, net->grad[T_E1B], 32, 1, st);
    gr::relu_mask(net->grad[T_E1B], net->act[T_E1B], nvox(net, 1) * 32, st);
    back(3, CONV_MASK);
    back(2, CONV_PLAIN);
    gr::pool_back(net->grad[T_P1], 16, net->lg0, net->grad[T_E0B], 16, 1, st);
    gr::relu_mask(net->grad[T_E0B], net->act[T_E0B], nv0 * 16, st);
    back(1, CONV_MASK);
    back(0, -1);
}

gr_status net_check(const char *where, cudaStream_t st = nullptr)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
        return nfail(GR_ERR_CUDA, buf);
    }
    if (st && gr::conv3d_tc_error(st) != 0) {  // synchronises the network's stream
        char buf[256];
        snprintf(buf, sizeof(buf), "%s: a bounded wait of the tcgen05 convolution ran out", where);
        return nfail(GR_ERR_CUDA, buf);
    }
    return GR_OK;
}

}  // namespace

extern "C" {

gr_status gr_net_create(int n, void *stream, uint64_t seed, gr_net **out)
{
    if (!out) return nfail(GR_ERR_ARG, "gr_net_create: out is NULL");
    *out = nullptr;
    if (n < 32 || n > 512 || (n & (n - 1))) return nfail(GR_ERR_ARG, "gr_net_create: n must be a power of two in [32, 512]");
    gr_net *net = new (std::nothrow) gr_net();
    if (!net) return nfail(GR_ERR_NOMEM, "gr_net_create: host allocation");
    net->n = n;
    while ((1 << net->lg0) < n) net->lg0++;
    net->st = (cudaStream_t)stream;
    size_t off = 0, boff = 0;
    for (int k = 0; k < 14; k++) {
        Conv &c = net->conv[k];
        c.cin = kConvSpec[k][0];
        c.cout = kConvSpec[k][1];
        c.lev = kConvSpec[k][2];
        c.w = off;
        off += (size_t)27 * c.cout * c.cin;
        c.b = off;
        off += c.cout;
        c.wb = boff;
        boff += (size_t)27 * c.cout * c.cin;
    }
    net->head_w = off;
    off += (size_t)kNetOut * 16;
    net->head_b = off;
    off += kNetOut;
    net->nparams = off;
    net->nbf = boff;
    bool ok = nalloc(net, &net->params, off) && nalloc(net, &net->grads, off) && nalloc(net, &net->adam_m, off) &&
              nalloc(net, &net->adam_v, off) && nalloc(net, &net->wb, boff) && nalloc(net, &net->wt, boff) &&
              nalloc(net, &net->norm, 28) && nalloc(net, &net->loss, 1);
    net->act.assign(T_NT, nullptr);
    net->grad.assign(T_NT, nullptr);
    for (int t = 0; t < T_NT && ok; t++) {
        const size_t cnt = (size_t)nvox(net, kTensor[t][0]) * kTensor[t][1];
        ok = nalloc(net, &net->act[t], cnt) && nalloc(net, &net->grad[t], cnt);
    }
    ok = ok && nalloc(net, &net->out, (size_t)nvox(net, 0) * kNetOut) &&
         nalloc(net, &net->tgt, (size_t)nvox(net, 0) * kNetOut);
    if (ok && cudaMallocHost((void **)&net->hloss, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
    }
    if (!ok) {
        gr_net_destroy(net);
        return nfail(GR_ERR_NOMEM, "gr_net_create: device allocation failed");
    }
    // He-normal weights (std sqrt(2 / fan_in)), zero biases, identity normalisation
    std::vector<float> h(off, 0.0f);
    std::mt19937_64 rng(seed);
    for (int k = 0; k < 14; k++) {
        const Conv &c = net->conv[k];
        const int fan_in = 27 * (k == 0 ? 4 : c.cin);
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / fan_in));
        for (size_t e = 0; e < (size_t)27 * c.cout * c.cin; e++) {
            const int ci = (int)(e % c.cin);
            h[c.w + e] = (k == 0 && ci >= 4) ? 0.0f : nd(rng);
        }
    }
    std::normal_distribution<float> nh(0.0f, std::sqrt(1.0f / 16.0f));
    for (int e = 0; e < kNetOut * 16; e++) h[net->head_w + e] = nh(rng);
    for (int k = 0; k < 28; k++) net->hnorm[k] = (k < 4 || (k >= 8 && k < 18)) ? 0.0f : 1.0f;
    cudaMemcpyAsync(net->params, h.data(), off * sizeof(float), cudaMemcpyHostToDevice, net->st);
    cudaMemcpyAsync(net->norm, net->hnorm, sizeof(net->hnorm), cudaMemcpyHostToDevice, net->st);
    cudaMemsetAsync(net->adam_m, 0, off * sizeof(float), net->st);
    cudaMemsetAsync(net->adam_v, 0, off * sizeof(float), net->st);
    refresh_bf16(net);
    cudaStreamSynchronize(net->st);
    gr_status s = net_check("gr_net_create");
    if (s != GR_OK) {
        gr_net_destroy(net);
        return s;
    }
    *out = net;
    return GR_OK;
}

void gr_net_destroy(gr_net *net)
{
    if (!net) return;
    if (net->st) cudaStreamSynchronize(net->st);
    else cudaDeviceSynchronize();
    for (void *p : net->allocs) cudaFree(p);
    if (net->hloss) cudaFreeHost(net->hloss);
    delete net;
}

size_t gr_net_num_params(const gr_net *net) { return net ? net->nparams : 0; }

gr_status gr_net_get_params(gr_net *net, float *host)
{
    if (!net || !host) return nfail(GR_ERR_ARG, "gr_net_get_params: NULL argument");
    cudaMemcpyAsync(host, net->params, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, net->st);
    cudaStreamSynchronize(net->st);
    return net_check("gr_net_get_params");
}

gr_status gr_net_set_params(gr_net *net, const float *host)
{
    if (!net || !host) return nfail(GR_ERR_ARG, "gr_net_set_params: NULL argument");
    cudaMemcpyAsync(net->params, host, net->nparams * sizeof(float), cudaMemcpyHostToDevice, net->st);
    cudaMemsetAsync(net->adam_m, 0, net->nparams * sizeof(float), net->st);
    cudaMemsetAsync(net->adam_v, 0, net->nparams * sizeof(float), net->st);
    net->step = 0;
    refresh_bf16(net);
    cudaStreamSynchronize(net->st);
    return net_check("gr_net_set_params");
}

gr_status gr_net_set_norm(gr_net *net, const float *in_mean, const float *in_std, const float *out_mean,
                          const float *out_std)
{
    if (!net || !in_mean || !in_std || !out_mean || !out_std) return nfail(GR_ERR_ARG, "gr_net_set_norm: NULL argument");
    for (int k = 0; k < 4; k++) {
        if (!(in_std[k] > 0)) return nfail(GR_ERR_ARG, "gr_net_set_norm: in_std must be > 0");
        net->hnorm[k] = in_mean[k];
        net->hnorm[4 + k] = in_std[k];
    }
    for (int k = 0; k < kNetOut; k++) {
        if (!(out_std[k] > 0)) return nfail(GR_ERR_ARG, "gr_net_set_norm: out_std must be > 0");
        net->hnorm[8 + k] = out_mean[k];
        net->hnorm[18 + k] = out_std[k];
    }
    cudaMemcpyAsync(net->norm, net->hnorm, sizeof(net->hnorm), cudaMemcpyHostToDevice, net->st);
    cudaStreamSynchronize(net->st);
    return net_check("gr_net_set_norm");
}

gr_status gr_net_infer(gr_net *net, const gr_sources *s, double rho_hat, double v_rms, gr_fields *guess)
{
    if (!net || !s || !guess || !s->s0 || !s->s[0] || !s->s[1] || !s->s[2])
        return nfail(GR_ERR_ARG, "gr_net_infer: NULL argument");
    if (!(rho_hat > 0) || !(v_rms > 0)) return nfail(GR_ERR_ARG, "gr_net_infer: rho_hat and v_rms must be > 0");
    forward(net, s, rho_hat, v_rms);
    gr::net_output(net->out, nvox(net, 0), net->norm + 8, net->norm + 18, field_ptrs(guess), net->st);
    return net_check("gr_net_infer", net->st);
}

gr_status gr_net_guess(gr_net *net, int n_fine, const gr_sources *s, double rho_hat, double v_rms, gr_fields *guess)
{
    if (!net || !s || !guess || !s->s0 || !s->s[0] || !s->s[1] || !s->s[2])
        return nfail(GR_ERR_ARG, "gr_net_guess: NULL argument");
    if (!(rho_hat > 0) || !(v_rms > 0)) return nfail(GR_ERR_ARG, "gr_net_guess: rho_hat and v_rms must be > 0");
    int lr = 0;
    while ((net->n << lr) < n_fine && lr < 8) ++lr;
    if (n_fine < net->n || (net->n << lr) != n_fine || n_fine > 1024)
        return nfail(GR_ERR_ARG, "gr_net_guess: n_fine must be the network's n times a power of two, at most 1024");
    if (lr == 0) return gr_net_infer(net, s, rho_hat, v_rms, guess);
    const int64_t nv = nvox(net, 0);
    if (!net->coarse_src && !nalloc(net, &net->coarse_src, 4 * (size_t)nv))
        return nfail(GR_ERR_NOMEM, "gr_net_guess: cudaMalloc");
    FieldPtrs in = {}, cs = {};
    const double *fin[4] = {s->s0, s->s[0], s->s[1], s->s[2]};
    for (int a = 0; a < 4; a++) {
        in.p[a] = const_cast<double *>(fin[a]);
        cs.p[a] = net->coarse_src + a * nv;
    }
    gr::avg_down(in, cs, 4, net->lg0, lr, net->st);
    gr_sources sc = {};
    sc.s0 = cs.p[0];
    sc.s[0] = cs.p[1];
    sc.s[1] = cs.p[2];
    sc.s[2] = cs.p[3];
    sc.sigma = nullptr;
    forward(net, &sc, rho_hat, v_rms);
    gr::net_output_fine(net->out, net->lg0, lr, net->norm + 8, net->norm + 18, field_ptrs(guess), net->st);
    return net_check("gr_net_guess");
}

gr_status gr_net_loss_grad(gr_net *net, const gr_sources *s, const gr_fields *target, double rho_hat, double v_rms,
                           float *loss_out, float *host_grads)
{
    if (!net || !s || !target) return nfail(GR_ERR_ARG, "gr_net_loss_grad: NULL argument");
    if (!(rho_hat > 0) || !(v_rms > 0)) return nfail(GR_ERR_ARG, "gr_net_loss_grad: rho_hat and v_rms must be > 0");
    forward(net, s, rho_hat, v_rms);
    gr::net_target(field_ptrs(target), nvox(net, 0), net->norm + 8, net->norm + 18, net->tgt, net->st);
    backward(net);
    cudaMemcpyAsync(net->hloss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, net->st);
    if (host_grads)
        cudaMemcpyAsync(host_grads, net->grads, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, net->st);
    cudaStreamSynchronize(net->st);
    if (loss_out) *loss_out = *net->hloss;
    return net_check("gr_net_loss_grad", net->st);
}

gr_status gr_net_train_step(gr_net *net, const gr_sources *s, const gr_fields *target, double rho_hat, double v_rms,
                            float lr, float *loss_out)
{
    if (!(lr > 0)) return nfail(GR_ERR_ARG, "gr_net_train_step: lr must be > 0");
    gr_status st = GR_OK;
    if (!net || !s || !target) return nfail(GR_ERR_ARG, "gr_net_train_step: NULL argument");
    if (!(rho_hat > 0) || !(v_rms > 0)) return nfail(GR_ERR_ARG, "gr_net_train_step: rho_hat and v_rms must be > 0");
    forward(net, s, rho_hat, v_rms);
    gr::net_target(field_ptrs(target), nvox(net, 0), net->norm + 8, net->norm + 18, net->tgt, net->st);
    backward(net);
    net->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    gr::adam(net->params, net->adam_m, net->adam_v, net->grads, (int64_t)net->nparams, lr, b1, b2, 1e-8f,
             1.0f - std::pow(b1, (float)net->step), 1.0f - std::pow(b2, (float)net->step), net->st);
    refresh_bf16(net);
    if (loss_out) {
        cudaMemcpyAsync(net->hloss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, net->st);
        cudaStreamSynchronize(net->st);
        *loss_out = *net->hloss;
    }
    st = net_check("gr_net_train_step", net->st);
    return st;
}

gr_status gr_net_activation(gr_net *net, int tensor, float *host, size_t count)
{
    if (!net || !host || tensor < 0 || tensor >= T_NT) return nfail(GR_ERR_ARG, "gr_net_activation: bad argument");
    const size_t cnt = (size_t)nvox(net, kTensor[tensor][0]) * kTensor[tensor][1];
    if (count != cnt) return nfail(GR_ERR_ARG, "gr_net_activation: count does not match the tensor size");
    std::vector<bf16> tmp(cnt);
    cudaMemcpyAsync(tmp.data(), net->act[tensor], cnt * sizeof(bf16), cudaMemcpyDeviceToHost, net->st);
    cudaStreamSynchronize(net->st);
    for (size_t e = 0; e < cnt; e++) host[e] = __bfloat162float(tmp[e]);
    return net_check("gr_net_activation");
}

}  // extern "C"
