"""FP64 CPU reference of the learned initial-guess network - TEST INFRASTRUCTURE.

Plain PyTorch CPU operations in float64 (conv3d with circular padding,
average pooling, rolls) and autograd for the gradients; only the tests use
it.  It is written from the architecture stated in include/gr.h, not from
the CUDA code: four levels of 16, 32, 64, 128 channels, two circular 3^3
convolutions with ReLU per level and side, 2^3 average pooling, cell-centred
trilinear x2 upsampling (weights 3/4, 1/4 per axis, periodic), skip
concatenation [upsampled | skip], 1x1 head to 10 channels, MSE loss on the
standardised fields.

The flat parameter vector is the one the GPU network exposes: per
convolution the weights [27][cout][cin] (tap = (dd+1)*9 + (dh+1)*3 + (dw+1),
the offset added to the output voxel's coordinates) then the bias [cout];
then the head weights [10][16] and bias [10].
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

CONVS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
         (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
N_OUT = 10
LOG_EPS = 0.01


def unpack(params):
    """Split the flat vector into [(W[cout][cin][3][3][3], b)] and the head."""
    p = torch.as_tensor(params, dtype=torch.float64)
    out, off = [], 0
    for cin, cout in CONVS:
        w = p[off:off + 27 * cout * cin].reshape(27, cout, cin)
        off += 27 * cout * cin
        b = p[off:off + cout]
        off += cout
        # tap index t = kd*9 + kh*3 + kw with k = offset + 1 -> [cout][cin][kd][kh][kw]
        out.append((w.permute(1, 2, 0).reshape(cout, cin, 3, 3, 3), b))
    hw = p[off:off + N_OUT * 16].reshape(N_OUT, 16)
    off += N_OUT * 16
    hb = p[off:off + N_OUT]
    return out, (hw, hb)


def conv(x, w, b, relu=True):
    """Circular 3^3 cross-correlation: y[v] = b + sum_taps W[tap] x[v + offset(tap)]."""
    y = F.conv3d(F.pad(x, (1, 1, 1, 1, 1, 1), mode="circular"), w, b)
    return F.relu(y) if relu else y


def pool(x):
    return F.avg_pool3d(x, 2)


def up2(x):
    """Cell-centred trilinear x2 with periodic wrap: along each axis the fine
    cell 2I takes 3/4 of I and 1/4 of I-1, the fine cell 2I+1 3/4 of I and
    1/4 of I+1."""
    for ax in (2, 3, 4):
        lo = 0.75 * x + 0.25 * torch.roll(x, 1, dims=ax)
        hi = 0.75 * x + 0.25 * torch.roll(x, -1, dims=ax)
        shape = list(x.shape)
        x = torch.stack((lo, hi), dim=ax + 1).reshape(shape[:ax] + [2 * shape[ax]] + shape[ax + 1:])
    return x


def net_input(s0, sx, sy, sz, rho, v_rms, in_mean, in_std):
    """[1, 16, n, n, n]: standardised log(0.01 + s0/rho), s_i/(rho v_rms), zeros."""
    ch = [torch.log(LOG_EPS + torch.as_tensor(s0, dtype=torch.float64) / rho)]
    for s in (sx, sy, sz):
        ch.append(torch.as_tensor(s, dtype=torch.float64) / (rho * v_rms))
    ch = [(c - in_mean[k]) / in_std[k] for k, c in enumerate(ch)]
    n = ch[0].shape[0]
    x = torch.zeros((1, 16, n, n, n), dtype=torch.float64)
    for k in range(4):
        x[0, k] = ch[k]
    return x


def forward(layers, head, x, keep=None):
    """Network output [1, 10, n, n, n] (standardised); keep (dict) receives
    the named activations."""
    keep = {} if keep is None else keep
    (w0, b0), (w1, b1), (w2, b2), (w3, b3), (w4, b4), (w5, b5), (w6, b6), (w7, b7), \
        (w8, b8), (w9, b9), (w10, b10), (w11, b11), (w12, b12), (w13, b13) = layers
    keep["x0"] = x
    keep["e0a"] = e0a = conv(x, w0, b0)
    keep["e0b"] = e0b = conv(e0a, w1, b1)
    keep["p1"] = p1 = pool(e0b)
    keep["e1a"] = e1a = conv(p1, w2, b2)
    keep["e1b"] = e1b = conv(e1a, w3, b3)
    keep["p2"] = p2 = pool(e1b)
    keep["e2a"] = e2a = conv(p2, w4, b4)
    keep["e2b"] = e2b = conv(e2a, w5, b5)
    keep["p3"] = p3 = pool(e2b)
    keep["e3a"] = e3a = conv(p3, w6, b6)
    keep["e3b"] = e3b = conv(e3a, w7, b7)
    keep["cat2"] = cat2 = torch.cat((up2(e3b), e2b), dim=1)
    keep["d2a"] = d2a = conv(cat2, w8, b8)
    keep["d2b"] = d2b = conv(d2a, w9, b9)
    keep["cat1"] = cat1 = torch.cat((up2(d2b), e1b), dim=1)
    keep["d1a"] = d1a = conv(cat1, w10, b10)
    keep["d1b"] = d1b = conv(d1a, w11, b11)
    keep["cat0"] = cat0 = torch.cat((up2(d1b), e0b), dim=1)
    keep["d0a"] = d0a = conv(cat0, w12, b12)
    keep["d0b"] = d0b = conv(d0a, w13, b13)
    hw, hb = head
    return torch.einsum("oc,bcdhw->bodhw", hw, d0b) + hb.view(1, -1, 1, 1, 1)


def loss_and_grad(params, x, target_std):
    """MSE of the standardised output against target_std [1, 10, n, n, n] and
    its gradient with respect to the flat parameter vector (autograd)."""
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    layers, head = unpack(p)
    y = forward(layers, head, x)
    loss = torch.mean((y - target_std) ** 2)
    loss.backward()
    return float(loss.detach()), p.grad.numpy()


def conv_layer(params, k, x_channels_last):
    """Convolution k with ReLU applied to a channels-last activation [n, n, n, c]."""
    layers, _ = unpack(params)
    w, b = layers[k]
    x = torch.as_tensor(x_channels_last, dtype=torch.float64).permute(3, 0, 1, 2).unsqueeze(0)
    return conv(x, w, b)[0].permute(1, 2, 3, 0).numpy()


def standardise_fields(fields: dict, out_mean, out_std):
    """[1, 10, n, n, n] target: (field - mean)/std with psi, alpha psi as deviations."""
    names = ("psi", "apsi", "Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b")
    chans = []
    for k, nme in enumerate(names):
        f = torch.as_tensor(fields[nme], dtype=torch.float64)
        if k < 2:
            f = f - 1.0
        chans.append((f - out_mean[k]) / out_std[k])
    return torch.stack(chans).unsqueeze(0)


__all__ = ["CONVS", "unpack", "conv", "pool", "up2", "net_input", "forward", "loss_and_grad", "conv_layer",
           "standardise_fields", "math"]
