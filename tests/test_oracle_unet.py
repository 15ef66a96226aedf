"""Pins of the FP64 reference network (oracle/unet_ref.py) used to check the
GPU network: tap orientation and circular wrap of the convolution, pooling
and upsampling against the multigrid transfers of the C oracle, and the
autograd gradient against finite differences."""
import numpy as np
import pytest
import torch

from oracle import unet_ref


def _params(seed, scale=0.05):
    n = sum(27 * ci * co + co for ci, co in unet_ref.CONVS) + 170
    return np.random.default_rng(seed).standard_normal(n) * scale


def test_convolution_tap_orientation_and_wrap():
    """A unit impulse at voxel v0 gives y[v0 - offset(tap)] = W[tap]: the layer
    adds W[tap] x[v + offset], offsets wrapping around the periodic box."""
    n = 4
    p = _params(0)
    layers, _ = unet_ref.unpack(p)
    flat = torch.as_tensor(p[:27 * 16 * 16]).reshape(27, 16, 16)  # [tap][cout][cin]
    x = torch.zeros((1, 16, n, n, n), dtype=torch.float64)
    v0 = (0, 3, 1)
    x[0, 5, v0[0], v0[1], v0[2]] = 1.0
    w, b = layers[0]
    y = unet_ref.conv(x, w, b * 0, relu=False)
    for tap in (0, 4, 13, 22, 26):
        dd, dh, dw = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
        v = ((v0[0] - dd) % n, (v0[1] - dh) % n, (v0[2] - dw) % n)
        assert torch.allclose(y[0, :, v[0], v[1], v[2]], flat[tap, :, 5]), tap


def test_pool_and_upsample_equal_the_multigrid_transfers(orc):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((8, 8, 8))
    pooled = unet_ref.pool(torch.as_tensor(f).view(1, 1, 8, 8, 8))[0, 0].numpy()
    assert np.allclose(pooled, orc.restrict(f), atol=1e-14)
    c = rng.standard_normal((4, 4, 4))
    up = unet_ref.up2(torch.as_tensor(c).view(1, 1, 4, 4, 4))[0, 0].numpy()
    want = np.zeros((8, 8, 8))
    orc.prolong_add(c, want)
    assert np.allclose(up, want, atol=1e-14)


def test_autograd_gradient_matches_finite_differences():
    n = 8
    p = _params(2)
    x = torch.randn((1, 16, n, n, n), dtype=torch.float64, generator=torch.Generator().manual_seed(0))
    t = torch.randn((1, 10, n, n, n), dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    loss, g = unet_ref.loss_and_grad(p, x, t)
    rng = np.random.default_rng(3)
    idx = list(rng.choice(p.size, 6, replace=False)) + [int(np.argmax(np.abs(g)))]
    for i in idx:
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp, _ = unet_ref.loss_and_grad(pp, x, t)
        lm, _ = unet_ref.loss_and_grad(pm, x, t)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-4, abs=1e-9), (i, fd, g[i])
