"""GPU checks of the learned initial-guess network against the FP64 CPU
reference (oracle/unet_ref.py): per-layer forward, whole-network output,
loss and every parameter gradient, a directional finite difference, and
training progress.  The GPU keeps activations in BF16 (8 significant bits),
so the tolerances are those of BF16 arithmetic, not of FP64."""
import numpy as np
import pytest

import oracle
from oracle import unet_ref
from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402

N = 32
V_RMS = 0.01


@pytest.fixture(scope="module")
def case():
    p = synth.zeldovich(N, 21, 1.0, V_RMS, True)
    src = oracle.deposit(N, p.x, p.u, p.mass)
    fld = oracle.initial_fields(N)
    st, _ = oracle.solve_constraints(src, fld, p.rho_hat, tol=1e-10, max_cycles=60)
    assert st == 0
    x_in = [np.log(unet_ref.LOG_EPS + src["s0"] / p.rho_hat)] + [src[k] / (p.rho_hat * V_RMS) for k in
                                                                  ("sx", "sy", "sz")]
    in_mean = np.array([a.mean() for a in x_in])
    in_std = np.array([a.std() for a in x_in])
    dev = [fld["psi"] - 1, fld["apsi"] - 1] + [fld[k] for k in ("Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b")]
    out_mean = np.array([a.mean() for a in dev])
    out_std = np.array([max(a.std(), 1e-30) for a in dev])
    net = gr.Net(N, seed=5)
    net.set_norm(in_mean, in_std, out_mean, out_std)
    gsrc = {k: torch.from_numpy(v).cuda() for k, v in src.items()}
    gfld = {k: torch.from_numpy(v).cuda() for k, v in fld.items()}
    xref = unet_ref.net_input(src["s0"], src["sx"], src["sy"], src["sz"], p.rho_hat, V_RMS, in_mean, in_std)
    tref = unet_ref.standardise_fields(fld, out_mean, out_std)
    yield dict(p=p, src=src, fld=fld, net=net, gsrc=gsrc, gfld=gfld, xref=xref, tref=tref, out_mean=out_mean,
               out_std=out_std)
    net.close()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _abs_conv(params, k, x_channels_last):
    """sum over taps and input channels of |W| |x| plus |b| for convolution k
    (the scale of every rounding in that output element)."""
    import torch.nn.functional as F

    layers, _ = unet_ref.unpack(params)
    w, b = layers[k]
    x = torch.as_tensor(np.abs(x_channels_last), dtype=torch.float64).permute(3, 0, 1, 2).unsqueeze(0)
    y = F.conv3d(F.pad(x, (1, 1, 1, 1, 1, 1), mode="circular"), w.abs(), b.abs())
    return y[0].permute(1, 2, 3, 0).numpy()


def test_each_convolution_matches_fp64_on_its_gpu_input(case):
    """One layer at a time: the GPU layer output against the FP64 layer applied
    to the GPU's own (BF16) input, so errors do not accumulate.  Elementwise
    bound: the GPU rounds the weights to BF16 (relative 2^-9 each) and its
    output to BF16 (relative 2^-9 of |y|), and accumulates in FP32
    (negligible), so |y_gpu - y_fp64| <= c 2^-8 (sum |W||x| + |b|) with c = 1
    in every output element, ReLU or not.  The relative L2 error stays below
    1e-2 as well."""
    net = case["net"]
    out = {k: torch.empty((N, N, N), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    net.infer(case["gsrc"], out, case["p"].rho_hat, V_RMS)
    params = net.get_params()
    io = [("x0", "e0a"), ("e0a", "e0b"), ("p1", "e1a"), ("e1a", "e1b"), ("p2", "e2a"), ("e2a", "e2b"),
          ("p3", "e3a"), ("e3a", "e3b"), ("cat2", "d2a"), ("d2a", "d2b"), ("cat1", "d1a"), ("d1a", "d1b"),
          ("cat0", "d0a"), ("d0a", "d0b")]
    for k, (a, b) in enumerate(io):
        x = net.activation(a)
        want = unet_ref.conv_layer(params, k, x)
        got = net.activation(b)
        bound = 2.0 ** -8 * _abs_conv(params, k, x)
        excess = np.abs(got - want) - bound
        assert excess.max() <= 0, (k, float(excess.max()), int((excess > 0).sum()))
        assert _rel(got, want) < 1e-2, (k, _rel(got, want))


def test_pool_upsample_and_concat_match_fp64(case):
    """Elementwise: pooling and upsampling average BF16 values in FP32 and
    round the result to BF16, so each element is within 2^-8 of the same
    operation applied to |x| (c = 1)."""
    net = case["net"]
    x = torch.as_tensor(net.activation("e0b")).permute(3, 0, 1, 2).unsqueeze(0).double()
    got = net.activation("p1")
    want = unet_ref.pool(x)[0].permute(1, 2, 3, 0).numpy()
    assert (np.abs(got - want) <= 2.0 ** -8 * unet_ref.pool(x.abs())[0].permute(1, 2, 3, 0).numpy()).all()
    assert _rel(got, want) < 5e-3
    e3b = torch.as_tensor(net.activation("e3b")).permute(3, 0, 1, 2).unsqueeze(0).double()
    up = unet_ref.up2(e3b)[0].permute(1, 2, 3, 0).numpy()
    up_abs = unet_ref.up2(e3b.abs())[0].permute(1, 2, 3, 0).numpy()
    cat2 = net.activation("cat2")
    assert (np.abs(cat2[..., :128] - up) <= 2.0 ** -8 * up_abs).all()
    assert _rel(cat2[..., :128], up) < 5e-3
    assert np.array_equal(cat2[..., 128:], net.activation("e2b"))


def test_network_output_matches_fp64(case):
    net = case["net"]
    params = net.get_params()
    out = {k: torch.empty((N, N, N), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    net.infer(case["gsrc"], out, case["p"].rho_hat, V_RMS)
    layers, head = unet_ref.unpack(params)
    y = unet_ref.forward(layers, head, case["xref"])[0].numpy()
    for k, name in enumerate(gr.FIELDS):
        got = (out[name].cpu().numpy() - (1.0 if k < 2 else 0.0) - case["out_mean"][k]) / case["out_std"][k]
        assert _rel(got, y[k]) < 3e-2, (name, _rel(got, y[k]))
        # elementwise after 14 BF16 layers: every voxel within 5% of the channel's largest value
        assert np.abs(got - y[k]).max() <= 5e-2 * np.abs(y[k]).max(), (name, np.abs(got - y[k]).max())


def test_loss_and_every_gradient_match_fp64_autograd(case):
    net = case["net"]
    params = net.get_params()
    loss, g = net.loss_grad(case["gsrc"], case["gfld"], case["p"].rho_hat, V_RMS)
    lref, gref = unet_ref.loss_and_grad(params, case["xref"], case["tref"])
    assert abs(loss - lref) <= 2e-2 * lref, (loss, lref)
    off = 0
    for k, (cin, cout) in enumerate(unet_ref.CONVS):
        for part, size in (("w", 27 * cout * cin), ("b", cout)):
            a, b = g[off:off + size], gref[off:off + size]
            off += size
            if k == 0 and part == "w":  # the 12 zero-padded input channels carry no gradient
                a = a.reshape(27, cout, cin)[:, :, :4]
                b = b.reshape(27, cout, cin)[:, :, :4]
            cos = float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))
            assert cos > 0.99 and _rel(a, b) < 0.1, (k, part, cos, _rel(a, b))
    for size in (10 * 16, 10):
        a, b = g[off:off + size], gref[off:off + size]
        off += size
        assert _rel(a, b) < 0.05
    assert off == g.size


def test_directional_finite_difference(case):
    """L(w + eps d) - L(w - eps d) = 2 eps |g| for d = g/|g|, to first order."""
    net = case["net"]
    w0 = net.get_params()
    loss, g = net.loss_grad(case["gsrc"], case["gfld"], case["p"].rho_hat, V_RMS)
    d = g / np.linalg.norm(g)
    eps = 0.05 * np.linalg.norm(w0) / np.sqrt(w0.size) * 0.2
    vals = []
    for s in (-1.0, 1.0):
        net.set_params(w0 + s * eps * d)
        vals.append(net.loss_grad(case["gsrc"], case["gfld"], case["p"].rho_hat, V_RMS, want_grads=False)[0])
    net.set_params(w0)
    fd = (vals[1] - vals[0]) / (2 * eps)
    assert fd == pytest.approx(np.linalg.norm(g), rel=0.1), (fd, np.linalg.norm(g))


def test_training_steps_reduce_the_loss(case):
    net = gr.Net(N, seed=9)
    net.set_norm(*case["net"].norm)
    first = net.train_step(case["gsrc"], case["gfld"], case["p"].rho_hat, V_RMS, 5e-4)
    losses = [net.train_step(case["gsrc"], case["gfld"], case["p"].rho_hat, V_RMS, 5e-4) for _ in range(150)]
    assert min(losses) < 0.5 * first and np.mean(losses[-10:]) < 0.7 * first, (first, losses[::15])
    net.close()


def _trilinear_up(a, r):
    """Periodic trilinear interpolation between cell centres from an m^3 grid
    to the (r m)^3 grid of the same box (numpy, FP64)."""
    m = a.shape[0]
    c = (np.arange(r * m) + 0.5) / r - 0.5
    lo = np.floor(c).astype(int)
    w1 = c - lo
    out = a
    for ax in range(3):
        a0 = np.take(out, lo % m, axis=ax)
        a1 = np.take(out, (lo + 1) % m, axis=ax)
        shape = [1, 1, 1]
        shape[ax] = r * m
        w = w1.reshape(shape)
        out = (1 - w) * a0 + w * a1
    return out


def test_guess_on_a_finer_grid(case):
    """gr_net_guess for a 2x finer grid: the sources averaged over 2^3 blocks
    (dyadic values, so the average is exact in any order and the network sees
    the same input as gr_net_infer on the numpy average), the network's fields
    interpolated trilinearly to the fine grid (numpy reference; the GPU
    interpolates the FP32 standardised outputs, hence the FP32-size bar)."""
    net, rho = case["net"], case["p"].rho_hat
    nf = 2 * N
    rng = np.random.default_rng(12)
    fine = {}
    for k in oracle.SOURCES:
        base = rho if k == "s0" else rho * V_RMS
        v = np.round(rng.random((nf, nf, nf)) * 2 ** 20) / 2 ** 20
        fine[k] = base * (0.5 + v) if k == "s0" else base * (v - 0.5)
    coarse = {k: v.reshape(N, 2, N, 2, N, 2).mean(axis=(1, 3, 5)) for k, v in fine.items()}
    out_c = {k: torch.empty((N, N, N), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    net.infer({k: torch.from_numpy(v).cuda() for k, v in coarse.items()}, out_c, rho, V_RMS)
    out_f = {k: torch.empty((nf, nf, nf), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    net.guess(nf, {k: torch.from_numpy(v).cuda() for k, v in fine.items()}, out_f, rho, V_RMS)
    torch.cuda.synchronize()
    for k, name in enumerate(gr.FIELDS):
        d = 1.0 if k < 2 else 0.0
        want = _trilinear_up(out_c[name].cpu().numpy() - d, 2)
        got = out_f[name].cpu().numpy() - d
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max() + 1e-6 * case["out_std"][k], name
    with pytest.raises(gr.GRError):
        net.guess(3 * N, {k: torch.from_numpy(v).cuda() for k, v in fine.items()}, out_f, rho, V_RMS)


def _sampled_conv(params, k, x, vox):
    """FP64 convolution k (with ReLU) and its rounding scale sum |W||x| + |b|
    at the sampled output voxels vox (rows of (d, h, w)) of a channels-last
    activation x [n, n, n, cin] (periodic)."""
    layers, _ = unet_ref.unpack(params)
    W, b = (t.numpy() for t in layers[k])  # W [cout][cin][3][3][3]
    n = x.shape[0]
    want = np.tile(b, (len(vox), 1)).astype(np.float64)
    scale = np.tile(np.abs(b), (len(vox), 1)).astype(np.float64)
    for dd in (-1, 0, 1):
        for dh in (-1, 0, 1):
            for dw in (-1, 0, 1):
                xs = x[(vox[:, 0] + dd) % n, (vox[:, 1] + dh) % n, (vox[:, 2] + dw) % n].astype(np.float64)
                Wt = W[:, :, dd + 1, dh + 1, dw + 1]
                want += xs @ Wt.T
                scale += np.abs(xs) @ np.abs(Wt).T
    return np.maximum(want, 0.0), scale


def test_tcgen05_convolutions_at_128_cubed(monkeypatch):
    """At 128^3 the finest level's convolutions with 16 input channels, and
    the decoder's 48 -> 16 one, run on the 5th-generation tensor cores
    (conv_tc.cu: tcgen05.mma, TMEM accumulator).  Each finest-level layer is held, at 6000 sampled voxels
    including both row ends (the wrapped halo), to the FP64 convolution of its
    own GPU input within 2^-8 (sum |W||x| + |b|) (the per-layer bound above);
    the whole output agrees with the mma.sync path (GR_CONV_TC=0) to BF16
    rounding; and the loss gradients of the two paths point the same way (the
    data gradients of these layers into 16 and 48 channels run on tcgen05
    too)."""
    n = 128
    p = synth.zeldovich(n, 33, 1.5, V_RMS, True)
    ctx = gr.Context(n)
    src = ctx.deposit(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.u).cuda(), p.mass)
    x_in = [torch.log(unet_ref.LOG_EPS + src["s0"] / p.rho_hat)] + [src[k] / (p.rho_hat * V_RMS) for k in
                                                                     ("sx", "sy", "sz")]
    in_mean = np.array([float(a.mean()) for a in x_in])
    in_std = np.array([float(a.std()) for a in x_in])
    net = gr.Net(n, seed=11)
    net.set_norm(in_mean, in_std, np.zeros(10), np.ones(10) * 1e-4)
    params = net.get_params()
    outs, grads = [], []
    target = {k: torch.zeros((n, n, n), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    target["psi"] += 1.0
    target["apsi"] += 1.0
    for flag in ("1", "0"):
        monkeypatch.setenv("GR_CONV_TC", flag)
        out = {k: torch.empty((n, n, n), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
        net.infer(src, out, p.rho_hat, V_RMS)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in out.items()})
        if flag == "1":
            rng = np.random.default_rng(5)
            vox = rng.integers(0, n, size=(6000, 3))
            vox[:200, 2] = 0
            vox[200:400, 2] = n - 1
            for k, (a, b) in ((0, ("x0", "e0a")), (1, ("e0a", "e0b")), (12, ("cat0", "d0a")), (13, ("d0a", "d0b"))):
                x = net.activation(a)
                got = net.activation(b)[vox[:, 0], vox[:, 1], vox[:, 2]]
                want, scale = _sampled_conv(params, k, x, vox)
                excess = np.abs(got - want) - 2.0 ** -8 * scale
                assert excess.max() <= 0, (k, float(excess.max()))
        loss, g = net.loss_grad(src, target, p.rho_hat, V_RMS)
        grads.append(g)
    for k in gr.FIELDS:
        d = 1.0 if k in ("psi", "apsi") else 0.0
        a, b = outs[0][k] - d, outs[1][k] - d
        assert np.abs(a - b).max() <= 5e-2 * np.abs(b).max(), k
    ga, gb = grads
    cos = float(np.dot(ga, gb) / (np.linalg.norm(ga) * np.linalg.norm(gb)))
    assert cos > 0.999, cos
    net.close()
    ctx.close()
