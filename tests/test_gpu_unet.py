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


def test_each_convolution_matches_fp64_on_its_gpu_input(case):
    """One layer at a time: the GPU layer output against the FP64 layer applied
    to the GPU's own (BF16) input, so errors do not accumulate."""
    net = case["net"]
    out = {k: torch.empty((N, N, N), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    net.infer(case["gsrc"], out, case["p"].rho_hat, V_RMS)
    params = net.get_params()
    io = [("x0", "e0a"), ("e0a", "e0b"), ("p1", "e1a"), ("e1a", "e1b"), ("p2", "e2a"), ("e2a", "e2b"),
          ("p3", "e3a"), ("e3a", "e3b"), ("cat2", "d2a"), ("d2a", "d2b"), ("cat1", "d1a"), ("d1a", "d1b"),
          ("cat0", "d0a"), ("d0a", "d0b")]
    for k, (a, b) in enumerate(io):
        want = unet_ref.conv_layer(params, k, net.activation(a))
        got = net.activation(b)
        assert _rel(got, want) < 1e-2, (k, _rel(got, want))


def test_pool_upsample_and_concat_match_fp64(case):
    net = case["net"]
    ref = {}
    x = torch.as_tensor(net.activation("e0b")).permute(3, 0, 1, 2).unsqueeze(0).double()
    assert _rel(net.activation("p1"), unet_ref.pool(x)[0].permute(1, 2, 3, 0).numpy()) < 5e-3
    e3b = torch.as_tensor(net.activation("e3b")).permute(3, 0, 1, 2).unsqueeze(0).double()
    up = unet_ref.up2(e3b)[0].permute(1, 2, 3, 0).numpy()
    cat2 = net.activation("cat2")
    assert _rel(cat2[..., :128], up) < 5e-3
    assert np.array_equal(cat2[..., 128:], net.activation("e2b"))
    del ref


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
