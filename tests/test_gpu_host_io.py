"""GPU checks of host-buffer I/O through the C ABI: a deposit from host
particle arrays (pinned or pageable, several staging chunks) equals the
deposit from device arrays, mixed host/device inputs are an argument error,
and gr_opts.host_out receives every solved field."""
import numpy as np
import pytest

import oracle
from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("pinned", [True, False])
def test_host_particle_deposit_matches_device_deposit(monkeypatch, pinned):
    monkeypatch.setenv("GR_HOST_CHUNK", "3000")  # 12345 particles -> five chunks through two buffers
    n, npart = 16, 12345
    rng = np.random.default_rng(7)
    x = rng.random((3, npart)) * 1.2 - 0.1
    u = 0.05 * rng.standard_normal((3, npart))
    xh, uh = torch.from_numpy(x), torch.from_numpy(u)
    if pinned:
        xh, uh = xh.pin_memory(), uh.pin_memory()
    ctx = gr.Context(n)
    dev = ctx.deposit(xh.cuda(), uh.cuda(), 0.3)
    host = ctx.deposit(xh, uh, 0.3)
    torch.cuda.synchronize()
    want = oracle.deposit(n, x, u, 0.3)
    for k in oracle.SOURCES:
        assert _rel(host[k].cpu().numpy(), dev[k].cpu().numpy()) <= 1e-14, k
        assert _rel(host[k].cpu().numpy(), want[k]) <= 1e-13, k
    # a second call reuses the staging buffers
    host2 = ctx.deposit(xh, uh, 0.3)
    torch.cuda.synchronize()
    for k in oracle.SOURCES:
        assert _rel(host2[k].cpu().numpy(), dev[k].cpu().numpy()) <= 1e-14, k
    ctx.close()


def test_mixed_host_and_device_particles_is_an_argument_error():
    ctx = gr.Context(8)
    x = torch.rand((3, 10), dtype=torch.float64)
    with pytest.raises(gr.GRError) as ei:
        ctx.deposit(x, x.cuda(), 1.0)
    assert ei.value.status == gr.GR_ERR_ARG
    ctx.close()


def test_host_out_receives_every_solved_field():
    n = 32
    p = synth.zeldovich(n, 9, 0.5, 0.01, True)
    ctx = gr.Context(n)
    src = ctx.deposit(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.u).cuda(), p.mass)
    fld = ctx.initial_fields()
    host = {k: torch.full((n, n, n), np.nan, dtype=torch.float64).pin_memory() for k in gr.FIELDS}
    rep = ctx.solve(src, fld, tol=1e-9, max_cycles=60, prec="mixed_df", rho_hat=p.rho_hat, host_out=host)
    torch.cuda.current_stream().synchronize()
    assert rep["status_code"] == gr.GR_OK
    for k in gr.FIELDS:
        assert torch.equal(host[k], fld[k].cpu()), k
    ctx.close()


@pytest.mark.parametrize("prec", ["mixed_df", "fp64"])
def test_host_out_solve_equals_device_solve(prec):
    """The norms that decide every cycle reach the host through mapped memory
    while field copies are in flight: the solve with host buffers takes the
    same cycles and gives the same fields bit for bit."""
    n = 32
    p = synth.zeldovich(n, 12, 2.0, 0.01, True)
    ctx = gr.Context(n)
    src = ctx.deposit(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.u).cuda(), p.mass)
    opts = dict(tol=1e-10, max_cycles=60, prec=prec, rho_hat=p.rho_hat)
    f_dev = ctx.initial_fields()
    r_dev = ctx.solve(src, f_dev, **opts)
    f_host = ctx.initial_fields()
    host = {k: torch.full((n, n, n), np.nan, dtype=torch.float64).pin_memory() for k in gr.FIELDS}
    r_host = ctx.solve(src, f_host, host_out=host, **opts)
    torch.cuda.current_stream().synchronize()
    assert r_dev["status_code"] == gr.GR_OK and r_host["status_code"] == gr.GR_OK
    assert r_dev["cycles"] == r_host["cycles"]
    assert r_dev["res"] == r_host["res"]
    for k in gr.FIELDS:
        assert torch.equal(f_dev[k], f_host[k]), k
        assert torch.equal(host[k], f_dev[k].cpu()), k
    ctx.close()
