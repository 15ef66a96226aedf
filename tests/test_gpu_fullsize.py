"""Full-size check in the bench's launch configuration: the 512^3 lognormal
(rms delta 5) workload, double-float mixed solve to 1e-8.  The oracle cannot
solve this grid in test time, so it checks (a) the whole deposit against its
own, and (b) the discrete equations at sampled cells: it evaluates every
equation's residual at the GPU's final fields, pointwise in FP64."""
import numpy as np
import pytest

import oracle
from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402


def test_bench_workload_deposit_and_sampled_residuals():
    name = "zeldovich512_lognormal5"
    w = synth.WORKLOADS[name]
    p = synth.workload(name)
    n = p.n
    ctx = gr.Context(n)
    src = ctx.deposit(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.u).cuda(), p.mass)
    fld = ctx.initial_fields()
    rep = ctx.solve(src, fld, tol=w["tol"], max_cycles=60, prec="mixed_df", rho_hat=p.rho_hat)
    assert rep["status_code"] == gr.GR_OK and max(rep["res"]) <= w["tol"]
    gsrc = {k: v.cpu().numpy() for k, v in src.items()}
    gfld = {k: v.cpu().numpy() for k, v in fld.items()}
    ctx.close()
    del src, fld
    osrc = oracle.deposit(n, p.x, p.u, p.mass)
    for k in oracle.SOURCES:
        assert np.abs(gsrc[k] - osrc[k]).max() <= 1e-12 * np.abs(osrc[k]).max(), k
    cells = np.random.default_rng(0).choice(n ** 3, 20000, replace=False)
    for e, nm in enumerate(oracle.EQUATIONS):
        eps, f = oracle.residual_at(e, osrc, gfld, p.rho_hat, cells)
        rel = np.sqrt(np.mean(eps ** 2)) / np.sqrt(np.mean(f ** 2))
        assert rel <= 3 * w["tol"], (nm, rel)


def test_bench_workload_with_nested_patches():
    """The full-scale configuration with two 128^3 patches (2x and 4x the base
    resolution) centred on the densest base cell, as the bench times it:
    composite solve to 1e-8 on every level; the patch deposits equal the
    oracle's windows of the full-resolution deposit; on the finest patch the
    oracle's pointwise residual of every equation, with ghosts interpolated
    afresh from the GPU's patch-1 solution, is at the tolerance's level
    (Poisson-type equations after their uniform solvability constant)."""
    name = "zeldovich512_lognormal5"
    w = synth.WORKLOADS[name]
    p = synth.workload(name)
    n = p.n
    ctx = gr.Context(n)
    x, u = torch.from_numpy(p.x).cuda(), torch.from_numpy(p.u).cuda()
    src = ctx.deposit(x, u, p.mass)
    c = int(torch.argmax(src["s0"]).item())
    chain = gr.centred_chain(n, (c // (n * n), (c // n) % n, c % n), (128, 128))
    ctx.deposit_patches(chain, x, u, p.mass)
    ctx.initial_patch_fields(chain)
    fld = ctx.initial_fields()
    rep = ctx.solve(src, fld, tol=w["tol"], max_cycles=60, prec="mixed_df", rho_hat=p.rho_hat, patches=chain)
    assert rep["status_code"] == gr.GR_OK
    assert max(max(r[:3]) for r in rep["res_level"]) <= w["tol"]
    gsrc = [{k: v.cpu().numpy() for k, v in q["src"].items()} for q in chain]
    gfld = [{k: v.cpu().numpy() for k, v in q["fld"].items()} for q in chain]
    ctx.close()
    del src, fld
    osrc = oracle.deposit_patches(n, chain, p.x, p.u, p.mass)
    for g, o in zip(gsrc, osrc):
        for k in oracle.SOURCES:
            assert np.abs(g[k] - o[k]).max() <= 1e-12 * np.abs(o[k]).max(), k
    base = oracle.deposit(n, p.x, p.u, p.mass)
    smeans = [float(base[k].mean()) for k in ("sx", "sy", "sz")]
    del base
    G = {k: oracle.patch_ghosted(gfld[1][k], chain[1]["origin"], gfld[0][k], False) for k in oracle.FIELDS}
    cells = np.random.default_rng(1).choice(128 ** 3, 20000, replace=False)
    for e, nm in enumerate(oracle.EQUATIONS):
        eps, f = oracle.patch_residual_at(e, 128, 4.0 * n, osrc[1], G, smeans[e] if e <= 2 else 0.0, p.rho_hat, cells)
        if e not in (4, 5):
            eps = eps - eps.mean()
        r = np.sqrt(np.mean(eps ** 2)) / max(np.sqrt(np.mean(f ** 2)), 1e-300)
        assert r <= 3e-8, (nm, r)
