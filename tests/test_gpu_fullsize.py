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
