"""GPU parity of the code-unit solve (gr_solve_code_units, Sec. 4.1) against
the oracle's code-unit solve, at the scale factors, matter densities and
Hubble rates of the oracle pins (a = 1 with H0 = 1/3 is the geometric
problem of the other tests; H0 = 0.085 is a 256 Mpc/h box).  Code-unit
fields measure deviations from the homogeneous background, so they are
compared relative to their own maxima: the residual tolerance sets their
accuracy (about 100 times the tolerance, as for psi - 1 in the geometric
form)."""
import numpy as np
import pytest

import oracle
from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402

CASES = [(1.0, 1.0, 1.0 / 3.0), (0.5, 0.3, 0.2), (0.1, 1.0, 1.0 / 3.0), (1.0, 0.3, 0.085)]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _code_problem(n, seed=3, v_rms=0.02):
    p = synth.zeldovich(n, seed, 1.0, v_rms, True)
    s = oracle.deposit(n, p.x, p.u, p.mass)
    return {k: v / p.rho_hat for k, v in s.items()}


@pytest.mark.parametrize("a,Om,H0", CASES)
@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-12, 1e-9), ("mixed_df", 1e-11, 1e-8)])
def test_code_unit_solve_matches_the_oracle(a, Om, H0, prec, tol, bar):
    n = 32
    src = _code_problem(n)
    want = oracle.code_initial_fields(n)
    st, _ = oracle.solve_code_units(src, want, a, Om, H0, tol=1e-13, max_cycles=80)
    assert st == 0
    ctx = gr.Context(n)
    got = {k: _t(v) for k, v in oracle.code_initial_fields(n).items()}
    rep = ctx.solve_code_units({k: _t(v) for k, v in src.items()}, got, a, Om, H0, Omega_L=1 - Om, tol=tol,
                               max_cycles=80, prec=prec)
    assert rep["status_code"] == gr.GR_OK and max(rep["cycles"]) <= 20, rep["cycles"]
    for k in oracle.FIELDS:
        err = rel_linf(got[k].cpu().numpy(), want[k])
        assert err <= bar, (k, err)
    # and the GPU's solution satisfies the paper's printed code-unit equations
    rel = oracle.code_units_residual(src, {k: v.cpu().numpy() for k, v in got.items()}, a, Om, H0)
    assert rel.max() <= 100 * tol + 1e-9, rel
    ctx.close()


def test_code_unit_entry_point_refuses_bad_parameters():
    ctx = gr.Context(8)
    src = {k: torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda") for k in gr.SOURCES}
    fld = {k: torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda") for k in gr.FIELDS}
    for a, Om, H0 in ((0.0, 1.0, 0.3), (1.0, -1.0, 0.3), (1.0, 1.0, 0.0)):
        with pytest.raises(gr.GRError) as ei:
            ctx.solve_code_units(src, fld, a, Om, H0)
        assert ei.value.status == gr.GR_ERR_ARG
    ctx.close()
    ctx2 = gr.Context(8, L=2.0)
    with pytest.raises(gr.GRError):
        ctx2.solve_code_units(src, fld, 1.0, 1.0, 0.3)
    ctx2.close()
