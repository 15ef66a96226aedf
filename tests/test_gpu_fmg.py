"""GPU checks of the full multigrid start (gr_opts.fmg): the first correction
of every equation is a nested-iteration cycle instead of a V-cycle.  It is a
warm start, so the converged fields must be the oracle's, and it must leave a
smaller residual after the first cycle and need no more cycles in total."""
import numpy as np
import pytest

import oracle
from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu(d):
    return {k: _t(v) for k, v in d.items()}


def _np(t):
    return t.cpu().numpy()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _problem(n, seed, sigma):
    p = synth.zeldovich(n, seed, sigma, 0.003, True)
    return p, oracle.deposit(n, p.x, p.u, p.mass)


@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
@pytest.mark.parametrize("n", [32, 64])
def test_fmg_start_converges_to_the_oracle_solution(n, prec):
    p, src = _problem(n, 3, 1.0)
    ofld = oracle.initial_fields(n)
    ost, _ = oracle.solve_constraints(src, ofld, p.rho_hat, tol=1e-12, max_cycles=60)
    assert ost == 0
    ctx = gr.Context(n)
    gf = _gpu(oracle.initial_fields(n))
    rep = ctx.solve(_gpu(src), gf, tol=1e-9, max_cycles=60, prec=prec, rho_hat=p.rho_hat, fmg=1)
    assert rep["status_code"] == gr.GR_OK and max(rep["res"]) <= 1e-9
    for k in oracle.FIELDS:
        assert rel_linf(_np(gf[k]), ofld[k]) <= 1e-8, (k, rel_linf(_np(gf[k]), ofld[k]))
    ctx.close()


@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
def test_fmg_start_deviations_within_1e8(prec):
    """psi - 1 and alpha psi - 1 (and every other field) within 1e-8 of the
    oracle's relative to their own maxima, at residual 1e-11: the relative
    residual measures psi's equation against RMS(2 pi s0) and the lapse's
    against |Kdot|, both some 25 times the deviations' own forcing, so the
    deviations need a tolerance that much tighter than 1e-8."""
    n = 64
    p, src = _problem(n, 3, 1.0)
    ofld = oracle.initial_fields(n)
    assert oracle.solve_constraints(src, ofld, p.rho_hat, tol=1e-13, max_cycles=80)[0] == 0
    ctx = gr.Context(n)
    gf = _gpu(oracle.initial_fields(n))
    rep = ctx.solve(_gpu(src), gf, tol=1e-11, max_cycles=80, prec=prec, rho_hat=p.rho_hat, fmg=1)
    assert rep["status_code"] == gr.GR_OK
    for k in oracle.FIELDS:
        d = 1.0 if k in ("psi", "apsi") else 0.0
        err = rel_linf(_np(gf[k]) - d, ofld[k] - d)
        assert err <= 1e-8, (k, err)
    ctx.close()


def _solve(n, src, rho, **kw):
    ctx = gr.Context(n)
    gf = _gpu(oracle.initial_fields(n))
    rep = ctx.solve(_gpu(src), gf, rho_hat=rho, prec="mixed_df", allow_noconv=True, **kw)
    ctx.close()
    return rep


def test_fmg_first_cycle_leaves_a_smaller_residual():
    """One correction cycle per equation: for the three V_i equations (whose
    sources do not depend on earlier solutions) the nested iteration leaves
    under half the V-cycle's relative residual."""
    n = 128
    p, src = _problem(n, 4, 3.0)
    v = _solve(n, src, p.rho_hat, tol=0.0, max_cycles=1)
    f = _solve(n, src, p.rho_hat, tol=0.0, max_cycles=1, fmg=1)
    for eq in range(3):
        assert f["res"][eq] < 0.5 * v["res"][eq], (eq, f["res"][eq], v["res"][eq])


def test_fmg_needs_no_more_cycles():
    n = 128
    p, src = _problem(n, 5, 3.0)
    v = _solve(n, src, p.rho_hat, tol=1e-8, max_cycles=60)
    f = _solve(n, src, p.rho_hat, tol=1e-8, max_cycles=60, fmg=1)
    assert v["status_code"] == f["status_code"] == gr.GR_OK
    assert all(a <= b for a, b in zip(f["cycles"], v["cycles"])), (f["cycles"], v["cycles"])
    assert sum(f["cycles"]) < sum(v["cycles"])


def test_fmg_is_ignored_below_32_cubed():
    """Grids without the 16^3 coarse tail keep the V-cycle start."""
    n = 16
    p, src = _problem(n, 6, 1.0)
    v = _solve(n, src, p.rho_hat, tol=1e-9, max_cycles=60)
    f = _solve(n, src, p.rho_hat, tol=1e-9, max_cycles=60, fmg=1)
    assert f["cycles"] == v["cycles"] and f["res"] == v["res"]
