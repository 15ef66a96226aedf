"""The coarse levels 64^3 .. 2^3 in one 16-CTA thread-block cluster
(k_coarse_cluster): slabs of the 64^3 and 32^3 levels in the CTAs' shared
memory, neighbour planes read through distributed shared memory, the 16^3 ..
2^3 tail in CTA 0.  Cell by cell it performs the operations of the per-level
colour pass, restriction and prolongation kernels in their order, so whole
solves with it (GR_COARSE_CLUSTER=1, read when a context is created; it is
off by default, being measured slower than the per-level launches) and
without it give the same fields bit for bit with the same cycle counts; the
profile shows one coarse launch per cycle in place of the per-level ones."""
import os

import pytest

from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402


def _ctx(n, cluster):
    old = os.environ.get("GR_COARSE_CLUSTER")
    os.environ["GR_COARSE_CLUSTER"] = "1" if cluster else "0"
    try:
        return gr.Context(n)
    finally:
        if old is None:
            os.environ.pop("GR_COARSE_CLUSTER", None)
        else:
            os.environ["GR_COARSE_CLUSTER"] = old


def _solve_both(n, prec, sigma=2.0, **kw):
    out = []
    src = None  # one deposit for both (its atomic additions are not ordered)
    for cluster in (True, False):
        ctx = _ctx(n, cluster)
        if src is None:
            x, u, mass = synth.zeldovich_torch(n, 21, sigma, 0.01, True)
            src = ctx.deposit(x, u, mass)
        fld = ctx.initial_fields()
        rep = ctx.solve(src, fld, prec=prec, rho_hat=synth.RHO_BAR, profile=1, **kw)
        torch.cuda.synchronize()
        out.append((fld, rep))
        ctx.close()
    return out


@pytest.mark.parametrize("prec", ["mixed_df", "mixed"])
@pytest.mark.parametrize("n,fmg", [(128, 0), (128, 1), (256, 0)])
def test_cluster_levels_give_the_per_level_fields_bit_for_bit(n, prec, fmg):
    (fa, ra), (fb, rb) = _solve_both(n, prec, tol=1e-9, max_cycles=40, fmg=fmg)
    assert ra["status_code"] == gr.GR_OK and rb["status_code"] == gr.GR_OK
    assert ra["cycles"] == rb["cycles"]
    for k in fa:
        assert torch.equal(fa[k], fb[k]), k
    # the per-level path spends more coarse launches on the same cycles
    assert ra["prof"]["coarse"]["launches"] < rb["prof"]["coarse"]["launches"]


def test_cluster_path_off_below_128_cubed():
    """A 64^3 top level has no 64^3 interior level: both contexts take the
    same launches."""
    (fa, ra), (fb, rb) = _solve_both(64, "mixed_df", tol=1e-9, max_cycles=40)
    assert ra["cycles"] == rb["cycles"]
    assert ra["prof"]["coarse"]["launches"] == rb["prof"]["coarse"]["launches"]
    for k in fa:
        assert torch.equal(fa[k], fb[k]), k
