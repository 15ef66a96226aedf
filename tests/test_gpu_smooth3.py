"""The fused three-colour-pass smoother (k_smooth3): three red-black passes of
the FP32 correction equation in one pass over memory, with shared-memory
staging of the input planes.  It performs the same floating-point operations
on the same operands as the three separate passes, so whole solves with and
without it must give the same fields bit for bit, in every mode that uses it,
with the same cycle counts; the profile must show the fused launches.
GR_SMOOTH3=1 turns the fused passes on (they are off by default: measured at
512^3 they take as long as the separate passes, both being bound by the SM's
L1/shared-memory pipe); GR_SMOOTH3_MIN lowers the grid size from which
contexts fuse (512 by default) so the small grids exercise the kernel's
wrap-around and tiling."""
import os

import pytest

from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402


def _ctx(n, fused, min_n=64):
    keys = ("GR_SMOOTH3", "GR_SMOOTH3_MIN")
    old = {k: os.environ.get(k) for k in keys}
    os.environ["GR_SMOOTH3"] = "1" if fused else "0"
    os.environ["GR_SMOOTH3_MIN"] = str(min_n)
    try:
        return gr.Context(n)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _sources(ctx, n, seed, sigma):
    x, u, mass = synth.zeldovich_torch(n, seed, sigma, 0.01, True)
    return ctx.deposit(x, u, mass)


def _solve_both(n, prec, min_n=64, **kw):
    out = []
    src = None  # one deposit for both (its atomic additions are not ordered)
    for fused in (True, False):
        ctx = _ctx(n, fused, min_n)
        if src is None:
            src = _sources(ctx, n, 11, 2.0)
        fld = ctx.initial_fields()
        rep = ctx.solve(src, fld, prec=prec, rho_hat=synth.RHO_BAR, profile=1, **kw)
        torch.cuda.synchronize()
        out.append((fld, rep))
        ctx.close()
    return out


@pytest.mark.parametrize("prec", ["mixed_df", "mixed"])
@pytest.mark.parametrize("n,fmg", [(64, 0), (128, 0), (128, 1)])
def test_fused_passes_give_the_separate_passes_fields_bit_for_bit(n, prec, fmg):
    (fa, ra), (fb, rb) = _solve_both(n, prec, tol=1e-9, max_cycles=40, fmg=fmg)
    assert ra["status_code"] == gr.GR_OK and rb["status_code"] == gr.GR_OK
    assert ra["cycles"] == rb["cycles"]
    assert ra["prof"]["smooth3"]["launches"] > 0
    assert rb["prof"]["smooth3"]["launches"] == 0
    for k in fa:
        assert torch.equal(fa[k], fb[k]), k


def test_fused_passes_at_512_cubed():
    """The configuration GR_SMOOTH3=1 gives without GR_SMOOTH3_MIN: fused at 512^3."""
    (fa, ra), (fb, rb) = _solve_both(512, "mixed_df", min_n=512, tol=1e-8, max_cycles=30)
    assert ra["status_code"] == gr.GR_OK and rb["status_code"] == gr.GR_OK
    assert ra["cycles"] == rb["cycles"]
    # two fused launches per correction cycle of every equation
    assert ra["prof"]["smooth3"]["launches"] == 2 * sum(ra["cycles"])
    for k in fa:
        assert torch.equal(fa[k], fb[k]), k
