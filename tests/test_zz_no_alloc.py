"""The allocation-free momentum-constraint residual against gr_residual.

gr_momentum_residual_noalloc serves callers that cannot allocate device
memory (their memory belongs to another allocator, or they cannot afford the
device synchronisation of cudaMalloc/cudaFree) and therefore cannot create a
context.  Its scratch is an array compiled into the library and shared by
every call.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects this on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr, synth  # noqa: E402


def _case(n, seed):
    p = synth.zeldovich(n, seed, 1.0, 0.01, True)
    p.u[0] += 0.002  # bulk flow: the momentum source has a non-zero mean
    ctx = gr.Context(n)
    src = ctx.deposit(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.u).cuda(), p.mass)
    fld = ctx.initial_fields()
    ctx.solve(src, fld, tol=0.0, max_cycles=2, rho_hat=p.rho_hat, allow_noconv=True)  # V not converged
    return p, ctx, src, fld


def test_noalloc_residual_matches_gr_residual_on_two_calls_in_a_row():
    # largest grid first, so each later call runs on a scratch array still
    # holding the previous call's partial sums; 256 fills every partial slot
    # (the totals sit right after the last one), 4 is a single part-filled block
    for n, seed, comp in ((256, 10, 1), (64, 11, 0), (32, 12, 2), (4, 13, 0)):
        p, ctx, src, fld = _case(n, seed)
        vname, sname = ("Vx", "Vy", "Vz")[comp], ("sx", "sy", "sz")[comp]
        want = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        rel_want = ctx.residual(gr.GR_VX + comp, src, fld, res_field=want, rho_hat=p.rho_hat)
        got = torch.full((n, n, n), float("nan"), dtype=torch.float64, device="cuda")
        rel_got = gr.gr_momentum_residual_noalloc(n, 1.0, fld[vname], src[sname], got)
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - w).max() <= 1e-12 * np.abs(w).max(), n
        assert rel_got == pytest.approx(rel_want, rel=1e-10), n
        assert 1e-6 < rel_got < 10
        ctx.close()
        del ctx, src, fld, want, got
        torch.cuda.empty_cache()


def test_noalloc_rejects_grids_beyond_its_scratch():
    # straight through the C entry point: it refuses n = 512 before touching the buffers
    import ctypes

    x = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda")
    r = ctypes.c_double(-1.0)
    st = gr.lib().gr_momentum_residual_noalloc(512, 1.0, x.data_ptr(), x.data_ptr(), None, ctypes.byref(r),
                                                torch.cuda.current_stream().cuda_stream)
    assert st == gr.GR_ERR_ARG and "256" in gr.gr_last_error()
    assert r.value == -1.0


def test_noalloc_binding_checks_sizes_and_device():
    x = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        gr.gr_momentum_residual_noalloc(8, 1.0, x, x)  # 64 elements, 8^3 wanted
    with pytest.raises(ValueError):
        gr.gr_momentum_residual_noalloc(4, 1.0, x, x.cpu())
    with pytest.raises(TypeError):
        gr.gr_momentum_residual_noalloc(4, 1.0, x.float(), x)
