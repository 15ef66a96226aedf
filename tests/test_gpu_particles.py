"""GPU parity of the particle update (gr_particle_update, gr_kick, gr_drift)
and of the deposit with the metric (gr_deposit_metric) against the FP64
oracle, and a short time loop (Sec. 4.2 steps 3 and 5-8) on both sides.

Tolerance of the update: the GPU interpolates the 20 grid quantities and
runs the substeps in FP32 (positions and velocities accumulate in FP64), so
each velocity or position change carries a relative error of a few tens of
FP32 roundings (2^-24 = 6e-8 each, over an 8-term weighted sum and about ten
dependent operations); the bar is 2e-5 of the largest change of that
component over all particles, with an FP64 floor for the unchanged digits."""
import numpy as np
import pytest

import oracle
from paper_1905_08890_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402

TP = 2 * np.pi
BAR = 2e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _coords(n):
    c = (np.arange(n) + 0.5) / n
    return np.meshgrid(c, c, c, indexing="ij")


def _strong_fields(n):
    """Smooth fields with every term of the kick well above the bar."""
    X, Y, Z = _coords(n)
    f = oracle.initial_fields(n)
    psi = 1 + 0.02 * np.cos(TP * (Y - Z)) + 0.01 * np.sin(TP * 2 * X)
    alpha = 1 + 0.03 * np.sin(TP * (X + 2 * Y)) * np.cos(TP * Z)
    f["psi"][:] = psi
    f["apsi"][:] = alpha * psi
    f["Bx"][:] = 0.02 * np.sin(TP * Z)
    f["By"][:] = 0.03 * np.cos(TP * (X + Y))
    f["Bz"][:] = 0.01 * np.sin(TP * 2 * Y)
    f["b"][:] = 0.004 * np.cos(TP * (X - Z)) * np.sin(TP * Y)
    return f


def _wrapdiff(a, b):
    return (a - b + 0.5) % 1.0 - 0.5


def _compare(x0, u0, xg, ug, xo, uo):
    for d in range(3):
        du_o = uo[d] - u0[d]
        err = np.abs((ug[d] - u0[d]) - du_o).max()
        assert err <= BAR * np.abs(du_o).max() + 4e-16 * np.abs(u0[d]).max(), ("u", d, err, np.abs(du_o).max())
        dx_o = _wrapdiff(xo[d], x0[d])
        err = np.abs(_wrapdiff(xg[d], xo[d])).max()
        assert err <= BAR * np.abs(dx_o).max() + 4e-16, ("x", d, err, np.abs(dx_o).max())


def _run_both(n, fld_np, x0, u0, dt, flags):
    ctx = gr.Context(n)
    xg, ug = _t(x0), _t(u0)
    ctx.particle_update(xg, ug, {k: _t(v) for k, v in fld_np.items()}, dt, flags)
    torch.cuda.synchronize()
    xo, uo = x0.copy(), u0.copy()
    oracle.particle_update(fld_np, xo, uo, dt, sync=bool(flags & gr.GR_KICK_SYNC), open_=bool(flags & gr.GR_KICK_OPEN),
                           drift=bool(flags & gr.GR_DRIFT))
    ctx.close()
    return xg.cpu().numpy(), ug.cpu().numpy(), xo, uo


@pytest.mark.parametrize("flags", [gr.GR_KICK_SYNC, gr.GR_KICK_OPEN, gr.GR_DRIFT,
                                   gr.GR_KICK_SYNC | gr.GR_KICK_OPEN | gr.GR_DRIFT])
@pytest.mark.parametrize("n,npart", [(16, 1000), (32, 12345)])
def test_update_matches_oracle_in_strong_fields(n, npart, flags):
    """Relativistic velocities (|u| up to 0.5) in smooth fields of a few per
    cent; a particle count that leaves a ragged last block; particles on
    the box faces and cell centres (wrap and zero fractions)."""
    rng = np.random.default_rng(npart + flags)
    x0 = rng.random((3, npart))
    x0[:, :4] = [[0.0, 1 - 1e-16, 0.5 / n, 0.999], [0.0, 0.25, 0.5 / n, 1 - 1e-16], [0.0, 0.5, 0.5 / n, 0.0]]
    u0 = 0.5 * (2 * rng.random((3, npart)) - 1)
    fld = _strong_fields(n)
    xg, ug, xo, uo = _run_both(n, fld, x0, u0, 0.05, flags)
    if not flags & gr.GR_DRIFT:
        assert np.array_equal(xg, x0)
    if not flags & (gr.GR_KICK_SYNC | gr.GR_KICK_OPEN):
        assert np.array_equal(ug, u0)
    assert np.all((xg >= 0) & (xg <= 1))
    _compare(x0, u0, xg, ug, xo, uo)


def test_update_in_solved_fields_of_zeldovich_particles():
    """The fields of an oracle solve of Zel'dovich sources (rms delta 1,
    rms |u| 0.01) and the same particles: one full update."""
    n = 32
    p = synth.zeldovich(n, 21, 1.0, 0.01, True)
    src = oracle.deposit(n, p.x, p.u, p.mass)
    fld = oracle.initial_fields(n)
    st, _ = oracle.solve_constraints(src, fld, p.rho_hat, tol=1e-12, max_cycles=60)
    assert st == 0
    dt = 0.05 / n / 0.01  # 0.05 cells at the rms speed
    xg, ug, xo, uo = _run_both(n, fld, p.x, p.u, dt, gr.GR_KICK_SYNC | gr.GR_KICK_OPEN | gr.GR_DRIFT)
    _compare(p.x, p.u, xg, ug, xo, uo)
    assert np.abs(uo - p.u).max() > 1e-9  # the kick is not empty


def test_kick_and_drift_entry_points_equal_the_fused_update():
    n = 16
    rng = np.random.default_rng(3)
    x0, u0 = rng.random((3, 777)), 0.3 * (2 * rng.random((3, 777)) - 1)
    fld = {k: _t(v) for k, v in _strong_fields(n).items()}
    ctx = gr.Context(n)
    xa, ua = _t(x0), _t(u0)
    ctx.particle_update(xa, ua, fld, 0.04)
    xb, ub = _t(x0), _t(u0)
    gr.gr_kick(ctx.h, xb, ub, fld, 0.04, gr.GR_KICK_SYNC | gr.GR_KICK_OPEN)
    gr.gr_drift(ctx.h, xb, ub, fld, 0.04)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    # the fused drift takes the kicked velocity before its FP64 rounding
    dx = (_wrapdiff(xa.cpu().numpy(), x0))
    assert np.abs(_wrapdiff(xa.cpu().numpy(), xb.cpu().numpy())).max() <= 1e-6 * np.abs(dx).max()
    ctx.particle_update(xa[:, :0].contiguous(), ua[:, :0].contiguous(), fld, 0.04)  # np = 0: nothing to do
    with pytest.raises(gr.GRError) as ei:
        gr.gr_kick(ctx.h, xb, ub, fld, 0.04, gr.GR_DRIFT)
    assert ei.value.status == gr.GR_ERR_ARG
    with pytest.raises(gr.GRError):
        ctx.particle_update(xb, ub, fld, float("nan"))
    ctx.close()


@pytest.mark.parametrize("n,npart", [(8, 1), (32, 20000)])
def test_deposit_metric_matches_oracle(n, npart):
    rng = np.random.default_rng(n)
    x = rng.random((3, npart))
    u = 0.4 * (2 * rng.random((3, npart)) - 1)
    psi = _strong_fields(n)["psi"] + 0.05 * _coords(n)[0] ** 2
    want = oracle.deposit_metric(n, x, u, 0.7, psi)
    ctx = gr.Context(n)
    got = ctx.deposit_metric(_t(x), _t(u), 0.7, _t(psi))
    plain = ctx.deposit_metric(_t(x), _t(u), 0.7, None)
    torch.cuda.synchronize()
    ref_plain = oracle.deposit(n, x, u, 0.7)
    for k in oracle.SOURCES:
        g, w = got[k].cpu().numpy(), want[k]
        # FP64 throughout; the atomic adds and the gather's order differ from the oracle's
        assert np.abs(g - w).max() <= 1e-13 * np.abs(w).max(), k
        assert np.abs(plain[k].cpu().numpy() - ref_plain[k]).max() <= 1e-13 * np.abs(ref_plain[k]).max(), k
    ctx.close()


def test_three_step_time_loop_matches_oracle():
    """Sec. 4.2: deposit with the previous psi, solve from the previous
    solution, synchronising + opening kick and drift; three steps at 16^3
    (the first step opens without a synchronising kick), GPU (FP64 solve)
    against the oracle."""
    n = 16
    p = synth.zeldovich(n, 31, 1.0, 0.05, True)
    dt = 0.2 / n / 0.05
    xo, uo = p.x.copy(), p.u.copy()
    fo = oracle.initial_fields(n)
    ctx = gr.Context(n)
    xg, ug = _t(p.x), _t(p.u)
    fg = ctx.initial_fields()
    src = ctx.new_sources()
    steps = []
    for step in range(3):
        so = oracle.deposit_metric(n, xo, uo, p.mass, fo["psi"] if step else None)
        st, _ = oracle.solve_constraints(so, fo, p.rho_hat, tol=1e-12, max_cycles=60)
        assert st == 0
        flags = (gr.GR_KICK_SYNC if step else 0) | gr.GR_KICK_OPEN | gr.GR_DRIFT
        x_before, u_before = xo.copy(), uo.copy()
        oracle.particle_update(fo, xo, uo, dt, sync=step > 0, open_=True, drift=True)
        ctx.deposit_metric(xg, ug, p.mass, fg["psi"] if step else None, src)
        ctx.solve(src, fg, tol=1e-12, max_cycles=60, rho_hat=p.rho_hat)
        ctx.particle_update(xg, ug, fg, dt, flags)
        torch.cuda.synchronize()
        for k in oracle.FIELDS:
            a, b = fg[k].cpu().numpy(), fo[k]
            assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1e-300), (step, k)
        steps.append((x_before, u_before))
        _compare(x_before, u_before, xg.cpu().numpy(), ug.cpu().numpy(), xo, uo)
        # carry the oracle's state into the next step on both sides, so each
        # step's comparison starts from the same particles and fields
        xg.copy_(_t(xo))
        ug.copy_(_t(uo))
        for k in oracle.FIELDS:
            fg[k].copy_(_t(fo[k]))
    ctx.close()


def test_box_side_scaling_is_exact():
    """A box of side L = 2 with the same grid values of psi, alpha psi and B^i
    and twice those of b: the shift beta = B + grad b is then the same, every
    force term holds one gradient (halved, h doubles), and the CIC position in
    cells is unchanged, so particles at 2x stepped by dt end at exactly twice
    the positions, with exactly the velocities, of particles at x in the unit
    box stepped by dt/2 (all scalings are powers of two).  Particles near the
    faces drift out and must wrap into [0, L)."""
    n, npart = 16, 3000
    rng = np.random.default_rng(11)
    x0 = rng.random((3, npart))
    x0[:, :6] = [[1e-9, 1 - 1e-9, 0.5, 0.999, 0.001, 0.25]] * 3
    u0 = 0.5 * (2 * rng.random((3, npart)) - 1)
    u0[:, :6] = [[-0.4, 0.4, 0.1, 0.4, -0.4, 0.0]] * 3
    f1 = _strong_fields(n)
    fld = {k: _t(v) for k, v in f1.items()}
    fld2 = dict(fld, b=_t(2 * f1["b"]))
    dt = 0.05
    flags = gr.GR_KICK_SYNC | gr.GR_KICK_OPEN | gr.GR_DRIFT
    c1, c2 = gr.Context(n), gr.Context(n, L=2.0)
    xa, ua = _t(x0), _t(u0)
    xb, ub = _t(2 * x0), _t(u0)
    c1.particle_update(xa, ua, fld, dt / 2, flags)
    c2.particle_update(xb, ub, fld2, dt, flags)
    torch.cuda.synchronize()
    assert torch.equal(ub, ua)
    assert torch.equal(xb, 2 * xa)
    assert bool(((xb >= 0) & (xb < 2)).all())
    assert bool((xb[:, :6] < 0.1).any() and (xb[:, :6] > 1.9).any())  # some wrapped each way
    c1.close()
    c2.close()
