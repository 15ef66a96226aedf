"""Oracle pins of the particle update (Sec. 4.4 Eqs. geodesic-acceleration,
3-velocity, force, Lorentz-factor, coeff_j, coeff_4, coeff_5; App. A Eqs.
GR-K1, GR-D, GR-K2) and of the deposit with the metric (Sec. 4.5).

The expected values come from what the paper and the mathematics fix, not
from the oracle's own formulas:
  * the geodesic equation and 3-velocity of Sec. 3 (Eqs. geodesic-eq,
    3-velocity-1, written with u^0 and d_i gamma^jk), which the five-substep
    split of Sec. 4.4 must reproduce term by term;
  * the interpolation to a particle is the transpose of the (already pinned)
    cloud-in-cell deposit: sum_c g_c s0_c h^3 / m for a lone particle at rest;
  * exact invariants: uniform fields move a particle on a straight line,
    fields that vary along x alone leave u_y and u_z untouched;
  * convergence of whole trajectories to scipy's integration of the Sec. 3
    equations in analytic fields: second order in h, first order in dt
    (the drift takes the fields at the old position, App. A)."""
import numpy as np
import pytest

RHO = 1.0 / (24.0 * np.pi)
TP = 2 * np.pi


def _roll_d(f, a, n):  # 3-point central difference (Sec. 4.3.1)
    return (np.roll(f, -1, a) - np.roll(f, 1, a)) * (0.5 * n)


def _fields(orc, n, psi=1.0, alpha=1.0, B=(0.0, 0.0, 0.0), b=0.0):
    f = orc.initial_fields(n)
    f["psi"][:] = psi
    f["apsi"][:] = np.asarray(alpha) * np.asarray(psi)
    for k, v in zip(("Bx", "By", "Bz"), B):
        f[k][:] = v
    f["b"][:] = b
    return f


def _grid_coords(n):
    c = (np.arange(n) + 0.5) / n
    return np.meshgrid(c, c, c, indexing="ij")


def _interp(orc, n, g, xp):
    """Value of grid array g at xp by the transpose of the deposit (a lone
    particle at rest, unit mass: s0 h^3 are its cloud-in-cell weights)."""
    s = orc.deposit(n, xp.reshape(3, 1), np.zeros((3, 1)), 1.0)["s0"] / n**3
    assert abs(s.sum() - 1) < 1e-14
    return float((g * s).sum())


def _rand_particles(rng, npart, umax):
    return rng.random((3, npart)), umax * (2 * rng.random((3, npart)) - 1)


def test_free_particle_in_uniform_fields(orc):
    """Uniform psi, alpha, beta: no force; the drift is the 3-velocity of
    Eq. 3-velocity-1, gamma^ij u_j / u^0 - beta^i with u^0 = alpha^-1 W."""
    n = 8
    psi, alpha, beta = 1.1, 0.9, np.array([0.01, -0.02, 0.005])
    f = _fields(orc, n, psi, alpha, beta)
    rng = np.random.default_rng(1)
    x, u = _rand_particles(rng, 50, 0.5)
    x0, u0 = x.copy(), u.copy()
    dt, steps = 0.01, 7
    for _ in range(steps):
        orc.particle_update(f, x, u, dt)
    assert np.array_equal(u, u0)
    up0 = np.sqrt(1 + (u0**2).sum(0) / psi**4) / alpha
    v = u0 / psi**4 / up0 - beta[:, None]
    d = (x - (x0 + steps * dt * v)) % 1.0
    d = np.minimum(d, 1 - d)
    assert d.max() < 1e-14


def test_alpha_term_is_the_interpolated_gradient_at_rest(orc):
    """psi = 1, beta = 0, a particle at rest: the opening kick is
    -dt/2 grad alpha at the particle (W = 1), with grad alpha the central
    difference of alpha = (alpha psi)/psi interpolated by the deposit's
    transpose."""
    n = 16
    X, Y, Z = _grid_coords(n)
    alpha = 1 + 0.01 * np.sin(TP * (X + 2 * Y)) * np.cos(TP * Z) + 0.004 * np.cos(TP * 3 * Y)
    f = _fields(orc, n, alpha=alpha)
    rng = np.random.default_rng(2)
    x, u = rng.random((3, 40)), np.zeros((3, 40))
    x0 = x.copy()
    dt = 0.3
    orc.particle_update(f, x, u, dt, sync=False, open_=True, drift=False)
    assert np.array_equal(x, x0)
    for p in range(40):
        for i in range(3):
            want = -0.5 * dt * _interp(orc, n, _roll_d(alpha, i, n), x0[:, p])
            assert u[i, p] == pytest.approx(want, rel=1e-12, abs=1e-18)


def test_psi_term_matches_the_geodesic_equation(orc):
    """alpha = 1, beta = 0, relativistic u: one kick adds dt/2 times the
    last term of Eq. geodesic-eq, -(u_j u_k / 2u^0) d_i gamma^jk with
    gamma^jk = psi^-4 delta^jk, u^0 = W/alpha (Sec. 3), against the c_4 f_4
    substep of Sec. 4.4."""
    n = 16
    X, Y, Z = _grid_coords(n)
    psi = 1 + 0.02 * np.cos(TP * (Y - Z)) + 0.01 * np.sin(TP * 2 * X)
    f = _fields(orc, n, psi=psi)
    rng = np.random.default_rng(3)
    x, u = _rand_particles(rng, 30, 0.4)
    x0, u0 = x.copy(), u.copy()
    dt = 1e-3
    for sync, opn in ((True, False), (False, True)):
        u = u0.copy()
        orc.particle_update(f, x, u, dt, sync=sync, open_=opn, drift=False)
        for p in range(30):
            ps = _interp(orc, n, psi, x0[:, p])
            dps = np.array([_interp(orc, n, _roll_d(psi, i, n), x0[:, p]) for i in range(3)])
            uu = u0[:, p] @ u0[:, p]
            W = np.sqrt(1 + uu / ps**4)
            d_gamma = -4 * ps**-5 * dps  # d_i of psi^-4
            want = 0.5 * dt * (-(uu / (2 * W)) * d_gamma)  # alpha = 1: u^0 = W
            assert np.allclose(u[:, p] - u0[:, p], want, rtol=1e-9, atol=1e-20)  # u - u0 cancels digits


def test_shift_terms_match_the_geodesic_equation(orc):
    """alpha = psi = 1: the three shift substeps add dt/2 u_j d_i beta^j
    (Eq. geodesic-eq) to first order in dt; beta^j = B^j + d_j b."""
    n = 16
    X, Y, Z = _grid_coords(n)
    B = (0.02 * np.sin(TP * Z), 0.03 * np.cos(TP * (X + Y)), 0.01 * np.sin(TP * 2 * Y))
    b = 0.004 * np.cos(TP * (X - Z)) * np.sin(TP * Y)
    f = _fields(orc, n, B=B, b=b)
    beta = [B[j] + _roll_d(b, j, n) for j in range(3)]
    rng = np.random.default_rng(4)
    x, u0 = _rand_particles(rng, 20, 0.3)
    dt = 1e-5
    for sync, opn in ((True, False), (False, True)):
        u = u0.copy()
        orc.particle_update(f, x, u, dt, sync=sync, open_=opn, drift=False)
        for p in range(20):
            G = np.array([[_interp(orc, n, _roll_d(beta[j], i, n), x[:, p]) for j in range(3)] for i in range(3)])
            want = 0.5 * dt * (G @ u0[:, p])
            # the substeps see each other's changes: O(dt^2) relative to the largest component
            assert np.abs(u[:, p] - u0[:, p] - want).max() <= 1e-5 * np.abs(want).max()
            assert np.abs(want).max() > 1e-9


def test_fields_along_x_alone_leave_transverse_momentum(orc):
    n = 16
    X, _, _ = _grid_coords(n)
    f = _fields(orc, n, psi=1 + 0.02 * np.sin(TP * X), alpha=1 + 0.03 * np.cos(TP * X),
                B=(0.01 * np.sin(TP * 2 * X), 0.02 * np.cos(TP * X), 0.0), b=0.003 * np.sin(TP * X))
    rng = np.random.default_rng(5)
    x, u = _rand_particles(rng, 64, 0.5)
    u0 = u.copy()
    for _ in range(20):
        orc.particle_update(f, x, u, 0.05)
    assert np.array_equal(u[1:], u0[1:])
    assert np.abs(u[0] - u0[0]).max() > 1e-4


A1, P1, B1 = 0.02, 0.01, 0.01


def _analytic(X):
    x, y, z = X
    al = 1 + A1 * np.sin(TP * (x + 2 * y))
    ps = 1 + P1 * np.cos(TP * (y - z))
    be = [B1 * np.sin(TP * z), B1 * np.cos(TP * x), 0.5 * B1 * np.sin(TP * (x + y))]
    return al, ps, be


def _geodesic_rhs(t, Y):
    """Sec. 3 Eqs. geodesic-eq and 3-velocity-1 in the analytic fields."""
    X, u = Y[:3], Y[3:]
    x, y, z = X
    al, ps, be = _analytic(X)
    dal = np.array([A1 * TP * np.cos(TP * (x + 2 * y)), 2 * A1 * TP * np.cos(TP * (x + 2 * y)), 0.0])
    dps = np.array([0.0, -P1 * TP * np.sin(TP * (y - z)), P1 * TP * np.sin(TP * (y - z))])
    dbe = np.array([[0, 0, B1 * TP * np.cos(TP * z)], [-B1 * TP * np.sin(TP * x), 0, 0],
                    [0.5 * B1 * TP * np.cos(TP * (x + y))] * 2 + [0]])  # dbe[j][i] = d_i beta^j
    gi = ps**-4
    u0 = np.sqrt(1 + gi * (u @ u)) / al
    d_gi = -4 * ps**-5 * dps
    du = -al * u0 * dal + dbe.T @ u - (u @ u) / (2 * u0) * d_gi
    dx = gi * u / u0 - np.array(be)
    return np.concatenate([dx, du])


def _kdk(orc, f, g, x0, u0, T, steps):
    dt = T / steps
    x, u = x0.reshape(3, 1).copy(), u0.reshape(3, 1).copy()
    orc.particle_update(f, x, u, dt, sync=False, open_=True, drift=True, fields=g)
    for _ in range(steps - 1):
        orc.particle_update(f, x, u, dt, fields=g)
    orc.particle_update(f, x, u, dt, sync=True, open_=False, drift=False, fields=g)
    return x[:, 0], u[:, 0]


def test_trajectories_converge_to_the_geodesic_equation(orc):
    """Whole kick-drift-kick trajectories in grid samples of analytic fields
    converge to the Sec. 3 equations integrated by scipy: error O(h^2) at
    fixed small dt, and O(dt) at a fine grid."""
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    T = 2.0
    x0, u0 = np.array([0.3, 0.6, 0.1]), np.array([0.2, -0.25, 0.1])
    ex = solve_ivp(_geodesic_rhs, (0, T), np.concatenate([x0, u0]), rtol=1e-12, atol=1e-14).y[:, -1]
    errs = {}
    for n in (32, 64, 128):
        X = _grid_coords(n)
        al, ps, be = _analytic(X)
        f = _fields(orc, n, psi=ps, alpha=al, B=be)
        g = orc.particle_fields(f)
        for steps in (200, 400, 800):
            x, u = _kdk(orc, f, g, x0, u0, T, steps)
            dx = (x - ex[:3] + 0.5) % 1 - 0.5
            errs[n, steps] = (np.abs(dx).max(), np.abs(u - ex[3:]).max(), x, u)
    for k in (0, 1):  # second order in h
        assert errs[64, 800][k] < errs[32, 800][k] / 3
        assert errs[128, 800][k] < errs[64, 800][k] / 3
    assert errs[128, 800][0] < 1e-3 and errs[128, 800][1] < 1.5e-3  # displacement 0.42, velocity change 0.25
    # first order in dt: successive differences at the finest grid halve
    d1 = np.abs(errs[128, 200][2] - errs[128, 400][2]).max()
    d2 = np.abs(errs[128, 400][2] - errs[128, 800][2]).max()
    assert 1.6 < d1 / d2 < 2.6


def test_deposit_with_unit_psi_is_the_plain_deposit(orc):
    rng = np.random.default_rng(6)
    x, u = _rand_particles(rng, 500, 0.4)
    a = orc.deposit(8, x, u, 0.3)
    b = orc.deposit_metric(8, x, u, 0.3, np.ones((8, 8, 8)))
    c = orc.deposit_metric(8, x, u, 0.3, None)
    for k in orc.SOURCES:
        assert np.allclose(a[k], b[k], rtol=1e-15, atol=0) and np.array_equal(a[k], c[k])


def test_deposit_with_uniform_psi_rescales_the_velocities(orc):
    """Sec. 4.5: W = sqrt(1 + psi^-4 |u|^2).  A uniform psi = c gives the
    plain deposit of u / c^2 with s_i scaled by c^2 and sigma by c^4."""
    rng = np.random.default_rng(7)
    x, u = _rand_particles(rng, 500, 0.6)
    c = 1.07
    got = orc.deposit_metric(8, x, u, 0.3, np.full((8, 8, 8), c))
    ref = orc.deposit(8, x, u / c**2, 0.3)
    assert np.allclose(got["s0"], ref["s0"], rtol=1e-14)
    for k in ("sx", "sy", "sz"):
        assert np.allclose(got[k], c**2 * ref[k], rtol=1e-13, atol=1e-13 * np.abs(ref[k]).max())
    assert np.allclose(got["sigma"], c**4 * ref["sigma"], rtol=1e-13)


def test_deposit_takes_psi_at_the_particle(orc):
    """A lone particle: its W uses psi interpolated by the deposit's own
    weights (the transpose pin above)."""
    n = 8
    X, Y, Z = _grid_coords(n)
    psi = 1 + 0.05 * np.sin(TP * X) * np.cos(TP * Y) + 0.02 * np.cos(TP * Z)
    rng = np.random.default_rng(8)
    for _ in range(5):
        x, u = _rand_particles(rng, 1, 0.5)
        got = orc.deposit_metric(n, x, u, 1.0, psi)
        ps = _interp(orc, n, psi, x[:, 0])
        W = np.sqrt(1 + (u[:, 0] @ u[:, 0]) / ps**4)
        assert got["s0"].sum() / n**3 == pytest.approx(W, rel=1e-13)
        assert got["sigma"].sum() / n**3 == pytest.approx((u[:, 0] @ u[:, 0]) / W, rel=1e-13)
