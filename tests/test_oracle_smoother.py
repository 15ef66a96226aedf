"""Oracle pins: the single multigrid steps - Gauss-Seidel/Newton colour pass,
restriction and prolongation (Sec. 4.3.1 relaxation and coarse-grid
correction; R and P are named, not given, in the paper)."""
import numpy as np
import pytest


def _red(n):
    i, j, k = np.indices((n, n, n))
    return (i + j + k) % 2 == 0


@pytest.mark.parametrize("kind", ["POISSON", "HELMHOLTZ"])
def test_linear_colour_pass_zeroes_the_residual_on_that_colour(orc, kind):
    """Gauss-Seidel on a linear equation solves each visited cell's equation
    exactly given its (other-colour) neighbours."""
    n = 8
    rng = np.random.default_rng(0)
    u = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    c0 = 0.5 + rng.random((n, n, n)) if kind == "HELMHOLTZ" else None
    k = getattr(orc, kind)
    orc.gs_colour(k, u, f, c0, color=0)
    eps, _ = orc.residual(k, u, f, c0)
    red = _red(n)
    assert np.abs(eps[red]).max() < 1e-12 * np.abs(f).max() * n * n
    assert np.abs(eps[~red]).max() > 1e-3  # the other colour is untouched


def test_psi_colour_pass_is_a_newton_step(orc):
    """Repeating the red pass with black fixed is Newton's method on each red
    cell's scalar equation: the red residual falls quadratically.  Strong
    nonlinear terms (large rho_hat, s0, AA) make a wrong derivative visible."""
    n = 4
    rng = np.random.default_rng(1)
    rho = 10.0
    s0 = rho * (1 + 0.5 * rng.random((n, n, n)))
    AA = 20 * rng.random((n, n, n))
    f = np.zeros((n, n, n))
    u = 0.1 * rng.random((n, n, n))
    red = _red(n)
    hist = []
    for _ in range(4):
        orc.gs_colour(orc.PSI, u, f, s0, AA, rho, color=0)
        eps, _ = orc.residual(orc.PSI, u, f, s0, AA, rho)
        hist.append(np.abs(eps[red]).max())
    # quadratic: r_{k+1} <= C r_k^2 (C ~ 2e-3 here), down to rounding
    assert hist[1] <= 0.01 * hist[0] ** 2 and hist[2] <= 0.01 * hist[1] ** 2, hist
    assert hist[3] < 1e-12, hist


def test_restriction_is_the_eight_child_average(orc):
    n = 8
    rng = np.random.default_rng(2)
    f = rng.standard_normal((n, n, n))
    R = orc.restrict(f)
    want = f.reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5))
    assert np.allclose(R, want, rtol=0, atol=1e-15)


def test_prolongation_is_cell_centred_trilinear(orc):
    """P reproduces fields that are linear along each axis between coarse
    centres (fine centre 2I + a sits 1/4 of a coarse cell from centre I), and
    preserves the mean of any periodic field."""
    nc = 8
    X = np.arange(nc, dtype=float)
    coarse = 1.0 + 0.5 * X[:, None, None] - 0.25 * X[None, :, None] + 2.0 * X[None, None, :]
    fine = np.zeros((2 * nc,) * 3)
    orc.prolong_add(coarse, fine)
    xf = (np.arange(2 * nc) - 0.5) / 2.0  # fine centres in coarse-index units
    want = 1.0 + 0.5 * xf[:, None, None] - 0.25 * xf[None, :, None] + 2.0 * xf[None, None, :]
    interior = slice(1, 2 * nc - 1)  # away from the periodic wrap of the linear ramp
    assert np.allclose(fine[interior, interior, interior], want[interior, interior, interior], rtol=0, atol=1e-13)
    rng = np.random.default_rng(3)
    c = rng.standard_normal((nc,) * 3)
    fine = np.zeros((2 * nc,) * 3)
    orc.prolong_add(c, fine)
    assert abs(fine.mean() - c.mean()) < 1e-15
