"""Oracle pins: cloud-in-cell deposit of the conformal sources
(Sec. 3, Eqs. s_0 - s_ij; Sec. 4.1.2, Eqs. s0/si/sij-code-unit-cic)."""
import json
import math
import os

import numpy as np
import pytest

from paper_1905_08890_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_bounds.json")))


def _analytic_per_particle(p):
    u2 = np.sum(p.u * p.u, axis=0)
    W = np.sqrt(1.0 + u2)
    return W, u2


def test_particles_on_cell_centres_deposit_exactly(orc):
    """Sec. 5.1.1 test: uniform particles, u_i = 0.3 sin(2 pi x_i).  A particle
    on a cell centre puts all of its weight in that cell, so every cell equals
    m W / h^3 (etc.) of its own particle; the paper's bound is 1e-5."""
    n = 16
    p = synth.lattice(n, 1, 0.5, velocity=lambda x: 0.3 * np.sin(2 * np.pi * x))
    src = orc.deposit(n, p.x, p.u, p.mass)
    W, u2 = _analytic_per_particle(p)
    vol = 1.0 / n**3
    err = np.abs(src["s0"].reshape(-1) - p.mass * W / vol).max() / synth.RHO_BAR
    assert err < 1e-14 and err < GOLDEN["cic_source_error"]["value"]
    for d, k in enumerate(("sx", "sy", "sz")):
        assert np.allclose(src[k].reshape(-1), p.mass * p.u[d] / vol, rtol=0, atol=1e-15)
    assert np.allclose(src["sigma"].reshape(-1), p.mass * u2 / W / vol, rtol=1e-13, atol=0)


def test_corner_particle_splits_into_eighths(orc):
    n = 8
    x = np.array([[3 / n], [5 / n], [0.0]])  # on a cell corner: halfway between 8 centres
    u = np.array([[0.1], [0.0], [0.0]])
    m = 2.0
    src = orc.deposit(n, x, u, m)
    W = math.sqrt(1.01)
    expect = m * W * n**3 / 8
    nz = np.argwhere(src["s0"] != 0)
    assert len(nz) == 8
    got = sorted(tuple(c) for c in nz)
    want = sorted((i, j, k) for i in (2, 3) for j in (4, 5) for k in (n - 1, 0))
    assert got == want
    assert np.allclose(src["s0"][src["s0"] != 0], expect, rtol=1e-15)


def test_weights_equal_the_cic_tent_function(orc):
    """The f+/f- weights of Sec. 4.1.2 are the CIC tent W(x) = max(0, 1 - |x - x_c|/h)
    per axis (periodic distance) - checked for random single particles."""
    n = 8
    rng = np.random.default_rng(5)
    h = 1.0 / n
    centres = (np.arange(n) + 0.5) * h
    for _ in range(20):
        xp = rng.random(3)
        src = orc.deposit(n, xp.reshape(3, 1), np.zeros((3, 1)), 1.0)
        tent = []
        for a in range(3):
            dist = np.abs(centres - xp[a])
            dist = np.minimum(dist, 1.0 - dist)
            tent.append(np.maximum(0.0, 1.0 - dist / h))
        want = tent[0][:, None, None] * tent[1][None, :, None] * tent[2][None, None, :] / h**3
        assert np.allclose(src["s0"], want, rtol=0, atol=1e-12 * want.max())


def test_conservation_random_particles(orc):
    """sum(s0) h^3 = m sum W, sum(s_l) h^3 = m sum u_l, sum(sigma) h^3 = m sum |u|^2/W."""
    n = 16
    rng = np.random.default_rng(11)
    npart = 5003  # not a multiple of anything
    x = rng.random((3, npart)) * 3.0 - 1.0  # outside [0,1): wrapped periodically
    u = 0.2 * rng.standard_normal((3, npart))
    m = 0.37
    src = orc.deposit(n, x, u, m)
    vol = 1.0 / n**3
    u2 = np.sum(u * u, axis=0)
    W = np.sqrt(1 + u2)
    assert math.isclose(src["s0"].sum() * vol, m * W.sum(), rel_tol=1e-12)
    for d, k in enumerate(("sx", "sy", "sz")):
        assert math.isclose(src[k].sum() * vol, m * u[d].sum(), rel_tol=1e-10, abs_tol=1e-12)
    assert math.isclose(src["sigma"].sum() * vol, m * (u2 / W).sum(), rel_tol=1e-12)
    assert np.all(src["s0"] >= 0) and np.all(src["sigma"] >= 0)


def test_periodic_wrap_equals_shifted_positions(orc):
    n = 8
    rng = np.random.default_rng(3)
    x = rng.random((3, 50))
    u = 0.1 * rng.standard_normal((3, 50))
    a = orc.deposit(n, x, u, 1.0)
    b = orc.deposit(n, x + np.array([[1.0], [-2.0], [3.0]]), u, 1.0)
    for k in orc.SOURCES:
        assert np.allclose(a[k], b[k], rtol=0, atol=1e-12 * np.abs(a[k]).max())


def test_no_particles_gives_zero_sources(orc):
    src = orc.deposit(4, np.zeros((3, 0)), np.zeros((3, 0)), 1.0)
    for k in orc.SOURCES:
        assert not src[k].any()


def test_smooth_velocity_field_converges_second_order(orc):
    """Offset lattice (8 particles per cell) carrying u_i = 0.3 sin(2 pi x_i):
    s_x at the cell centres approaches rho_bar * u_x(x_c) as O(h^2)."""
    errs = []
    for n in (8, 16, 32):
        p = synth.lattice(n, 2, 0.5, velocity=lambda x: 0.3 * np.sin(2 * np.pi * x))
        src = orc.deposit(n, p.x, p.u, p.mass)
        xc = (np.arange(n) + 0.5) / n
        want = synth.RHO_BAR * 0.3 * np.sin(2 * np.pi * xc)[:, None, None] * np.ones((n, n, n))
        errs.append(np.abs(src["sx"] - want).max() / synth.RHO_BAR)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs
