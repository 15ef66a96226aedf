"""Oracle pin of the whole ten-equation chain by a discrete manufactured
solution (Sec. 2.4 solution sequence; Sec. 4.3.1 Eqs. MG-linear-1a,
MG-linear-1, MG-linear-2a, MG-linear-2, Aij-discrete, Aij-discrete-2,
U-cross-deriv; Eqs. sol-scheme-H-constraint and sol-scheme-CMC).

Smooth V*, psi*, alpha psi* are chosen; every other field and every source is
built here from the paper's discrete formulas with numpy stencils written for
this test (np.roll), independently of the oracle's C code:

  s_i   = lap_h V*_i / (8 pi)                         (V*_i mean-free)
  U*    : lap_h U* = -1/4 div3 V*                     (FFT, discrete symbol)
  A_ij  = D_i V_j + D_j V_i - 1/2 delta_ij div3 V + 2 D_ij U
  s0    : from the psi equation at psi*
  sigma : from the lapse equation at psi*, alpha psi*
  B*^i  : lap_h B*^i = 2 D_j (alpha psi* psi*^-7 A^ij)   (FFT)
  b*    : lap_h b* = -1/4 div3 B*                       (FFT)

The oracle's ten-equation solve from the plain guess must return every
starred field.  Each field feeds a later equation's source through one named
slot (V -> U, (V, U) -> A -> psi, psi -> lapse, (A, psi, alpha psi) -> B,
B -> b), so a field put in the wrong slot, a swapped psi / alpha psi in the
shift source or a dropped term changes a returned field far above the
solver's tolerance."""
import numpy as np
import pytest

from test_oracle_linear import fft_solve

RHO = 1.0 / (24.0 * np.pi)


def _D(f, a, n):  # 3-point central difference along axis a (Eq. Aij-discrete)
    return (np.roll(f, -1, a) - np.roll(f, 1, a)) * (0.5 * n)


def _D2(f, a, n):  # 3-point second difference along axis a
    return (np.roll(f, -1, a) - 2.0 * f + np.roll(f, 1, a)) * (n * n)


def _Dx(f, a, b, n):  # 4-cell cross difference in the (a, b) plane (Eq. U-cross-deriv)
    pp = np.roll(np.roll(f, -1, a), -1, b)
    mm = np.roll(np.roll(f, 1, a), 1, b)
    mp = np.roll(np.roll(f, 1, a), -1, b)
    pm = np.roll(np.roll(f, -1, a), 1, b)
    return (pp + mm - mp - pm) * (0.25 * n * n)


def _lap(f, n):
    return sum(_D2(f, a, n) for a in range(3))


def _div(F, n):
    return sum(_D(F[a], a, n) for a in range(3))


def _aij(V, U, n):
    """Eq. Aij-discrete-2: returns the symmetric 3x3 table of arrays."""
    dv = _div(V, n)
    A = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(i, 3):
            a = _D(V[j], i, n) + _D(V[i], j, n)
            if i == j:
                a = a - 0.5 * dv + 2.0 * _D2(U, i, n)
            else:
                a = a + 2.0 * _Dx(U, i, j, n)
            A[i][j] = A[j][i] = a
    return A


def _smooth(n, seed, amp, modes=3, mmax=2):
    """Sum of a few low Fourier modes (wavenumbers 1..mmax per axis) with
    seeded phases, mean zero, scaled to max |f| = amp."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = np.zeros((n, n, n))
    for _ in range(modes):
        m = rng.integers(1, mmax + 1, size=3)
        ph = rng.random(3) * 2 * np.pi
        f += rng.standard_normal() * np.cos(2 * np.pi * m[0] * X + ph[0]) * np.cos(2 * np.pi * m[1] * Y + ph[1]) \
            * np.cos(2 * np.pi * m[2] * Z + ph[2])
    f -= f.mean()
    return amp * f / np.abs(f).max()


def manufactured(n, seed=0, v_amp=2e-3, psi_amp=1e-4, apsi_amp=2e-3):
    # amplitudes keep s0 > 0 and the lapse coefficient m > 0 (lap psi and
    # lap alpha psi stay below 2 pi rho and Kdot)
    V = [_smooth(n, seed + 1 + a, v_amp) for a in range(3)]
    psi = 1.0 + _smooth(n, seed + 10, psi_amp, mmax=1)
    apsi = 1.0 + _smooth(n, seed + 20, apsi_amp, mmax=1)
    s = [_lap(V[a], n) / (8 * np.pi) for a in range(3)]
    U = fft_solve(-0.25 * _div(V, n))
    A = _aij(V, U, n)
    AA = sum(A[i][i] ** 2 for i in range(3)) + 2 * (A[0][1] ** 2 + A[0][2] ** 2 + A[1][2] ** 2)
    # psi equation: lap psi = -2 pi s0 / psi - AA / (8 psi^7) + 2 pi rho psi^5
    s0 = psi / (2 * np.pi) * (-_lap(psi, n) - AA / (8 * psi**7) + 2 * np.pi * RHO * psi**5)
    # lapse equation: lap(alpha psi) = m alpha psi - psi^5 Kdot with
    # m = 2 pi psi^-2 (s0 + 2 psi^-4 sigma) + 7/8 psi^-8 AA + 5/12 psi^4 K^2
    K2, Kdot = 24 * np.pi * RHO, 12 * np.pi * RHO
    m = (_lap(apsi, n) + psi**5 * Kdot) / apsi
    sigma = (m - 7.0 / 8.0 * AA / psi**8 - 5.0 / 12.0 * psi**4 * K2 - 2 * np.pi * s0 / psi**2) * psi**6 / (4 * np.pi)
    # shift: lap B^i = 2 D_j (alpha psi^-6 A^ij) with alpha = (alpha psi)/psi
    w = apsi / psi**7
    B = [fft_solve(2.0 * sum(_D(w * A[i][j], j, n) for j in range(3))) for i in range(3)]
    b = fft_solve(-0.25 * _div(B, n))
    src = {"s0": s0, "sx": s[0], "sy": s[1], "sz": s[2], "sigma": sigma}
    fld = {"psi": psi, "apsi": apsi, "Vx": V[0], "Vy": V[1], "Vz": V[2], "U": U, "Bx": B[0], "By": B[1], "Bz": B[2],
           "b": b}
    return src, fld, m


def _dev(k, a):
    return a - 1.0 if k in ("psi", "apsi") else a


@pytest.mark.parametrize("n", [16, 32])
def test_ten_equation_chain_returns_the_manufactured_fields(orc, n):
    src, want, m = manufactured(n, seed=3 * n)
    assert m.min() > 0 and src["s0"].min() > 0  # a well-posed lapse equation, positive density
    for k in ("Bx", "By", "Bz", "b", "U"):  # every derived field is non-trivial
        assert np.abs(want[k]).max() > 1e-6 * np.abs(want["Vx"]).max(), k
    fld = orc.initial_fields(n)
    st, rep = orc.solve_constraints(src, fld, RHO, tol=1e-13, max_cycles=80)
    assert st == 0, rep
    for k in orc.FIELDS:
        w, g = _dev(k, want[k]), _dev(k, fld[k])
        err = np.abs(g - w).max() / np.abs(w).max()
        assert err <= 1e-9, (k, err)


def test_chain_pin_sees_a_swap_of_psi_and_alpha_psi_in_the_shift_source():
    """The shift source of the manufactured problem moves by far more than the
    tolerance above if psi and alpha psi trade places in it: the pin above
    would catch such a wiring mistake in the oracle."""
    n = 16
    src, want, _ = manufactured(n, seed=48)
    V = [want["Vx"], want["Vy"], want["Vz"]]
    A = _aij(V, want["U"], n)
    good = [2.0 * sum(_D(want["apsi"] / want["psi"] ** 7 * A[i][j], j, n) for j in range(3)) for i in range(3)]
    bad = [2.0 * sum(_D(want["psi"] / want["apsi"] ** 7 * A[i][j], j, n) for j in range(3)) for i in range(3)]
    for i in range(3):
        Bg, Bb = fft_solve(good[i]), fft_solve(bad[i])
        assert np.abs(Bb - Bg).max() > 1e-3 * np.abs(Bg).max()
