"""Oracle pins of the code-unit form at a fiducial scale factor a (Sec. 4.1
Eqs. Wi-code-units, H-constraint-MG-1, CMC-MG-1, Q-function,
MDC-code-units; Sec. 4.3.1 Eqs. MG-linear-1a, MG-linear-1, MG-linear-2a,
MG-linear-2).

  * a = 1, Omega_m = 1, H0 = 1/3 (ct = 3, rho_c = 1/(24 pi)) is the
    geometric problem the rest of the oracle solves: the code-unit solution
    is that solution under the Sec. 4.1 scalings, to rounding;
  * at several (a, Omega_m, H0) the solution satisfies the paper's printed
    code-unit equations (a different formulation from the geometric Sec. 2.4
    equations the solve uses) to the solve's tolerance;
  * the scale factor is a symmetry of the geometric equations: the solution
    at a with sources (s0, s_i, sigma) equals, with psi = a^(1/2) chi,
    alpha psi = a^(1/2) phi, V = a^2 V', U = a^2 U', B = B'/a, b = b'/a, the
    a = 1 solution (chi, phi, V', U', B', b') of the sources
    (s0/a, s_i/a^2, sigma/a^3) with rho_hat' = a^2 rho_hat(a) (the trace
    s = psi^-4 sigma of the lapse equation scales as s0)."""
import numpy as np
import pytest

from paper_1905_08890_gb300 import synth

CASES = [(1.0, 1.0, 1.0 / 3.0), (0.5, 0.3, 0.2), (0.1, 1.0, 1.0 / 3.0), (2.0, 0.7, 0.05), (1.0, 0.3, 0.085)]


def _code_sources(orc, n, seed=3, v_rms=0.01):
    p = synth.zeldovich(n, seed, 1.0, v_rms, True)
    s = orc.deposit(n, p.x, p.u, p.mass)
    return {k: v / p.rho_hat for k, v in s.items()}, p  # mean st0 close to 1 (rho_hat = rho_c at a = 1)


def test_code_units_at_a_equal_1_are_the_geometric_problem(orc):
    n = 16
    src, p = _code_sources(orc, n)
    fc = orc.code_initial_fields(n)
    st, rep = orc.solve_code_units(src, fc, 1.0, 1.0, 1.0 / 3.0, tol=1e-12, max_cycles=60)
    assert st == 0, rep
    geo = orc.initial_fields(n)
    st, _ = orc.solve_constraints({k: v * p.rho_hat for k, v in src.items()}, geo, p.rho_hat, tol=1e-12,
                                  max_cycles=60)
    assert st == 0
    ct = 3.0
    want = {"psi": 2 * ct**2 * (1 - geo["psi"]), "apsi": ct**2 * (geo["apsi"] / geo["psi"] - 1)}
    for k in ("Vx", "Vy", "Vz", "U"):
        want[k] = ct**2 * geo[k]
    for k in ("Bx", "By", "Bz", "b"):
        want[k] = ct * geo[k]
    for k in orc.FIELDS:
        assert np.abs(fc[k] - want[k]).max() <= 1e-10 * np.abs(want[k]).max(), k


@pytest.mark.parametrize("a,Om,H0", CASES)
def test_solution_satisfies_the_printed_code_unit_equations(orc, a, Om, H0):
    n = 16
    src, _ = _code_sources(orc, n, v_rms=0.05)
    fc = orc.code_initial_fields(n)
    st, rep = orc.solve_code_units(src, fc, a, Om, H0, tol=1e-12, max_cycles=80)
    assert st == 0, rep
    rel = orc.code_units_residual(src, fc, a, Om, H0)
    assert rel.max() <= 1e-9, rel
    # the plain guess is far from satisfying them: the check has teeth
    rel0 = orc.code_units_residual(src, orc.code_initial_fields(n), a, Om, H0)
    assert rel0[[0, 1, 2, 4, 5]].min() > 1e-3, rel0  # (U, B, b have no source at the zero guess)


def test_scale_factor_is_a_rescaling_of_the_geometric_equations(orc):
    n = 16
    p = synth.zeldovich(n, 5, 1.0, 0.05, True)
    s = orc.deposit(n, p.x, p.u, p.mass)
    a, rho0 = 0.4, p.rho_hat
    geo = orc.initial_fields(n)
    geo["psi"][:] = np.sqrt(a)
    geo["apsi"][:] = np.sqrt(a)
    st, _ = orc.solve_constraints(s, geo, rho0 / a**3, tol=1e-11, max_cycles=80)
    assert st == 0
    s1 = {"s0": s["s0"] / a, "sx": s["sx"] / a**2, "sy": s["sy"] / a**2, "sz": s["sz"] / a**2,
          "sigma": s["sigma"] / a**3}
    one = orc.initial_fields(n)
    st, _ = orc.solve_constraints(s1, one, rho0 / a, tol=1e-12, max_cycles=80)
    assert st == 0
    # the direct solve's unknown psi - 1 is -0.37 here: its FP64 residual floor is higher, so both sides stop at
    # 1e-12 only with the rescaled form; compare at the direct form's own accuracy
    back = {"psi": np.sqrt(a) * one["psi"], "apsi": np.sqrt(a) * one["apsi"]}
    for k in ("Vx", "Vy", "Vz", "U"):
        back[k] = a**2 * one[k]
    for k in ("Bx", "By", "Bz", "b"):
        back[k] = one[k] / a
    for k in orc.FIELDS:
        d = np.sqrt(a) if k in ("psi", "apsi") else 0.0
        err = np.abs(geo[k] - back[k]).max() / np.abs(back[k] - d).max()
        assert err <= 1e-8, (k, err)
