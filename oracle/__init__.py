"""FP64 CPU oracle of the constrained-GR elliptic solve - TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_1905_08890_gb300`` and its binding) never imports it and shares no
code with it.

The arithmetic lives in ``gr_oracle.c`` (plain C, FP64, one loop per
formula).  This module compiles it with gcc and exposes numpy-level wrappers.
Arrays are float64 [n][n][n] C-order, index (i*n + j)*n + k, i the x index,
h = 1/n (box L = 1, G = c = 1).

Equation kinds: POISSON (lap u = f), HELMHOLTZ (lap u - c0 u = f) and PSI
(lap u + 2 pi c0/psi + c1/(8 psi^7) - 2 pi rho psi^5 = f with psi = 1 + u:
the unknown of the psi kind is the deviation psi - 1).

Static nested refinement patches: ``deposit_window``/``deposit_patches``,
``composite_eq`` (one equation) and ``solve_composite`` (the ten) on a chain
of patches given as dicts {"n": cells per side, "origin": [3 parent cells]}.

Field order used throughout: psi, alpha psi, V_x, V_y, V_z, U, B^x, B^y, B^z, b.
Equation (solve) order: V_x, V_y, V_z, U, psi, alpha psi, B^x, B^y, B^z, b
(Sec. 2.4 solution sequence; Sec. 4.3.1 equations MG-linear-1a ... 2).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gr_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "gr_particles.c"), os.path.join(_HERE, "gr_codeunits.c")]
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

POISSON, HELMHOLTZ, PSI = 0, 1, 2
OK, ERR_ARG, ERR_NOMEM, ERR_NOCONV, ERR_NONFINITE = 0, 1, 3, 4, 5

FIELDS = ("psi", "apsi", "Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b")
EQUATIONS = ("Vx", "Vy", "Vz", "U", "psi", "apsi", "Bx", "By", "Bz", "b")
SOURCES = ("s0", "sx", "sy", "sz", "sigma")


def build(force: bool = False) -> str:
    """Compile gr_oracle.c into oracle/_lib/liboracle.so (gcc, OpenMP, no
    fast-math, no FMA contraction so x86 and Arm round alike)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in _SRCS):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            D, I, I64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            P = ctypes.c_void_p
            L.orc_deposit.argtypes = [I, I64, P, P, D, P, P, P, P, P]
            L.orc_mean.argtypes = [I, P]
            L.orc_mean.restype = D
            L.orc_rms.argtypes = [I, P]
            L.orc_rms.restype = D
            L.orc_laplacian.argtypes = [I, P, P]
            L.orc_grad.argtypes = [I, I, P, P]
            L.orc_div3.argtypes = [I, P, P, P, P]
            L.orc_aij.argtypes = [I, P, P, P, P, P]
            L.orc_aa.argtypes = [I, P, P]
            L.orc_lapse_coef.argtypes = [I, P, P, P, P, D, D, P, P]
            L.orc_shift_source.argtypes = [I, P, P, P, P]
            L.orc_residual.argtypes = [I, I, P, P, P, P, D, P]
            L.orc_residual.restype = D
            L.orc_gs_colour.argtypes = [I, I, P, P, P, P, D, I]
            L.orc_restrict.argtypes = [I, P, P]
            L.orc_prolong_add.argtypes = [I, P, P]
            L.orc_vcycle.argtypes = [I, I, P, P, P, P, D, I, I]
            L.orc_vcycle.restype = I
            L.orc_solve_eq.argtypes = [I, I, P, P, P, P, D, D, D, I, I, I, P, P, P]
            L.orc_solve_eq.restype = I
            L.orc_eq_setup.argtypes = [I, I, P, P, D, D, P, P, P, P]
            L.orc_eq_setup.restype = I
            L.orc_solve_constraints.argtypes = [I, P, P, D, D, D, I, I, I, P, P, P, P]
            L.orc_solve_constraints.restype = I
            L.orc_residual_at.argtypes = [I, I, P, P, D, D, I64, P, P, P]
            L.orc_residual_at.restype = None
            L.orc_deposit_window.argtypes = [I, P, I, I64, P, P, D, P, P, P, P, P]
            L.orc_deposit_window.restype = None
            L.orc_composite_eq.argtypes = [I, I, I, P, P, D, P, P, P, P, P, P, P, P, P, D, I, I, I, P, P, P]
            L.orc_composite_eq.restype = I
            L.orc_solve_composite.argtypes = [I, I, P, P, P, P, P, P, D, D, D, I, I, I, P, P, P]
            L.orc_solve_composite.restype = I
            L.orc_patch_ghosted.argtypes = [I, P, I, I, P, P, P]
            L.orc_patch_ghosted.restype = None
            L.orc_patch_residual_at.argtypes = [I, I, D, P, P, D, D, D, I64, P, P, P]
            L.orc_patch_residual_at.restype = None
            L.orc_patch_eq_setup.argtypes = [I, I, D, P, P, D, D, D, P, P, P, P]
            L.orc_patch_eq_setup.restype = I
            L.orc_particle_fields.argtypes = [I, P, P, P, P, P, P, P]
            L.orc_particle_fields.restype = None
            L.orc_particle_update.argtypes = [I, I64, P, P, P, D, I, I, I]
            L.orc_particle_update.restype = None
            L.orc_deposit_metric.argtypes = [I, I64, P, P, D, P, P, P, P, P, P]
            L.orc_deposit_metric.restype = None
            L.orc_solve_code_units.argtypes = [I, D, D, D, P, P, D, I, P, P, P, P]
            L.orc_solve_code_units.restype = I
            L.orc_code_units_residual.argtypes = [I, D, D, D, P, P, P]
            L.orc_code_units_residual.restype = I
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _grid(n):
    return np.zeros((n, n, n), dtype=np.float64)


# ---------------------------------------------------------------- deposit
def deposit(n: int, x: np.ndarray, u: np.ndarray, mass: float) -> dict:
    """CIC sources s0, s_x, s_y, s_z, sigma (Sec. 4.1.2); x, u are (3, np)."""
    x = _f64(x)
    u = _f64(u)
    npart = x.shape[1] if x.ndim == 2 else 0
    out = {k: _grid(n) for k in SOURCES}
    lib().orc_deposit(n, npart, _p(x), _p(u), mass, *[_p(out[k]) for k in SOURCES])
    return out


def deposit_metric(n: int, x: np.ndarray, u: np.ndarray, mass: float, psi=None) -> dict:
    """CIC sources with the Lorentz factor at the conformal factor psi (n^3,
    interpolated to each particle; None: psi = 1) (Sec. 4.5)."""
    x = _f64(x)
    u = _f64(u)
    npart = x.shape[1] if x.ndim == 2 else 0
    out = {k: _grid(n) for k in SOURCES}
    ps = None if psi is None else _f64(psi)
    lib().orc_deposit_metric(n, npart, _p(x), _p(u), mass, _p(ps), *[_p(out[k]) for k in SOURCES])
    return out


# ---------------------------------------------------------------- particles
PARTICLE_FIELDS = ("alpha", "psi", "beta_x", "beta_y", "beta_z", "dalpha_x", "dalpha_y", "dalpha_z", "dpsi_x",
                   "dpsi_y", "dpsi_z") + tuple(f"dbeta{j}_{i}" for j in "xyz" for i in "xyz")


def particle_fields(fld: dict) -> np.ndarray:
    """The 20 grid quantities of the particle update (Sec. 4.4): alpha, psi,
    beta^j and their central differences, as a (20, n, n, n) array in the
    order PARTICLE_FIELDS (dbeta{j}_{i} = D_i beta^j)."""
    n = fld["psi"].shape[0]
    out = np.zeros((20, n, n, n))
    a = [_f64(fld[k]) for k in ("psi", "apsi", "Bx", "By", "Bz", "b")]
    lib().orc_particle_fields(n, *[_p(v) for v in a], _p(out))
    return out


def particle_update(fld: dict, x: np.ndarray, u: np.ndarray, dt: float, sync=True, open_=True, drift=True,
                    fields=None):
    """Kick(s) and drift of the particles (x, u: (3, np), updated in place)
    in the solved fields (Sec. 4.4, App. A)."""
    n = fld["psi"].shape[0]
    assert x.dtype == np.float64 and x.flags.c_contiguous and u.dtype == np.float64 and u.flags.c_contiguous
    g = particle_fields(fld) if fields is None else fields
    npart = x.shape[1]
    lib().orc_particle_update(n, npart, _p(x), _p(u), _p(g), dt, int(sync), int(open_), int(drift))


# ---------------------------------------------------------------- code units (Sec. 4.1)
def solve_code_units(src_code: dict, fld_code: dict, a: float, Omega_m: float, H0: float, tol=1e-10,
                     max_cycles=50):
    """The ten-equation solve in code units at scale factor a: code-unit
    sources (s0, sx, sy, sz, sigma keys: st0, st_i, the trace) and fields
    (psi key: Psi, apsi key: Phi, the others the code-unit potentials; guesses
    in, solutions out, in place).  Returns (status, report)."""
    n = src_code["s0"].shape[0]
    srcs = [_f64(src_code[k]) for k in SOURCES]
    for k in FIELDS:
        assert fld_code[k].dtype == np.float64 and fld_code[k].flags.c_contiguous
    sp = (ctypes.c_void_p * 5)(*[v.ctypes.data for v in srcs])
    fp = (ctypes.c_void_p * 10)(*[fld_code[k].ctypes.data for k in FIELDS])
    cyc = (ctypes.c_int * 10)()
    r0 = (ctypes.c_double * 10)()
    r = (ctypes.c_double * 10)()
    sts = (ctypes.c_int * 10)()
    st = lib().orc_solve_code_units(n, a, Omega_m, H0, sp, fp, tol, max_cycles, cyc, r0, r, sts)
    return st, {"cycles": list(cyc), "res0": list(r0), "res": list(r), "status": list(sts)}


def code_units_residual(src_code: dict, fld_code: dict, a: float, Omega_m: float, H0: float):
    """Relative residuals of the paper's printed code-unit equations (solve
    order: V_x, V_y, V_z, U, Psi, Phi, B^x, B^y, B^z, b)."""
    n = src_code["s0"].shape[0]
    srcs = [_f64(src_code[k]) for k in SOURCES]
    flds = [_f64(fld_code[k]) for k in FIELDS]
    sp = (ctypes.c_void_p * 5)(*[v.ctypes.data for v in srcs])
    fp = (ctypes.c_void_p * 10)(*[v.ctypes.data for v in flds])
    rel = np.zeros(10)
    if lib().orc_code_units_residual(n, a, Omega_m, H0, sp, fp, _p(rel)) != 0:
        raise MemoryError("orc_code_units_residual")
    return rel


def code_initial_fields(n: int) -> dict:
    """The plain guess in code units: every potential 0 (psi = a^(1/2), alpha = 1)."""
    return {k: _grid(n) for k in FIELDS}


# ---------------------------------------------------------------- operators
def laplacian(f):
    f = _f64(f)
    out = np.empty_like(f)
    lib().orc_laplacian(f.shape[0], _p(f), _p(out))
    return out


def grad(f, axis: int):
    f = _f64(f)
    out = np.empty_like(f)
    lib().orc_grad(f.shape[0], axis, _p(f), _p(out))
    return out


def div3(Fx, Fy, Fz):
    Fx, Fy, Fz = _f64(Fx), _f64(Fy), _f64(Fz)
    out = np.empty_like(Fx)
    lib().orc_div3(Fx.shape[0], _p(Fx), _p(Fy), _p(Fz), _p(out))
    return out


def aij(Vx, Vy, Vz, U):
    """Six components xx, yy, zz, xy, xz, yz of A_ij (Eq. Aij-discrete-2)."""
    Vx, Vy, Vz, U = map(_f64, (Vx, Vy, Vz, U))
    n = U.shape[0]
    A = np.empty((6, n, n, n))
    lib().orc_aij(n, _p(Vx), _p(Vy), _p(Vz), _p(U), _p(A))
    return A


def aa(A):
    A = _f64(A)
    out = np.empty(A.shape[1:])
    lib().orc_aa(A.shape[1], _p(A), _p(out))
    return out


def lapse_coef(psi, s0, sigma, AA, rho_hat, S_hat=0.0):
    """m and f of  lap(alpha psi) - m alpha psi = f  (Eq. sol-scheme-CMC)."""
    psi, s0, sigma, AA = map(_f64, (psi, s0, sigma, AA))
    K2, Kdot = background(rho_hat, S_hat)
    m = np.empty_like(psi)
    f = np.empty_like(psi)
    lib().orc_lapse_coef(psi.shape[0], _p(psi), _p(s0), _p(sigma), _p(AA), K2, Kdot, _p(m), _p(f))
    return m, f


def shift_source(A, psi, apsi):
    A, psi, apsi = map(_f64, (A, psi, apsi))
    n = psi.shape[0]
    SB = np.empty((3, n, n, n))
    lib().orc_shift_source(n, _p(A), _p(psi), _p(apsi), _p(SB))
    return SB


def background(rho_hat: float, S_hat: float = 0.0):
    """K^2 = 24 pi rho_hat and Kdot = 12 pi rho_hat + 4 pi S_hat (Sec. 2.3)."""
    return 24.0 * math.pi * rho_hat, 12.0 * math.pi * rho_hat + 4.0 * math.pi * S_hat


# ---------------------------------------------------------------- multigrid
def residual(kind, u, f, c0=None, c1=None, rho=0.0):
    """(eps, RMS(eps)) with eps = L(u) - f."""
    u, f = _f64(u), _f64(f)
    c0 = None if c0 is None else _f64(c0)
    c1 = None if c1 is None else _f64(c1)
    eps = np.empty_like(u)
    r = lib().orc_residual(kind, u.shape[0], _p(u), _p(f), _p(c0), _p(c1), rho, _p(eps))
    return eps, r


def gs_colour(kind, u, f, c0=None, c1=None, rho=0.0, color=0):
    """One Gauss-Seidel (Newton for the psi kind) pass over the cells with
    (i + j + k) % 2 == color, in place on u."""
    f = _f64(f)
    c0 = None if c0 is None else _f64(c0)
    c1 = None if c1 is None else _f64(c1)
    lib().orc_gs_colour(kind, u.shape[0], _p(u), _p(f), _p(c0), _p(c1), rho, color)


def restrict(fine):
    fine = _f64(fine)
    n = fine.shape[0] // 2
    out = np.empty((n, n, n))
    lib().orc_restrict(fine.shape[0], _p(fine), _p(out))
    return out


def prolong_add(coarse, fine):
    """fine += P(coarse), in place."""
    coarse = _f64(coarse)
    lib().orc_prolong_add(fine.shape[0], _p(coarse), _p(fine))


def vcycle(kind, u, f, c0=None, c1=None, rho=0.0, nu1=2, nu2=2):
    """One V(nu1, nu2) cycle, in place on u (float64 C-contiguous)."""
    f = _f64(f)
    c0 = None if c0 is None else _f64(c0)
    c1 = None if c1 is None else _f64(c1)
    st = lib().orc_vcycle(kind, u.shape[0], _p(u), _p(f), _p(c0), _p(c1), rho, nu1, nu2)
    if st != OK:
        raise RuntimeError(f"orc_vcycle status {st}")


def solve_eq(kind, u, f, c0=None, c1=None, rho=0.0, ref=0.0, tol=1e-10, max_cycles=50, nu1=2, nu2=2):
    """Solve one equation in place on u; returns (status, cycles, res0, res)."""
    f = _f64(f)
    c0 = None if c0 is None else _f64(c0)
    c1 = None if c1 is None else _f64(c1)
    cyc = ctypes.c_int(0)
    r0 = ctypes.c_double(0)
    r = ctypes.c_double(0)
    st = lib().orc_solve_eq(kind, u.shape[0], _p(u), _p(f), _p(c0), _p(c1), rho, ref, tol, max_cycles, nu1, nu2,
                            ctypes.byref(cyc), ctypes.byref(r0), ctypes.byref(r))
    return st, cyc.value, r0.value, r.value


def eq_setup(eq: int, src: dict, fld: dict, rho_hat: float, S_hat: float = 0.0):
    """(kind, f, c0, c1, ref) of equation eq (solve order) from sources and fields."""
    n = src["s0"].shape[0]
    srcs = [_f64(src[k]) for k in SOURCES]
    order = ("Vx", "Vy", "Vz", "U", "psi", "apsi", "Bx", "By", "Bz", "b")
    flds = [_f64(fld[k]) for k in order]
    sp = (ctypes.c_void_p * 5)(*[a.ctypes.data for a in srcs])
    fp = (ctypes.c_void_p * 10)(*[a.ctypes.data for a in flds])
    f, c0, c1 = _grid(n), _grid(n), _grid(n)
    ref = ctypes.c_double(0)
    kind = lib().orc_eq_setup(eq, n, sp, fp, rho_hat, S_hat, _p(f), _p(c0), _p(c1), ctypes.byref(ref))
    if kind < 0:
        raise MemoryError("orc_eq_setup")
    return kind, f, (c0 if kind != POISSON else None), (c1 if kind == PSI else None), ref.value


def initial_fields(n: int) -> dict:
    """The plain guess: psi = alpha psi = 1, vectors and scalars 0."""
    fld = {k: _grid(n) for k in FIELDS}
    fld["psi"][:] = 1.0
    fld["apsi"][:] = 1.0
    return fld


def solve_constraints(src: dict, fld: dict, rho_hat: float, S_hat: float = 0.0, tol=1e-10, max_cycles=50, nu1=2,
                      nu2=2):
    """Ten-equation solve, in place on the float64 arrays of fld.  Returns
    (status, report) with per-equation cycles, res0, res, status in solve order."""
    n = src["s0"].shape[0]
    srcs = [_f64(src[k]) for k in SOURCES]
    for k in FIELDS:
        a = fld[k]
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == (n, n, n)
    sp = (ctypes.c_void_p * 5)(*[a.ctypes.data for a in srcs])
    fp = (ctypes.c_void_p * 10)(*[fld[k].ctypes.data for k in FIELDS])
    cyc = (ctypes.c_int * 10)()
    r0 = (ctypes.c_double * 10)()
    r = (ctypes.c_double * 10)()
    sts = (ctypes.c_int * 10)()
    st = lib().orc_solve_constraints(n, sp, fp, rho_hat, S_hat, tol, max_cycles, nu1, nu2, cyc, r0, r, sts)
    rep = {"cycles": list(cyc), "res0": list(r0), "res": list(r), "status": list(sts)}
    return st, rep


def residual_at(eq: int, src: dict, fld: dict, rho_hat: float, cells, S_hat: float = 0.0):
    """(eps, f) of equation eq at the natural indices `cells`, from the given
    sources and fields (for sampled checks of grids too large to solve here);
    f is the local value of the quantity whose RMS is the equation's reference.
    Poisson-type right-hand sides here carry only the source mean of V_i (the
    divergence sources are mean-free up to rounding)."""
    order = ("Vx", "Vy", "Vz", "U", "psi", "apsi", "Bx", "By", "Bz", "b")
    srcs = [_f64(src[k]) for k in SOURCES]
    flds = [_f64(fld[k]) for k in order]
    n = srcs[0].shape[0]
    sp = (ctypes.c_void_p * 5)(*[a.ctypes.data for a in srcs])
    fp = (ctypes.c_void_p * 10)(*[a.ctypes.data for a in flds])
    idx = np.ascontiguousarray(cells, dtype=np.int64)
    eps = np.empty(idx.size)
    f = np.empty(idx.size)
    lib().orc_residual_at(eq, n, sp, fp, rho_hat, S_hat, idx.size, idx.ctypes.data, eps.ctypes.data, f.ctypes.data)
    return eps, f


# ---------------------------------------------------------------- patches
# A chain of static patches: patch p (1-based) has n_p cells per side at
# spacing h0 / 2^p and refines the parent block origin_p .. origin_p + n_p/2 - 1
# (parent cells per axis; patch 1's block may wrap on the periodic base).
def patch_window(n0: int, patches, p: int):
    """(N, O): the resolution N = n0 2^p and the origin O (cells of that
    resolution, per axis) of patch p (1-based) of the chain."""
    O = [0, 0, 0]
    for q in range(1, p + 1):
        O = [2 * (O[d] + patches[q - 1]["origin"][d]) for d in range(3)]
    N = n0 << p
    return N, [o % N for o in O]


def deposit_window(N: int, O, nw: int, x: np.ndarray, u: np.ndarray, mass: float) -> dict:
    """CIC sources at resolution N on the nw^3 window of cells O + a (mod N)."""
    x = _f64(x)
    u = _f64(u)
    npart = x.shape[1] if x.ndim == 2 else 0
    out = {k: np.zeros((nw, nw, nw)) for k in SOURCES}
    Oa = (ctypes.c_int * 3)(*[int(o) for o in O])
    lib().orc_deposit_window(N, Oa, nw, npart, _p(x), _p(u), mass, *[_p(out[k]) for k in SOURCES])
    return out


def deposit_patches(n0: int, patches, x, u, mass: float):
    """Sources of every patch of the chain (list of dicts)."""
    out = []
    for p in range(1, len(patches) + 1):
        N, O = patch_window(n0, patches, p)
        out.append(deposit_window(N, O, patches[p - 1]["n"], x, u, mass))
    return out


def _chain(patches):
    pn = (ctypes.c_int * max(1, len(patches)))(*[int(q["n"]) for q in patches])
    po = (ctypes.c_int * max(3, 3 * len(patches)))(*[int(o) for q in patches for o in q["origin"]])
    return pn, po


def composite_eq(kind, u0, f0, patches, up, fp, c00=None, c10=None, c0p=None, c1p=None, rho=0.0, refs=None,
                 tol=1e-10, max_cycles=50, nu1=2, nu2=2):
    """Composite solve of one equation, in place on u0 (base, n0^3) and the
    patch interiors up[p] (n_p^3); fp, c0p, c1p: per-patch arrays (or None).
    Returns (status, cycles, res0, res) with per-level residual lists."""
    n0 = u0.shape[0]
    np_ = len(patches)
    f0 = _f64(f0)
    c00 = None if c00 is None else _f64(c00)
    c10 = None if c10 is None else _f64(c10)
    for a in up:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    fp = [_f64(a) for a in fp]
    c0p = [None if a is None else _f64(a) for a in (c0p or [None] * np_)]
    c1p = [None if a is None else _f64(a) for a in (c1p or [None] * np_)]
    arr = lambda lst: (ctypes.c_void_p * max(1, np_))(*[None if a is None else a.ctypes.data for a in lst])
    pn, po = _chain(patches)
    rf = (ctypes.c_double * (np_ + 1))(*([0.0] * (np_ + 1) if refs is None else refs))
    cyc = ctypes.c_int(0)
    r0 = (ctypes.c_double * (np_ + 1))()
    r = (ctypes.c_double * (np_ + 1))()
    st = lib().orc_composite_eq(kind, n0, np_, pn, po, rho, _p(u0), _p(f0), _p(c00), _p(c10), arr(up), arr(fp),
                                arr(c0p), arr(c1p), rf, tol, max_cycles, nu1, nu2, ctypes.byref(cyc), r0, r)
    return st, cyc.value, list(r0), list(r)


def initial_patch_fields(patches):
    return [initial_fields(q["n"]) for q in patches]


def solve_composite(src0: dict, srcp, fld0: dict, fldp, patches, rho_hat: float, S_hat: float = 0.0, tol=1e-10,
                    max_cycles=50, nu1=2, nu2=2):
    """Ten-equation composite solve, in place on fld0 (base) and fldp (one
    field dict per patch).  Returns (status, report): per-equation cycles and
    status in solve order, res[e][l] the final residual of level l."""
    n0 = src0["s0"].shape[0]
    np_ = len(patches)
    s0 = [_f64(src0[k]) for k in SOURCES]
    sp = [_f64(d[k]) for d in srcp for k in SOURCES]
    for d in [fld0] + list(fldp):
        for k in FIELDS:
            assert d[k].dtype == np.float64 and d[k].flags.c_contiguous
    f0 = [fld0[k] for k in FIELDS]
    fpl = [d[k] for d in fldp for k in FIELDS]
    vp = lambda lst: (ctypes.c_void_p * max(1, len(lst)))(*[a.ctypes.data for a in lst])
    pn, po = _chain(patches)
    cyc = (ctypes.c_int * 10)()
    r = (ctypes.c_double * (10 * (np_ + 1)))()
    sts = (ctypes.c_int * 10)()
    st = lib().orc_solve_composite(n0, np_, pn, po, vp(s0), vp(sp), vp(f0), vp(fpl), rho_hat, S_hat, tol,
                                   max_cycles, nu1, nu2, cyc, r, sts)
    res = [list(r[e * (np_ + 1):(e + 1) * (np_ + 1)]) for e in range(10)]
    return st, {"cycles": list(cyc), "res": res, "status": list(sts)}


def patch_ghosted(interior, origin, parent, parent_periodic: bool):
    """(n + 4)^3 array: the patch interior with two ghost layers interpolated
    (trilinear) from the parent (natural array; periodic for the base)."""
    interior = _f64(interior)
    parent = _f64(parent)
    n = interior.shape[0]
    out = np.zeros((n + 4,) * 3)
    o = (ctypes.c_int * 3)(*[int(v) for v in origin])
    lib().orc_patch_ghosted(n, o, parent.shape[0], int(parent_periodic), _p(parent), _p(interior), _p(out))
    return out


def patch_residual_at(eq: int, n: int, nh: float, src: dict, G: dict, smean: float, rho_hat: float, cells,
                      S_hat: float = 0.0):
    """(eps, fscale) of equation eq (solve order) at the natural interior
    indices `cells` of a patch without a child; G: ghosted fields by name."""
    order = ("Vx", "Vy", "Vz", "U", "psi", "apsi", "Bx", "By", "Bz", "b")
    srcs = [_f64(src[k]) for k in SOURCES]
    gs = [_f64(G[k]) for k in order]
    sp = (ctypes.c_void_p * 5)(*[a.ctypes.data for a in srcs])
    gp = (ctypes.c_void_p * 10)(*[a.ctypes.data for a in gs])
    idx = np.ascontiguousarray(cells, dtype=np.int64)
    eps = np.empty(idx.size)
    f = np.empty(idx.size)
    lib().orc_patch_residual_at(eq, n, nh, sp, gp, smean, rho_hat, S_hat, idx.size, idx.ctypes.data,
                                eps.ctypes.data, f.ctypes.data)
    return eps, f


def patch_eq_setup(eq: int, n: int, nh: float, src: dict, G: dict, smean: float, rho_hat: float, S_hat: float = 0.0):
    """(kind, f, c0, c1, ref) of equation eq on a patch of n cells at 1/h = nh
    from its interior sources and ghosted fields G (by name); f, c0, c1 are
    ghosted (n + 4)^3 arrays with the interior written."""
    order = ("Vx", "Vy", "Vz", "U", "psi", "apsi", "Bx", "By", "Bz", "b")
    srcs = [_f64(src[k]) for k in SOURCES]
    gs = [_f64(G[k]) for k in order]
    sp = (ctypes.c_void_p * 5)(*[a.ctypes.data for a in srcs])
    gp = (ctypes.c_void_p * 10)(*[a.ctypes.data for a in gs])
    m = n + 4
    f, c0, c1 = np.zeros((m, m, m)), np.zeros((m, m, m)), np.zeros((m, m, m))
    ref = ctypes.c_double(0)
    kind = lib().orc_patch_eq_setup(eq, n, nh, sp, gp, smean, rho_hat, S_hat, _p(f), _p(c0), _p(c1),
                                    ctypes.byref(ref))
    return kind, f, c0, c1, ref.value
