"""Thin ctypes binding of the C ABI in include/gr.h.

Argument marshalling only: every step of the deposit and the solve runs in
the CUDA kernels of libgr.so.  Arrays are torch CUDA tensors (float64,
contiguous); torch provides device memory and streams.  There is no CPU
fallback: if libgr.so cannot be built or loaded, every call raises.

The functions keep the C names (gr_create, gr_deposit, gr_solve_constraints,
gr_vcycle, gr_residual, ...).  ``Context`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

GR_OK, GR_ERR_ARG, GR_ERR_CUDA, GR_ERR_NOMEM, GR_ERR_NOCONV, GR_ERR_NONFINITE, GR_ERR_STATE = range(7)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_NOMEM", "ERR_NOCONV", "ERR_NONFINITE", "ERR_STATE"]
EQUATIONS = ("Vx", "Vy", "Vz", "U", "psi", "apsi", "Bx", "By", "Bz", "b")
GR_VX, GR_VY, GR_VZ, GR_U, GR_PSI, GR_APSI, GR_BX, GR_BY, GR_BZ, GR_B_SCALAR = range(10)
GR_NEQ = 10
GR_PREC_FP64, GR_PREC_MIXED, GR_PREC_MIXED_DF = 0, 1, 2
FIELDS = ("psi", "apsi", "Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b")
SOURCES = ("s0", "sx", "sy", "sz", "sigma")

_P = ctypes.c_void_p


class gr_sources(ctypes.Structure):
    _fields_ = [("s0", _P), ("s", _P * 3), ("sigma", _P)]


class gr_fields(ctypes.Structure):
    _fields_ = [("psi", _P), ("apsi", _P), ("V", _P * 3), ("U", _P), ("B", _P * 3), ("b", _P)]


MAX_PATCHES = 4


class gr_patch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("origin", ctypes.c_int * 3), ("src", gr_sources), ("fld", gr_fields)]


class gr_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("prec", ctypes.c_int), ("rho_hat", ctypes.c_double), ("S_hat", ctypes.c_double),
                ("verbose", ctypes.c_int), ("profile", ctypes.c_int), ("check_guess", ctypes.c_int),
                ("fmg", ctypes.c_int), ("host_out", ctypes.POINTER(gr_fields)), ("npatch", ctypes.c_int),
                ("patch", ctypes.POINTER(gr_patch))]


class gr_report(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int * 10), ("res0", ctypes.c_double * 10), ("res", ctypes.c_double * 10),
                ("eq_status", ctypes.c_int * 10), ("seconds", ctypes.c_double), ("eq_seconds", ctypes.c_double * 10),
                ("cell_updates", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("prof_launches", ctypes.c_int * 11), ("prof_ms", ctypes.c_double * 11),
                ("guess_rejected", ctypes.c_int * 10), ("res_level", (ctypes.c_double * (MAX_PATCHES + 1)) * 10)]


PROF_CLASSES = ("sweep64", "sweep32", "resid_restrict", "prolong", "mixed_resid", "mixed_update", "norm64", "setup",
                "coarse", "patch", "smooth3")


_lib = None
_lock = threading.Lock()
EXPORTED = ("gr_default_opts", "gr_create", "gr_destroy", "gr_deposit", "gr_deposit_patches", "gr_solve_constraints",
            "gr_vcycle", "gr_residual", "gr_last_error", "gr_kernel_launches", "gr_momentum_residual_noalloc",
            "gr_particle_update", "gr_kick", "gr_drift", "gr_deposit_metric", "gr_solve_code_units", "gr_fma_rate")
GR_KICK_SYNC, GR_KICK_OPEN, GR_DRIFT = 1, 2, 4


def lib():
    """Build (if stale) and load libgr.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("GR_LIBRARY") or _build.build()
            L = ctypes.CDLL(path)
            L.gr_default_opts.argtypes = [ctypes.POINTER(gr_opts)]
            L.gr_default_opts.restype = None
            L.gr_create.argtypes = [ctypes.c_int, ctypes.c_double, _P, ctypes.POINTER(_P)]
            L.gr_create.restype = ctypes.c_int
            L.gr_destroy.argtypes = [_P]
            L.gr_destroy.restype = None
            L.gr_deposit.argtypes = [_P, ctypes.c_int64, _P, _P, ctypes.c_double, ctypes.POINTER(gr_sources)]
            L.gr_deposit.restype = ctypes.c_int
            L.gr_deposit_patches.argtypes = [_P, ctypes.c_int, ctypes.POINTER(gr_patch), ctypes.c_int64, _P, _P,
                                             ctypes.c_double]
            L.gr_deposit_patches.restype = ctypes.c_int
            L.gr_solve_constraints.argtypes = [_P, ctypes.POINTER(gr_sources), ctypes.POINTER(gr_fields),
                                               ctypes.POINTER(gr_opts), ctypes.POINTER(gr_report)]
            L.gr_solve_constraints.restype = ctypes.c_int
            L.gr_vcycle.argtypes = [_P, ctypes.c_int, ctypes.POINTER(gr_sources), ctypes.POINTER(gr_fields),
                                    ctypes.POINTER(gr_opts), ctypes.POINTER(ctypes.c_double)]
            L.gr_vcycle.restype = ctypes.c_int
            L.gr_residual.argtypes = [_P, ctypes.c_int, ctypes.POINTER(gr_sources), ctypes.POINTER(gr_fields),
                                      ctypes.POINTER(gr_opts), _P, ctypes.POINTER(ctypes.c_double)]
            L.gr_residual.restype = ctypes.c_int
            L.gr_last_error.argtypes = []
            L.gr_last_error.restype = ctypes.c_char_p
            L.gr_kernel_launches.argtypes = []
            L.gr_kernel_launches.restype = ctypes.c_longlong
            L.gr_fma_rate.argtypes = [ctypes.c_int, ctypes.c_longlong, _P, ctypes.POINTER(ctypes.c_double)]
            L.gr_fma_rate.restype = ctypes.c_int
            L.gr_momentum_residual_noalloc.argtypes = [ctypes.c_int, ctypes.c_double, _P, _P, _P,
                                                       ctypes.POINTER(ctypes.c_double), _P]
            L.gr_momentum_residual_noalloc.restype = ctypes.c_int
            L.gr_particle_update.argtypes = [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(gr_fields), ctypes.c_double,
                                             ctypes.c_int]
            L.gr_particle_update.restype = ctypes.c_int
            L.gr_kick.argtypes = [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(gr_fields), ctypes.c_double, ctypes.c_int]
            L.gr_kick.restype = ctypes.c_int
            L.gr_drift.argtypes = [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(gr_fields), ctypes.c_double]
            L.gr_drift.restype = ctypes.c_int
            L.gr_deposit_metric.argtypes = [_P, ctypes.c_int64, _P, _P, ctypes.c_double, _P,
                                            ctypes.POINTER(gr_sources)]
            L.gr_deposit_metric.restype = ctypes.c_int
            L.gr_solve_code_units.argtypes = [_P, ctypes.POINTER(gr_cosmology), ctypes.POINTER(gr_sources),
                                              ctypes.POINTER(gr_fields), ctypes.POINTER(gr_opts),
                                              ctypes.POINTER(gr_report)]
            L.gr_solve_code_units.restype = ctypes.c_int
            FP = ctypes.POINTER(ctypes.c_float)
            L.gr_net_create.argtypes = [ctypes.c_int, _P, ctypes.c_uint64, ctypes.POINTER(_P)]
            L.gr_net_create.restype = ctypes.c_int
            L.gr_net_destroy.argtypes = [_P]
            L.gr_net_destroy.restype = None
            L.gr_net_num_params.argtypes = [_P]
            L.gr_net_num_params.restype = ctypes.c_size_t
            L.gr_net_get_params.argtypes = [_P, _P]
            L.gr_net_get_params.restype = ctypes.c_int
            L.gr_net_set_params.argtypes = [_P, _P]
            L.gr_net_set_params.restype = ctypes.c_int
            L.gr_net_set_norm.argtypes = [_P, _P, _P, _P, _P]
            L.gr_net_set_norm.restype = ctypes.c_int
            L.gr_net_infer.argtypes = [_P, ctypes.POINTER(gr_sources), ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(gr_fields)]
            L.gr_net_infer.restype = ctypes.c_int
            L.gr_net_loss_grad.argtypes = [_P, ctypes.POINTER(gr_sources), ctypes.POINTER(gr_fields), ctypes.c_double,
                                           ctypes.c_double, FP, _P]
            L.gr_net_loss_grad.restype = ctypes.c_int
            L.gr_net_train_step.argtypes = [_P, ctypes.POINTER(gr_sources), ctypes.POINTER(gr_fields),
                                            ctypes.c_double, ctypes.c_double, ctypes.c_float, FP]
            L.gr_net_train_step.restype = ctypes.c_int
            L.gr_net_guess.argtypes = [_P, ctypes.c_int, ctypes.POINTER(gr_sources), ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(gr_fields)]
            L.gr_net_guess.restype = ctypes.c_int
            L.gr_net_activation.argtypes = [_P, ctypes.c_int, _P, ctypes.c_size_t]
            L.gr_net_activation.restype = ctypes.c_int
            _lib = L
    return _lib


class GRError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


def _check(st: int, where: str, allow=()):
    if st != GR_OK and st not in allow:
        raise GRError(st, where, lib().gr_last_error().decode())
    return st


def _ptr(t, host_ok=False):
    """Address of a contiguous float64 tensor: CUDA, or also CPU (host
    memory, preferably pinned) where the C call accepts host arrays."""
    if t is None:
        return None
    import torch

    if not (t.dtype == torch.float64 and t.is_contiguous() and (t.is_cuda or (host_ok and t.device.type == "cpu"))):
        raise ValueError("expected a contiguous float64 CUDA tensor" + (" or CPU tensor" if host_ok else ""))
    return t.data_ptr()


def make_sources(src: dict) -> gr_sources:
    s = gr_sources()
    s.s0 = _ptr(src["s0"])
    for d, k in enumerate(("sx", "sy", "sz")):
        s.s[d] = _ptr(src[k])
    s.sigma = _ptr(src["sigma"])
    return s


def make_fields(fld: dict, host_ok=False) -> gr_fields:
    f = gr_fields()
    f.psi = _ptr(fld["psi"], host_ok)
    f.apsi = _ptr(fld["apsi"], host_ok)
    for d, k in enumerate(("Vx", "Vy", "Vz")):
        f.V[d] = _ptr(fld[k], host_ok)
    f.U = _ptr(fld["U"], host_ok)
    for d, k in enumerate(("Bx", "By", "Bz")):
        f.B[d] = _ptr(fld[k], host_ok)
    f.b = _ptr(fld["b"], host_ok)
    return f


def make_patches(patches) -> ctypes.Array:
    """A gr_patch array from dicts {"n", "origin", "src" (sources dict),
    "fld" (fields dict)}; "src"/"fld" may be missing where the call does not
    read them (they are then NULL)."""
    arr = (gr_patch * max(1, len(patches)))()
    for p, q in enumerate(patches):
        arr[p].n = int(q["n"])
        for d in range(3):
            arr[p].origin[d] = int(q["origin"][d])
        if q.get("src") is not None:
            arr[p].src = make_sources(q["src"])
        if q.get("fld") is not None:
            arr[p].fld = make_fields(q["fld"])
    return arr


def centred_chain(n0: int, centre, sizes) -> list:
    """A chain of patches (dicts with "n" and "origin") centred on base cell
    `centre` (i, j, k): patch 1 of sizes[0] cells covers the sizes[0]/2 base
    cells around it (its block may wrap around the periodic base), each
    further patch sits in the middle of its parent.  Host-side arithmetic
    only; gr_solve_constraints checks the chain."""
    out, npar = [], n0
    for p, n in enumerate(sizes):
        if p == 0:
            origin = [(int(c) - n // 4) % n0 for c in centre]
        else:
            o = (npar - n // 2) // 2
            origin = [o, o, o]
        out.append({"n": int(n), "origin": origin})
        npar = n
    return out


def make_opts(tol=1e-10, max_cycles=50, nu1=2, nu2=2, prec="fp64", rho_hat=0.0, S_hat=0.0, verbose=0,
              profile=0, check_guess=0, fmg=0, host_out=None, patches=None) -> gr_opts:
    """host_out: optional dict of ten CPU (pinned) float64 tensors that each
    solved field is copied into while the later equations solve.  patches:
    optional list of patch dicts (see make_patches) with "src" and "fld"."""
    o = gr_opts()
    lib().gr_default_opts(ctypes.byref(o))
    o.tol, o.max_cycles, o.nu1, o.nu2 = tol, max_cycles, nu1, nu2
    o.prec = ({"fp64": GR_PREC_FP64, "mixed": GR_PREC_MIXED, "mixed_df": GR_PREC_MIXED_DF}[prec]
              if isinstance(prec, str) else int(prec))
    o.rho_hat, o.S_hat, o.verbose, o.profile = rho_hat, S_hat, verbose, int(profile)
    o.check_guess = int(check_guess)
    o.fmg = int(fmg)
    if host_out is not None:
        o._host_out = make_fields(host_out, host_ok=True)  # kept alive with the options
        o.host_out = ctypes.pointer(o._host_out)
    if patches:
        o._patches = make_patches(patches)
        o.npatch = len(patches)
        o.patch = ctypes.cast(o._patches, ctypes.POINTER(gr_patch))
    return o


def report_dict(r: gr_report) -> dict:
    return {"cycles": list(r.cycles), "res0": list(r.res0), "res": list(r.res), "status": list(r.eq_status),
            "seconds": r.seconds, "eq_seconds": list(r.eq_seconds), "cell_updates": int(r.cell_updates),
            "kernel_launches": int(r.kernel_launches), "guess_rejected": list(r.guess_rejected),
            "res_level": [list(r.res_level[e]) for e in range(10)],
            "prof": {k: {"launches": int(r.prof_launches[i]), "ms": float(r.prof_ms[i])}
                     for i, k in enumerate(PROF_CLASSES)}}


# ------------------------------------------------------------------ C names
def gr_create(n: int, L: float = 1.0, stream=None):
    h = _P()
    st = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    _check(lib().gr_create(n, L, st, ctypes.byref(h)), "gr_create")
    return h


def gr_destroy(ctx):
    lib().gr_destroy(ctx)


def gr_deposit(ctx, x, u, mass: float, src: dict):
    npart = x.shape[1] if x.numel() else 0
    s = make_sources(src)
    _check(lib().gr_deposit(ctx, npart, _ptr(x, True) if npart else None, _ptr(u, True) if npart else None, mass,
                            ctypes.byref(s)), "gr_deposit")


def gr_deposit_patches(ctx, patches, x, u, mass: float):
    """Sources of every patch (dicts with "n", "origin", "src"); x, u CUDA tensors."""
    npart = x.shape[1] if x.numel() else 0
    arr = make_patches([{"n": q["n"], "origin": q["origin"], "src": q["src"]} for q in patches])
    _check(lib().gr_deposit_patches(ctx, len(patches), arr, npart, _ptr(x) if npart else None,
                                    _ptr(u) if npart else None, mass), "gr_deposit_patches")


def gr_solve_constraints(ctx, src: dict, fld: dict, opts: gr_opts, allow_noconv=False) -> dict:
    s, f, r = make_sources(src), make_fields(fld), gr_report()
    st = lib().gr_solve_constraints(ctx, ctypes.byref(s), ctypes.byref(f), ctypes.byref(opts), ctypes.byref(r))
    _check(st, "gr_solve_constraints", allow=(GR_ERR_NOCONV,) if allow_noconv else ())
    d = report_dict(r)
    d["status_code"] = st
    return d


def gr_vcycle(ctx, eq: int, src: dict, fld: dict, opts: gr_opts) -> float:
    s, f, r = make_sources(src), make_fields(fld), ctypes.c_double(0)
    _check(lib().gr_vcycle(ctx, eq, ctypes.byref(s), ctypes.byref(f), ctypes.byref(opts), ctypes.byref(r)),
           "gr_vcycle")
    return r.value


def gr_residual(ctx, eq: int, src: dict, fld: dict, opts: gr_opts, res_field=None) -> float:
    s, f, r = make_sources(src), make_fields(fld), ctypes.c_double(0)
    _check(lib().gr_residual(ctx, eq, ctypes.byref(s), ctypes.byref(f), ctypes.byref(opts), _ptr(res_field),
                             ctypes.byref(r)), "gr_residual")
    return r.value


def gr_last_error() -> str:
    return lib().gr_last_error().decode()


def gr_kernel_launches() -> int:
    return int(lib().gr_kernel_launches())


def gr_fma_rate(fp64: bool, iters: int = 1 << 16, stream=None) -> float:
    """Measured FMA issue rate of the current device in FLOP/s (a diagnostic)."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    out = ctypes.c_double(0.0)
    _check(lib().gr_fma_rate(int(bool(fp64)), int(iters), st, ctypes.byref(out)), "gr_fma_rate")
    return out.value


def gr_momentum_residual_noalloc(n: int, L: float, V, s, res_field=None, stream=None) -> float:
    """Allocation-free residual of lap V_i = 8 pi (s_i - <s_i>); returns the
    relative norm (see include/gr.h).  V, s, res_field: contiguous float64
    CUDA tensors of n^3 elements on the current device; stream: a
    torch.cuda.Stream or raw cudaStream_t (default: torch's current stream)."""
    import torch

    dev = torch.cuda.current_device()
    for name, t in (("V", V), ("s", s), ("res_field", res_field)):
        if t is None and name == "res_field":
            continue
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError(f"gr_momentum_residual_noalloc: {name} must be a contiguous float64 tensor")
        if t.device.type != "cuda" or t.device.index != dev:
            raise ValueError(f"gr_momentum_residual_noalloc: {name} must be on cuda:{dev}, not {t.device}")
        if t.numel() != n ** 3:
            raise ValueError(f"gr_momentum_residual_noalloc: {name} has {t.numel()} elements, n^3 = {n ** 3}")
    if stream is None:
        stream = torch.cuda.current_stream()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    r = ctypes.c_double(0)
    _check(lib().gr_momentum_residual_noalloc(n, L, _ptr(V), _ptr(s), _ptr(res_field), ctypes.byref(r), st),
           "gr_momentum_residual_noalloc")
    return r.value


class gr_cosmology(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("Omega_m", ctypes.c_double), ("Omega_L", ctypes.c_double),
                ("H0", ctypes.c_double)]


def _particles(x, u):
    np_ = int(x.shape[-1]) if x is not None and x.dim() == 2 else 0
    if np_ and (tuple(x.shape) != (3, np_) or tuple(u.shape) != (3, np_)):
        raise ValueError("x and u must both be (3, np)")
    return np_


def gr_particle_update(ctx, x, u, fld: dict, dt: float, flags: int = GR_KICK_SYNC | GR_KICK_OPEN | GR_DRIFT):
    f = make_fields(fld)
    _check(lib().gr_particle_update(ctx, _particles(x, u), _ptr(x), _ptr(u), ctypes.byref(f), dt, flags),
           "gr_particle_update")


def gr_kick(ctx, x, u, fld: dict, dt: float, flags: int):
    f = make_fields(fld)
    _check(lib().gr_kick(ctx, _particles(x, u), _ptr(x), _ptr(u), ctypes.byref(f), dt, flags), "gr_kick")


def gr_drift(ctx, x, u, fld: dict, dt: float):
    f = make_fields(fld)
    _check(lib().gr_drift(ctx, _particles(x, u), _ptr(x), _ptr(u), ctypes.byref(f), dt), "gr_drift")


def gr_deposit_metric(ctx, x, u, mass: float, psi, src: dict):
    s = make_sources(src)
    _check(lib().gr_deposit_metric(ctx, _particles(x, u), _ptr(x), _ptr(u), mass, _ptr(psi), ctypes.byref(s)),
           "gr_deposit_metric")


# ------------------------------------------------------------------ convenience
class Context:
    """One n^3 periodic grid of side L on the current CUDA device."""

    def __init__(self, n: int, L: float = 1.0, stream=None):
        import torch

        self.n, self.L = n, L
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = gr_create(n, L, self.stream)

    def close(self):
        if self.h:
            gr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _grid(self):
        import torch

        return torch.empty((self.n,) * 3, dtype=torch.float64, device=self.device)

    def new_sources(self) -> dict:
        return {k: self._grid() for k in SOURCES}

    def initial_fields(self) -> dict:
        """The plain guess psi = alpha psi = 1, vectors and scalars 0."""
        fld = {k: self._grid().zero_() for k in FIELDS}
        fld["psi"].fill_(1.0)
        fld["apsi"].fill_(1.0)
        return fld

    def deposit(self, x, u, mass: float, src: dict | None = None) -> dict:
        src = src if src is not None else self.new_sources()
        gr_deposit(self.h, x, u, mass, src)
        return src

    def deposit_metric(self, x, u, mass: float, psi, src: dict | None = None) -> dict:
        """CIC sources with the Lorentz factor at the conformal factor psi
        (the previous solution's; None: psi = 1)."""
        src = src if src is not None else self.new_sources()
        gr_deposit_metric(self.h, x, u, mass, psi, src)
        return src

    def particle_update(self, x, u, fld: dict, dt: float, flags: int = GR_KICK_SYNC | GR_KICK_OPEN | GR_DRIFT):
        """Kicks and drift of the particles (x, u: (3, np) float64 CUDA
        tensors, updated in place) in the solved fields."""
        gr_particle_update(self.h, x, u, fld, dt, flags)

    def patch_grid(self, n: int) -> dict:
        import torch

        return torch.empty((n,) * 3, dtype=torch.float64, device=self.device)

    def deposit_patches(self, patches, x, u, mass: float):
        """Fill (allocating where missing) each patch dict's "src"."""
        for q in patches:
            if q.get("src") is None:
                q["src"] = {k: self.patch_grid(q["n"]) for k in SOURCES}
        gr_deposit_patches(self.h, patches, x, u, mass)
        return patches

    def initial_patch_fields(self, patches):
        """Set each patch dict's "fld" to the plain guess."""
        for q in patches:
            fld = {k: self.patch_grid(q["n"]).zero_() for k in FIELDS}
            fld["psi"].fill_(1.0)
            fld["apsi"].fill_(1.0)
            q["fld"] = fld
        return patches

    def solve(self, src, fld, **kw) -> dict:
        allow = kw.pop("allow_noconv", False)
        return gr_solve_constraints(self.h, src, fld, make_opts(**kw), allow_noconv=allow)

    def solve_code_units(self, src, fld, a: float, Omega_m: float, H0: float, Omega_L: float = 0.0, **kw) -> dict:
        """The ten-equation solve in the paper's code units at scale factor a
        (include/gr.h gr_solve_code_units): src holds the code-unit sources
        (keys as for solve), fld the code-unit fields (psi key: Psi, apsi key:
        Phi, the others the code-unit potentials), guesses in, solutions out."""
        allow = kw.pop("allow_noconv", False)
        cm = gr_cosmology(a, Omega_m, Omega_L, H0)
        o = make_opts(**kw)
        s, f = make_sources(src), make_fields(fld)
        r = gr_report()
        st = lib().gr_solve_code_units(self.h, ctypes.byref(cm), ctypes.byref(s), ctypes.byref(f), ctypes.byref(o),
                                       ctypes.byref(r))
        _check(st, "gr_solve_code_units", allow=(GR_ERR_NOCONV,) if allow else ())
        d = report_dict(r)
        d["status_code"] = st
        return d

    def vcycle(self, eq: int, src, fld, **kw) -> float:
        return gr_vcycle(self.h, eq, src, fld, make_opts(**kw))

    def residual(self, eq: int, src, fld, res_field=None, **kw) -> float:
        return gr_residual(self.h, eq, src, fld, make_opts(**kw), res_field)


# ------------------------------------------------------------------ learned initial guess
NET_TENSORS = ("x0", "e0a", "e0b", "p1", "e1a", "e1b", "p2", "e2a", "e2b", "p3", "e3a", "e3b", "cat2", "d2a", "d2b",
               "cat1", "d1a", "d1b", "cat0", "d0a", "d0b")
NET_TENSOR_SHAPE = {"x0": (0, 16), "e0a": (0, 16), "e0b": (0, 16), "p1": (1, 16), "e1a": (1, 32), "e1b": (1, 32),
                    "p2": (2, 32), "e2a": (2, 64), "e2b": (2, 64), "p3": (3, 64), "e3a": (3, 128), "e3b": (3, 128),
                    "cat2": (2, 192), "d2a": (2, 64), "d2b": (2, 64), "cat1": (1, 96), "d1a": (1, 32),
                    "d1b": (1, 32), "cat0": (0, 48), "d0a": (0, 16), "d0b": (0, 16)}


class Net:
    """The U-Net initial-guess network of include/gr.h (gr_net_*)."""

    def __init__(self, n: int, seed: int = 0, stream=None):
        import torch

        self.n = n
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _P()
        _check(lib().gr_net_create(n, self.stream.cuda_stream, seed, ctypes.byref(h)), "gr_net_create")
        self.h = h

    def close(self):
        if self.h:
            lib().gr_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(lib().gr_net_num_params(self.h))

    def get_params(self):
        import numpy as np

        out = np.empty(self.num_params, dtype=np.float32)
        _check(lib().gr_net_get_params(self.h, out.ctypes.data), "gr_net_get_params")
        return out

    def set_params(self, params):
        import numpy as np

        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.num_params
        _check(lib().gr_net_set_params(self.h, p.ctypes.data), "gr_net_set_params")

    def set_norm(self, in_mean, in_std, out_mean, out_std):
        import numpy as np

        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (in_mean, in_std, out_mean, out_std)]
        _check(lib().gr_net_set_norm(self.h, *[a.ctypes.data for a in arrs]), "gr_net_set_norm")
        self.norm = arrs

    def infer(self, src: dict, fld: dict, rho_hat: float, v_rms: float):
        s, f = make_sources(src), make_fields(fld)
        _check(lib().gr_net_infer(self.h, ctypes.byref(s), rho_hat, v_rms, ctypes.byref(f)), "gr_net_infer")

    def guess(self, n_fine: int, src: dict, fld: dict, rho_hat: float, v_rms: float):
        """The network's guess on a finer grid (n_fine = n 2^k): sources
        averaged down, inference, trilinear interpolation back up."""
        s, f = make_sources(src), make_fields(fld)
        _check(lib().gr_net_guess(self.h, n_fine, ctypes.byref(s), rho_hat, v_rms, ctypes.byref(f)), "gr_net_guess")

    def loss_grad(self, src: dict, target: dict, rho_hat: float, v_rms: float, want_grads=True):
        import numpy as np

        s, f = make_sources(src), make_fields(target)
        loss = ctypes.c_float(0)
        g = np.empty(self.num_params, dtype=np.float32) if want_grads else None
        _check(lib().gr_net_loss_grad(self.h, ctypes.byref(s), ctypes.byref(f), rho_hat, v_rms, ctypes.byref(loss),
                                      g.ctypes.data if g is not None else None), "gr_net_loss_grad")
        return loss.value, g

    def train_step(self, src: dict, target: dict, rho_hat: float, v_rms: float, lr: float) -> float:
        s, f = make_sources(src), make_fields(target)
        loss = ctypes.c_float(0)
        _check(lib().gr_net_train_step(self.h, ctypes.byref(s), ctypes.byref(f), rho_hat, v_rms, lr,
                                       ctypes.byref(loss)), "gr_net_train_step")
        return loss.value

    def activation(self, name: str):
        import numpy as np

        lev, c = NET_TENSOR_SHAPE[name]
        m = self.n >> lev
        out = np.empty((m, m, m, c), dtype=np.float32)
        _check(lib().gr_net_activation(self.h, NET_TENSORS.index(name), out.ctypes.data, out.size),
               "gr_net_activation")
        return out
