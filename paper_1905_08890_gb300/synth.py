"""Seeded synthetic particle inputs for the constraint solve.

This module is shared by the CUDA path, the oracle-based tests and the bench.
It holds none of the solver's arithmetic: it only draws particles.  The paper's
simulations start from CAMB/2LPT initial conditions (Sec. 6), which are not
available here; the stand-in is a Zel'dovich displacement of a cell-centred
lattice by a Gaussian or lognormal random field with P(k) ~ k^-2.

Recipe (box L = 1, N_p^3 particles, N_p = n):
  1. white noise w ~ N(0, 1) on the N_p^3 lattice, numpy PCG64 seeded;
  2. G = IFFT(FFT(w) / |k|), k = 0 zeroed, normalised to unit variance;
  3. delta = sigma_t * G (Gaussian) or exp(lam*G - lam^2/2) - 1 with
     lam = sqrt(ln(1 + sigma_t^2)), clipped at -0.95 (lognormal);
  4. displacement D_k = i k delta_k / k^2, so div D = -delta;
  5. positions x = q + D (mod 1), q the lattice cell centres;
  6. lower-index velocities u = A * D with A fixed by RMS|u| = v_rms;
  7. identical particle mass m = rho_bar / N_p^3, rho_bar = 1 / (24 pi), so
     that K^2 = 24 pi rho_bar = 1 (Sec. 2.3, fiducial Friedmann equation).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # multithreaded FFTs where scipy is present; numpy otherwise
    import scipy.fft as _fft

    _FFT_KW = {"workers": -1}
except ImportError:  # pragma: no cover - scipy is in both images
    _fft = np.fft
    _FFT_KW = {}

RHO_BAR = 1.0 / (24.0 * math.pi)


@dataclasses.dataclass
class Particles:
    """Particles in structure-of-arrays FP64 layout: x[3, np], u[3, np]."""

    n: int
    x: np.ndarray  # (3, np) float64 positions in [0, 1)
    u: np.ndarray  # (3, np) float64 lower-index 4-velocity components u_i
    mass: float
    delta_rms: float  # sample rms of the density field drawn in step 3
    seed: int

    @property
    def np(self) -> int:
        return self.x.shape[1]

    @property
    def rho_hat(self) -> float:
        """Rest-mass mean density m * N_p / L^3."""
        return self.mass * self.np


def _kgrid(n: int):
    f = np.fft.fftfreq(n, d=1.0 / n) * 2.0 * math.pi
    fr = np.fft.rfftfreq(n, d=1.0 / n) * 2.0 * math.pi
    return f[:, None, None], f[None, :, None], fr[None, None, :]


def zeldovich(n: int, seed: int, sigma: float, v_rms: float, lognormal: bool) -> Particles:
    """Draw N_p = n^3 particles by the recipe in the module docstring."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    kx, ky, kz = _kgrid(n)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    wk = _fft.rfftn(w, **_FFT_KW)
    del w
    wk /= np.sqrt(k2)
    wk[0, 0, 0] = 0.0
    g = _fft.irfftn(wk, s=(n, n, n), **_FFT_KW)
    del wk
    g /= g.std()
    if lognormal:
        lam = math.sqrt(math.log1p(sigma * sigma))
        delta = np.exp(lam * g - 0.5 * lam * lam) - 1.0
        np.maximum(delta, -0.95, out=delta)
    else:
        delta = sigma * g
    del g
    delta_rms = float(delta.std())
    dk = _fft.rfftn(delta, **_FFT_KW)
    del delta
    dk[0, 0, 0] = 0.0
    q = (np.arange(n, dtype=np.float64) + 0.5) / n
    x = np.empty((3, n * n * n), dtype=np.float64)
    u = np.empty((3, n * n * n), dtype=np.float64)
    for d, kd in enumerate((kx, ky, kz)):
        disp = _fft.irfftn(1j * kd * dk / k2, s=(n, n, n), **_FFT_KW)
        u[d] = disp.reshape(-1)
        shape = [1, 1, 1]
        shape[d] = n
        x[d] = (disp + q.reshape(shape)).reshape(-1)
        del disp
    del dk
    np.mod(x, 1.0, out=x)
    x[x >= 1.0] = 0.0  # np.mod can round a tiny negative up to exactly 1.0
    norm = math.sqrt(float(np.mean(np.sum(u * u, axis=0))))
    if norm > 0:
        u *= v_rms / norm
    mass = RHO_BAR / float(n) ** 3
    return Particles(n=n, x=x, u=u, mass=mass, delta_rms=delta_rms, seed=seed)


# Workloads: grid n (= N_p), density field, velocity rms, tolerance.
WORKLOADS = {
    "zeldovich32_gauss0.3": dict(n=32, sigma=0.3, v_rms=0.01, lognormal=False, tol=1e-10, seed=1),
    "zeldovich128_lognormal1": dict(n=128, sigma=1.0, v_rms=0.003, lognormal=True, tol=1e-10, seed=2),
    "zeldovich256_lognormal3": dict(n=256, sigma=3.0, v_rms=0.003, lognormal=True, tol=1e-8, seed=3),
    "zeldovich512_lognormal5": dict(n=512, sigma=5.0, v_rms=0.003, lognormal=True, tol=1e-8, seed=4),
}


def workload(name: str, seed: int | None = None) -> Particles:
    w = WORKLOADS[name]
    return zeldovich(w["n"], w["seed"] if seed is None else seed, w["sigma"], w["v_rms"], w["lognormal"])


def lattice(n: int, per_dim: int = 1, offset: float = 0.5, velocity=None) -> Particles:
    """Regular lattice: per_dim^3 particles per cell at (c + offset) / per_dim
    within each cell, optional velocity callback u(x) -> (3, np)."""
    m = n * per_dim
    c = (np.arange(m, dtype=np.float64) + offset) / m
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    x = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])
    u = np.zeros_like(x) if velocity is None else np.ascontiguousarray(velocity(x), dtype=np.float64)
    return Particles(n=n, x=x, u=u, mass=RHO_BAR / float(m) ** 3, delta_rms=0.0, seed=-1)


def zeldovich_torch(n: int, seed: int, sigma: float, v_rms: float, lognormal: bool, device="cuda"):
    """The same recipe as zeldovich() drawn with torch on `device` (a torch
    Generator seeded with `seed`, so the noise stream differs from numpy's):
    for building training sets quickly.  Returns (x, u, mass) as float64
    tensors (3, n^3) and the particle mass."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    w = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float64)
    f = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64) * 2.0 * math.pi
    fr = torch.fft.rfftfreq(n, d=1.0 / n, device=device, dtype=torch.float64) * 2.0 * math.pi
    kx, ky, kz = f[:, None, None], f[None, :, None], fr[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    wk = torch.fft.rfftn(w) / torch.sqrt(k2)
    wk[0, 0, 0] = 0.0
    gf = torch.fft.irfftn(wk, s=(n, n, n))
    gf /= gf.std()
    if lognormal:
        lam = math.sqrt(math.log1p(sigma * sigma))
        delta = torch.clamp(torch.exp(lam * gf - 0.5 * lam * lam) - 1.0, min=-0.95)
    else:
        delta = sigma * gf
    dk = torch.fft.rfftn(delta)
    dk[0, 0, 0] = 0.0
    q = (torch.arange(n, device=device, dtype=torch.float64) + 0.5) / n
    x = torch.empty((3, n * n * n), device=device, dtype=torch.float64)
    u = torch.empty_like(x)
    for d, kd in enumerate((kx, ky, kz)):
        disp = torch.fft.irfftn(1j * kd * dk / k2, s=(n, n, n))
        u[d] = disp.reshape(-1)
        shape = [1, 1, 1]
        shape[d] = n
        x[d] = (disp + q.reshape(shape)).reshape(-1)
    x = torch.remainder(x, 1.0)
    x[x >= 1.0] = 0.0
    norm = torch.sqrt(torch.mean(torch.sum(u * u, dim=0)))
    if norm > 0:
        u *= v_rms / norm
    return x, u, RHO_BAR / float(n) ** 3
