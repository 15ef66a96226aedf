"""Closed-form derivatives of separable trigonometric fields on the periodic grid.

A field is a sum of terms  c * g_x(2 pi m_x x) g_y(2 pi m_y y) g_z(2 pi m_z z)
with g in {sin, cos}, sampled at cell centres x_i = (i + 1/2)/n.  On such
fields the central difference, the 3-point second difference and the 4-cell
cross difference act exactly as multiplication by the modified wavenumbers

    D   sin(2 pi m x) = sin(2 pi m h)/h * cos(2 pi m x)
    D2  g(2 pi m x)   = -(4/h^2) sin^2(pi m h) * g(2 pi m x)

so the discrete operators have closed forms independent of any stencil code,
and replacing the modified wavenumbers by 2 pi m gives the continuum
derivatives for convergence checks.
"""
from __future__ import annotations

import math

import numpy as np


class TrigSum:
    def __init__(self, terms=None):
        # term: (coef, (kx, ky, kz) with 's' or 'c', (mx, my, mz))
        self.terms = list(terms or [])

    @staticmethod
    def prod(kinds: str, modes, coef: float = 1.0) -> "TrigSum":
        return TrigSum([(coef, tuple(kinds), tuple(modes))])

    def __add__(self, other):
        return TrigSum(self.terms + other.terms)

    def __sub__(self, other):
        return self + other * -1.0

    def __mul__(self, s: float):
        return TrigSum([(c * s, k, m) for c, k, m in self.terms])

    __rmul__ = __mul__

    def grid(self, n: int) -> np.ndarray:
        x = (np.arange(n) + 0.5) / n
        out = np.zeros((n, n, n))
        for c, kinds, modes in self.terms:
            f = []
            for a in range(3):
                arg = 2 * math.pi * modes[a] * x
                f.append(np.sin(arg) if kinds[a] == "s" else np.cos(arg))
            out += c * f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]
        return out

    def d(self, a: int, n: int | None = None) -> "TrigSum":
        """First derivative along axis a: discrete central difference on the
        n-grid, or the continuum derivative when n is None."""
        out = []
        for c, kinds, modes in self.terms:
            m = modes[a]
            k1 = 2 * math.pi * m if n is None else math.sin(2 * math.pi * m / n) * n
            kinds2 = list(kinds)
            if kinds[a] == "s":
                kinds2[a] = "c"
                out.append((c * k1, tuple(kinds2), modes))
            else:
                kinds2[a] = "s"
                out.append((-c * k1, tuple(kinds2), modes))
        return TrigSum(out)

    def dd(self, a: int, n: int | None = None) -> "TrigSum":
        """Second derivative along axis a: 3-point second difference on the
        n-grid, or the continuum second derivative when n is None."""
        out = []
        for c, kinds, modes in self.terms:
            m = modes[a]
            k2 = (2 * math.pi * m) ** 2 if n is None else 4.0 * n * n * math.sin(math.pi * m / n) ** 2
            out.append((-c * k2, kinds, modes))
        return TrigSum(out)

    def lap(self, n: int | None = None) -> "TrigSum":
        return self.dd(0, n) + self.dd(1, n) + self.dd(2, n)
