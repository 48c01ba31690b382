"""Manufactured solutions u and sources f = -Laplace(u) (oracle, Section 3.1).

TEST INFRASTRUCTURE ONLY.

For the annulus maps (geometry.Annulus) the solution is written in the
coordinates with the twist and swell undone, (x', y', zeta):

    u = (rho^2 - r_in^2)(r_out^2 - rho^2) x' y' zeta (1 - zeta)
        * (1 + sum_k a_k sin(b_k . x + c_k)),          rho^2 = x'^2 + y'^2,

which vanishes on all six faces of the patch (homogeneous Dirichlet data).
With r_in = 1, r_out = 2, H = 1, no twist and no modes it is
(r^2 - 1)(4 - r^2) x y z (1 - z).  For geometry.Box the bubble is
sin(pi x/Lx) sin(pi y/Ly) sin(pi z/Lz) times the same modulation.
f = -Laplace(u) in physical coordinates, by hyper-dual differentiation.
"""
import math

import numpy as np

from . import hyperdual as hd
from .geometry import Annulus, Box


class Manufactured:
    def __init__(self, geom, modes=()):
        """modes: iterable of (a, (b1, b2, b3), c) for the factor 1 + sum a sin(b.x + c)."""
        self.geom = geom
        self.modes = [(float(a), tuple(float(v) for v in b), float(c)) for a, b, c in modes]

    def _u(self, x, y, z):
        g = self.geom
        if isinstance(g, Annulus):
            zeta = z * (1.0 / g.height)
            phi = zeta * g.twist
            s = 1.0 + g.swell * hd.sin(zeta * np.pi)
            cp, sp = hd.cos(phi), hd.sin(phi)
            xp = (cp * x + sp * y) / s
            yp = (cp * y - sp * x) / s
            rho2 = xp * xp + yp * yp
            bubble = (rho2 - g.r_in ** 2) * (g.r_out ** 2 - rho2) * xp * yp * zeta * (1.0 - zeta)
        elif isinstance(g, Box):
            bubble = (hd.sin(x * (np.pi / g.L[0])) * hd.sin(y * (np.pi / g.L[1]))
                      * hd.sin(z * (np.pi / g.L[2])))
        else:
            raise TypeError("unknown geometry")
        mod = 1.0
        for a, (b1, b2, b3), c in self.modes:
            mod = mod + a * hd.sin(x * b1 + y * b2 + z * b3 + c)
        return bubble * mod

    def u(self, X):
        """Exact solution at physical points X[..., 3]."""
        return np.asarray(self._u(X[..., 0], X[..., 1], X[..., 2]), dtype=np.float64) * np.ones(X.shape[:-1])

    def f(self, X):
        """Source term f = -Laplace(u) at physical points X[..., 3]."""
        return -hd.laplacian(self._u, X)


class ConstantSource:
    """f = value everywhere and no exact solution (volume / load-vector pins)."""

    def __init__(self, value=1.0):
        self.value = float(value)

    def f(self, X):
        return np.full(X.shape[:-1], self.value)


class RingLog:
    """Exact solution of -Laplace(u) = 0 on the quarter cylinder (no twist, no swell) with
    u = u_in on rho = r_in, u = u_out on rho = r_out and zero flux on the other faces
    (Section 4.3, the ring problem): u = u_in + (u_out - u_in) ln(rho / r_in) / ln(r_out / r_in)."""

    def __init__(self, r_in=1.0, r_out=2.0, u_in=1.0, u_out=2.0):
        self.r_in, self.r_out = float(r_in), float(r_out)
        self.u_in, self.u_out = float(u_in), float(u_out)

    def u(self, X):
        rho = np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2)
        return self.u_in + (self.u_out - self.u_in) * np.log(rho / self.r_in) / np.log(self.r_out / self.r_in)

    def f(self, X):
        return np.zeros(X.shape[:-1])



class RingMixed:
    """Exact radial solution u = A + B ln(rho / r_in) of -Laplace(u) = 0 on the quarter cylinder
    (no twist, no swell) with zero flux on the angular and axial faces and, on each radial face,
    either a value (Dirichlet) or an outward normal flux du/dn (Section 4.3 with Neumann data).
    The outward normal is -rho on rho = r_in and +rho on rho = r_out, so du/dn = -B / r_in there
    and +B / r_out here; a value fixes A + B ln(rho / r_in).  inner / outer are pairs
    ("value", a) or ("flux", q); at least one must be a value."""

    def __init__(self, r_in=1.0, r_out=2.0, inner=("value", 1.0), outer=("flux", 1.0)):
        self.r_in, self.r_out = float(r_in), float(r_out)
        L = math.log(self.r_out / self.r_in)
        (ki, vi), (ko, vo) = inner, outer
        assert "value" in (ki, ko), "flux data on both radial faces leaves A undetermined"
        if ki == "value" and ko == "value":
            self.A, self.B = vi, (vo - vi) / L
        elif ki == "value":
            self.A, self.B = vi, vo * self.r_out
        else:
            self.B = -vi * self.r_in
            self.A = vo - self.B * L

    def u(self, X):
        rho = np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2)
        return self.A + self.B * np.log(rho / self.r_in)

    def f(self, X):
        return np.zeros(X.shape[:-1])
