"""Pins of the hyper-dual Laplacian and the manufactured solutions."""
import numpy as np
import pytest

from oracle.geometry import Annulus, Box
from oracle.manufactured import Manufactured


def _pts(geom, m=40, seed=1):
    xi = np.random.default_rng(seed).uniform(0.05, 0.95, size=(3, m))
    X, _ = geom.map(*xi)
    return X.reshape(-1, 3)


def test_cylinder_laplacian_closed_form():
    """u = g(r) h(theta) k(z), g = (r^2-a^2)(b^2-r^2) r^2, h = sin(2 theta)/2, k = z(1-z):
    Laplace(u) = (-32 r^4 + 12 (a^2 + b^2) r^2) h k - 2 g h  (derived by hand in cylindrical coordinates)."""
    a, b = 1.0, 2.0
    g = Annulus(a, b, 1.0)
    X = _pts(g, 12)
    m = Manufactured(g)
    r2 = X[:, 0] ** 2 + X[:, 1] ** 2
    th = np.arctan2(X[:, 1], X[:, 0])
    h = 0.5 * np.sin(2 * th)
    k = X[:, 2] * (1 - X[:, 2])
    gg = (r2 - a * a) * (b * b - r2) * r2
    lap = (-32 * r2 ** 2 + 12 * (a * a + b * b) * r2) * h * k - 2 * gg * h
    f = m.f(X)
    assert np.max(np.abs(f + lap)) < 1e-11 * np.max(np.abs(lap))
    assert np.max(np.abs(m.u(X) - gg * h * k)) < 1e-13


def _fd_laplacian(fun, X, h=2e-3):
    tot = np.zeros(len(X))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        tot += (-fun(X + 2 * e) + 16 * fun(X + e) - 30 * fun(X) + 16 * fun(X - e) - fun(X - 2 * e)) / (12 * h * h)
    return tot


@pytest.mark.parametrize("geom,modes", [
    (Annulus(1.0, 2.0, 1.0, 0.8, 0.2), []),
    (Annulus(0.6, 1.7, 1.0, 1.1, 0.0), [(0.2, (1.0, -2.0, 0.5), 0.3), (-0.1, (0.0, 2.5, 1.0), 1.2)]),
    (Box(1.0, 2.0, 0.5), [(0.25, (2.0, 1.0, 0.0), 0.1)]),
])
def test_laplacian_matches_finite_differences(geom, modes):
    m = Manufactured(geom, modes)
    X = _pts(geom, 5, seed=7)
    fd = _fd_laplacian(m.u, X)
    assert np.max(np.abs(-m.f(X) - fd)) < 1e-6 * max(1.0, np.max(np.abs(fd)))


def test_box_sine_eigenfunction():
    g = Box(1.0, 2.0, 0.5)
    m = Manufactured(g)
    X = _pts(g, 6)
    lam = np.pi ** 2 * (1 + 1 / 4 + 4)
    assert np.max(np.abs(m.f(X) - lam * m.u(X))) < 1e-12 * lam


@pytest.mark.parametrize("geom", [Annulus(1.0, 2.0, 1.0, 0.8, 0.2), Box(1.0, 2.0, 0.5)])
def test_solution_vanishes_on_all_faces(geom):
    m = Manufactured(geom, [(0.3, (1.0, 1.0, 1.0), 0.0)])
    t = np.linspace(0, 1, 9)
    for d in range(3):
        for end in (0.0, 1.0):
            axes = [t, t, t]
            axes[d] = np.array([end])
            X, _ = geom.map(*axes)
            assert np.max(np.abs(m.u(X))) < 1e-13


def test_hyperdual_primitives_against_closed_forms():
    """Value, first and second derivative carried by each primitive and by the arithmetic:
    log(x^2 + 1) -> 2x / (1 + x^2), 2 (1 - x^2) / (1 + x^2)^2; sin(3x) / x and cos(x)^2
    against their hand-differentiated forms."""
    from oracle import hyperdual as hd
    x = np.linspace(0.3, 2.7, 9)
    X = hd.HD(x, 1.0, 1.0)
    f = hd.log(X * X + 1.0)
    assert np.allclose(f.a, np.log(x * x + 1), rtol=0, atol=1e-15)
    assert np.allclose(f.b, 2 * x / (1 + x * x), rtol=1e-14) and np.allclose(f.c, f.b)
    assert np.allclose(f.d, 2 * (1 - x * x) / (1 + x * x) ** 2, rtol=1e-13, atol=1e-15)
    g = hd.sin(3.0 * X) / X
    d1 = 3 * np.cos(3 * x) / x - np.sin(3 * x) / x ** 2
    d2 = -9 * np.sin(3 * x) / x - 6 * np.cos(3 * x) / x ** 2 + 2 * np.sin(3 * x) / x ** 3
    assert np.allclose(g.b, d1, rtol=1e-13) and np.allclose(g.d, d2, rtol=1e-12, atol=1e-14)
    h = hd.cos(X) * hd.cos(X)
    assert np.allclose(h.b, -np.sin(2 * x), atol=1e-15) and np.allclose(h.d, -2 * np.cos(2 * x), atol=1e-14)
