"""Pins of oracle.spline against library routines, closed forms and the Fig. 1 circle."""
import math
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline
from scipy.special import comb

from oracle.spline import (bspline_basis, gauss_legendre, nurbs_curve, open_uniform_knots,
                           quarter_arc)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_matches_numpy_and_is_exact(m):
    x, w = gauss_legendre(m)
    xr, wr = np.polynomial.legendre.leggauss(m)
    assert np.max(np.abs(x - xr)) < 1e-15
    assert np.max(np.abs(w - wr)) < 1e-14
    for k in range(2 * m):  # exact for degree <= 2m-1
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p,n", [(1, 5), (2, 7), (3, 9), (3, 16), (4, 11)])
def test_bspline_matches_scipy(p, n):
    t = open_uniform_knots(n, p)
    xs = np.concatenate([np.linspace(0.0, 1.0, 101), np.random.default_rng(0).uniform(0, 1, 50)])
    N, dN = bspline_basis(t, p, xs)
    assert N.shape == (len(xs), n)
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        b = BSpline(t, c, p)
        assert np.max(np.abs(b(xs) - N[:, i])) < 1e-14
        assert np.max(np.abs(b.derivative()(xs) - dN[:, i])) < 1e-11


@pytest.mark.parametrize("p,n", [(1, 4), (2, 16), (3, 20)])
def test_partition_of_unity(p, n):
    N, dN = bspline_basis(open_uniform_knots(n, p), p, np.linspace(0, 1, 333))
    assert np.max(np.abs(N.sum(axis=1) - 1.0)) < 1e-15
    assert np.max(np.abs(dN.sum(axis=1))) < 1e-12
    assert np.min(N) >= 0.0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_single_element_is_bernstein(p):
    x = np.linspace(0, 1, 57)
    N, _ = bspline_basis(open_uniform_knots(p + 1, p), p, x)
    for i in range(p + 1):
        bern = comb(p, i) * x ** i * (1 - x) ** (p - i)
        assert np.max(np.abs(N[:, i] - bern)) < 1e-15


def test_knot_vector_shape():
    t = open_uniform_knots(16, 2)
    assert len(t) == 19 and np.all(t[:3] == 0) and np.all(t[-3:] == 1)
    assert np.allclose(np.diff(t[2:-2]), 1.0 / 14)


def _read_golden(name):
    data = {"ctrl": []}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            key, *vals = line.split()
            conv = [1 / math.sqrt(2) if v == "1/sqrt(2)" else float(v) for v in vals]
            if key == "ctrl":
                data["ctrl"].append(conv)
            else:
                data[key] = conv
    return data


def test_fig1_circle_lies_on_unit_circle():
    g = _read_golden("nurbs_circle_fig1.txt")
    p = int(g["degree"][0])
    x = np.linspace(0, 1, 1001)
    C, dC = nurbs_curve(g["knots"], p, g["weights"], g["ctrl"], x)
    assert np.max(np.abs(np.hypot(C[:, 0], C[:, 1]) - g["radius"][0])) < 1e-15
    P, _ = nurbs_curve(g["knots"], p, g["weights"], g["ctrl"], np.array([0.0, 0.25, 0.5, 0.75]))
    assert np.allclose(P, [[1, 0], [0, 1], [-1, 0], [0, -1]], atol=1e-15)
    # tangent is perpendicular to the radius
    assert np.max(np.abs(np.sum(C * dC, axis=1))) < 1e-13


def test_quarter_arc_angular_speed():
    """theta'(0) = theta'(1) = sqrt 2 and theta'(1/2) = 4 (sqrt 2 - 1) for weights 1, sqrt2/2, 1."""
    C, dC = quarter_arc(np.array([0.0, 0.5, 1.0]))
    speed = (C[:, 0] * dC[:, 1] - C[:, 1] * dC[:, 0]) / np.sum(C * C, axis=1)
    assert np.allclose(speed, [math.sqrt(2), 4 * (math.sqrt(2) - 1), math.sqrt(2)], rtol=0, atol=1e-15)
    x, w = gauss_legendre(30)
    t = 0.5 * (x + 1)
    C, dC = quarter_arc(t)
    speed = (C[:, 0] * dC[:, 1] - C[:, 1] * dC[:, 0])
    assert abs(0.5 * np.sum(w * speed) - math.pi / 2) < 1e-14
