"""Pins of oracle.geometry: finite differences, closed-form det J and R, volumes."""
import math

import numpy as np
import pytest

from oracle.geometry import Annulus, Box, coefficient_tensor
from oracle.iga import Space1D
from oracle.spline import quarter_arc

XI = np.random.default_rng(3).uniform(0.02, 0.98, size=(3, 7))


@pytest.mark.parametrize("geom", [Annulus(), Annulus(1.0, 2.0, 1.0, 0.8, 0.2), Annulus(0.7, 1.9, 1.3, 1.1, 0.15)])
def test_jacobian_matches_finite_differences(geom):
    x1, x2, x3 = XI
    X, J = geom.map(x1, x2, x3)
    h = 1e-6
    for b, args in enumerate([(x1 + h, x2, x3), (x1, x2 + h, x3), (x1, x2, x3 + h)]):
        Xp, _ = geom.map(*args)
        am = [x1, x2, x3]
        am[b] = am[b] - h
        Xm, _ = geom.map(*am)
        fd = (Xp - Xm) / (2 * h)
        assert np.max(np.abs(fd - J[..., :, b])) < 1e-8


def test_det_j_closed_form():
    g = Annulus(1.0, 2.0, 1.0, 0.8, 0.2)
    x1, x2, x3 = XI
    _, J = g.map(x1, x2, x3)
    detJ, _ = coefficient_tensor(J)
    C, dC = quarter_arc(x2)
    theta_p = (C[:, 0] * dC[:, 1] - C[:, 1] * dC[:, 0])  # |C| = 1
    r = 1.0 + x1
    s = 1.0 + 0.2 * np.sin(np.pi * x3)
    expect = 1.0 * s[None, None, :] ** 2 * 1.0 * r[:, None, None] * theta_p[None, :, None]
    assert np.max(np.abs(detJ - expect)) < 1e-13


def test_cylinder_coefficients_are_diagonal_closed_form():
    """Untwisted cylinder: R = diag(H r th'/dr, H dr/(r th'), dr r th'/H), zero off-diagonal."""
    g = Annulus(1.0, 2.0, 1.5)
    x1, x2, x3 = XI
    _, J = g.map(x1, x2, x3)
    _, R = coefficient_tensor(J)
    C, dC = quarter_arc(x2)
    th = (C[:, 0] * dC[:, 1] - C[:, 1] * dC[:, 0])[None, :, None]
    r = (1.0 + x1)[:, None, None]
    H, dr = 1.5, 1.0
    assert np.max(np.abs(R[..., 0, 0] - H * r * th / dr)) < 1e-13
    assert np.max(np.abs(R[..., 1, 1] - H * dr / (r * th))) < 1e-13
    assert np.max(np.abs(R[..., 2, 2] - dr * r * th / H)) < 1e-13
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        assert np.max(np.abs(R[..., a, b])) < 1e-14
        assert np.max(np.abs(R[..., b, a])) < 1e-14


def test_box_coefficients():
    g = Box(2.0, 0.5, 3.0)
    _, J = g.map(*XI)
    detJ, R = coefficient_tensor(J)
    assert np.allclose(detJ, 3.0)
    assert np.allclose(R[..., 0, 0], 0.5 * 3.0 / 2.0) and np.allclose(R[..., 1, 1], 2.0 * 3.0 / 0.5)
    assert np.allclose(R[..., 2, 2], 2.0 * 0.5 / 3.0)


@pytest.mark.parametrize("twist,swell,expect", [
    (0.0, 0.0, 3 * math.pi / 4),
    (0.8, 0.2, 3 * math.pi / 4 * (1 + 0.8 / math.pi + 0.02)),
])
def test_volume(twist, swell, expect):
    """int det J = (3 pi / 4) int_0^1 (1 + swell sin(pi z))^2 dz; the twist preserves volume."""
    s = [Space1D(16, 3)] * 3
    x1, x2, x3 = (t.flat_points() for t in s)
    w1, w2, w3 = (t.flat_weights() for t in s)
    _, J = Annulus(1.0, 2.0, 1.0, twist, swell).map(x1, x2, x3)
    detJ, _ = coefficient_tensor(J)
    vol = np.einsum("i,j,k,ijk->", w1, w2, w3, detJ)
    assert abs(vol - expect) < 1e-9 * expect
