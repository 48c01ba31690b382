"""Pins of the oracle's generic NURBS patch: it reproduces the analytic quarter cylinder and the
box exactly, its Jacobian agrees with finite differences, and equal control points collapse it."""
import numpy as np

from oracle.geometry import Annulus, Box, NURBSPatch, quarter_cylinder_patch

X1 = np.linspace(0.0, 1.0, 7)
X2 = np.linspace(0.0, 1.0, 6)
X3 = np.array([0.0, 0.31, 0.77, 1.0])


def test_quarter_cylinder_patch_equals_the_annulus_map():
    a = Annulus(1.0, 2.0, 1.0)
    n = quarter_cylinder_patch(1.0, 2.0, 1.0)
    Xa, Ja = a.map(X1, X2, X3)
    Xn, Jn = n.map(X1, X2, X3)
    assert np.max(np.abs(Xa - Xn)) < 1e-14 and np.max(np.abs(Ja - Jn)) < 1e-13


def test_trilinear_patch_equals_the_box():
    L = (2.0, 0.5, 1.5)
    ctrl = np.zeros((2, 2, 2, 3))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                ctrl[i, j, k] = [L[0] * i, L[1] * j, L[2] * k]
    n = NURBSPatch((1, 1, 1), [[0, 0, 1, 1]] * 3, ctrl, np.ones((2, 2, 2)))
    Xb, Jb = Box(*L).map(X1, X2, X3)
    Xn, Jn = n.map(X1, X2, X3)
    assert np.max(np.abs(Xb - Xn)) < 1e-14 and np.max(np.abs(Jb - Jn)) < 1e-14


def _curved_patch(seed=2):
    import synthetic
    return NURBSPatch(*synthetic.curved_patch(seed))


def test_jacobian_matches_finite_differences():
    n = _curved_patch()
    x = (np.array([0.13, 0.62]), np.array([0.28, 0.81]), np.array([0.44]))
    _, J = n.map(*x)
    h = 1e-6
    for b in range(3):
        xp = [v.copy() for v in x]
        xm = [v.copy() for v in x]
        xp[b] = xp[b] + h
        xm[b] = xm[b] - h
        fd = (n.map(*xp)[0] - n.map(*xm)[0]) / (2 * h)
        assert np.max(np.abs(fd - J[..., :, b])) < 1e-6


def test_equal_control_points_collapse_the_patch():
    n = _curved_patch()
    n.ctrl[:] = [0.3, -1.0, 2.0]
    X, J = n.map(X1, X2, X3)
    assert np.max(np.abs(X - np.array([0.3, -1.0, 2.0]))) < 1e-14 and np.max(np.abs(J)) < 1e-12
