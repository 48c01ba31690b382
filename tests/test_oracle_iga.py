"""Pins of oracle.iga: Kronecker structure, symmetry, null space, SPD, volume, LU, energy, L2 rate."""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.geometry import Annulus, Box
from oracle.iga import (Space1D, assemble, l2_error, load_entries, pcg, restrict, solve,
                        stencil_matvec, stencil_to_dense, stiffness_rows, to_flat)
from oracle.manufactured import ConstantSource, Manufactured
from oracle.spline import open_uniform_knots


def textbook_1d(n, p):
    """1D stiffness and mass on [0,1] by scipy BSpline + numpy's 12-point Gauss rule per knot span
    (exact for the piecewise polynomials of degree <= 2p integrated here)."""
    t = open_uniform_knots(n, p)
    fs = []
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1
        fs.append(BSpline(t, c, p))
    ds = [f.derivative() for f in fs]
    spans = np.unique(t)
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    xg, wg = np.polynomial.legendre.leggauss(12)
    for a, b in zip(spans[:-1], spans[1:]):
        x = 0.5 * (a + b) + 0.5 * (b - a) * xg
        w = 0.5 * (b - a) * wg
        V = np.array([f(x) for f in fs])
        D = np.array([f(x) for f in ds])
        K += (D * w) @ D.T
        M += (V * w) @ V.T
    return K, M


def test_p1_closed_form_1d():
    n = 6
    K, M = textbook_1d(n, 1)
    h = 1.0 / (n - 1)
    Kc = (np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) / h
    Kc[0, 0] = Kc[-1, -1] = 1 / h
    Mc = (np.diag(np.full(n, 4.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) * h / 6
    Mc[0, 0] = Mc[-1, -1] = h / 3
    assert np.allclose(K, Kc, atol=1e-12) and np.allclose(M, Mc, atol=1e-13)


@pytest.mark.parametrize("n,p", [(5, 1), (6, 2), (6, 3)])
def test_identity_map_is_kronecker_sum(n, p):
    """Unit box: K = M (x) M (x) K1 + M (x) K1 (x) M + K1 (x) M (x) M (i1 fastest)."""
    sp = [Space1D(n, p)] * 3
    Kst, _ = assemble(sp, Box(), None)
    K = stencil_to_dense(Kst, (p, p, p))
    K1, M = textbook_1d(n, p)
    ref = np.kron(M, np.kron(M, K1)) + np.kron(M, np.kron(K1, M)) + np.kron(K1, np.kron(M, M))
    assert np.max(np.abs(K - ref)) < 1e-12 * np.max(np.abs(ref))


def test_symmetry_constant_nullspace_spd():
    sp = [Space1D(6, 2), Space1D(5, 2), Space1D(6, 3)]
    g = Annulus(1.0, 2.0, 1.0, 0.8, 0.2)
    Kst, _ = assemble(sp, g, None)
    K = stencil_to_dense(Kst, (2, 2, 3))
    scale = np.max(np.abs(K))
    assert np.max(np.abs(K - K.T)) < 1e-13 * scale
    assert np.max(np.abs(K @ np.ones(K.shape[0]))) < 1e-12 * scale
    Ki, _ = restrict(Kst, np.zeros(Kst.shape[:3]))
    ev = np.linalg.eigvalsh(stencil_to_dense(Ki, (2, 2, 3)))
    assert ev[0] > 0


@pytest.mark.parametrize("twist,swell", [(0.0, 0.0), (0.8, 0.2)])
def test_load_vector_sums_to_volume(twist, swell):
    sp = [Space1D(12, 3)] * 3
    _, F = assemble(sp, Annulus(1.0, 2.0, 1.0, twist, swell), ConstantSource(1.0))
    vol = 3 * math.pi / 4 * (1 + 4 * swell / math.pi + swell ** 2 / 2)
    assert abs(F.sum() - vol) < 1e-8 * vol


def test_pcg_matches_dense_lu_and_energy_identity():
    sp = [Space1D(7, 2)] * 3
    g = Annulus(1.0, 2.0, 1.0, 0.8, 0.2)
    m = Manufactured(g, [(0.2, (1.0, 0.5, -1.0), 0.4)])
    Kst, F = assemble(sp, g, m)
    Ki, Fi = restrict(Kst, F)
    x, it, rr = pcg(Ki, Fi, (2, 2, 2), tol=1e-14)
    assert rr < 1e-14
    A = stencil_to_dense(Ki, (2, 2, 2))
    xd = np.linalg.solve(A, to_flat(Fi))
    assert np.max(np.abs(to_flat(x) - xd)) < 1e-12 * np.max(np.abs(xd))
    e1 = np.vdot(x, stencil_matvec(Ki, x, (2, 2, 2)))
    assert abs(e1 - np.vdot(x, Fi)) < 1e-12 * abs(e1)


def test_rows_and_entries_match_full_assembly():
    sp = [Space1D(8, 3)] * 3
    g = Annulus(1.0, 2.0, 1.0, 0.8, 0.2)
    m = Manufactured(g)
    Kst, F = assemble(sp, g, m)
    rows = [(0, 0, 0), (3, 4, 5), (7, 2, 1), (4, 4, 4)]
    for a, blk in zip(rows, stiffness_rows(sp, g, rows)):
        assert np.max(np.abs(blk - Kst[a])) < 1e-13 * np.max(np.abs(Kst))
    vals = load_entries(sp, g, m, rows)
    assert np.max(np.abs(vals - np.array([F[a] for a in rows]))) < 1e-14 * np.max(np.abs(F))


def test_l2_rate_p2():
    """Slope p+1 = 3 of the L2 error against h (the paper reports ~3 for quadratic bases)."""
    g = Annulus(1.0, 2.0, 1.0, 0.8, 0.2)
    m = Manufactured(g)
    errs = []
    for n in (6, 10, 18):
        sp = [Space1D(n, 2)] * 3
        u, info = solve(sp, g, m)
        errs.append(l2_error(sp, g, u, m))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > 2.7, (errs, rates)
