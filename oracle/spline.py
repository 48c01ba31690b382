"""Univariate B-spline / NURBS machinery of the oracle (Section 2 of the paper).

TEST INFRASTRUCTURE ONLY. Plain FP64 numpy, written for readability, not speed.

Functions and the passage each follows:

* ``open_uniform_knots`` -- the non-decreasing knot vector Xi of Section 2.1
  (first equation), open: end knots repeated p+1 times (Section 2.3, NURBS
  paragraph), uniform interior knots from h-refinement (end of Section 2).
* ``gauss_legendre`` -- the per-element quadrature rule (p+1 Gauss points per
  element).  The paper does not print a rule; Gauss-Legendre by Newton
  iteration on the Legendre polynomial P_m (three-term recurrence).
* ``bspline_basis`` -- the degree-0 indicator functions and the Cox-de Boor
  recursion of Section 2.1, plus the first-derivative formula of Section 2.1.
* ``nurbs_basis`` / ``nurbs_curve`` -- the rational basis R_i^p, its quotient-rule
  derivative and the NURBS curve of Section 2.3.

Pins (tests/test_oracle_spline.py): scipy.interpolate.BSpline and
numpy.polynomial.legendre.leggauss as library special cases, partition of unity,
Bernstein polynomials on a single element, the Fig. 1 circle (golden fixture)
and the quarter arc's closed-form angular speed.
"""
import numpy as np


def open_uniform_knots(n, p):
    """Open uniform knot vector on [0, 1] for n basis functions of degree p.

    Length n+p+1, ends repeated p+1 times, n-p elements of width 1/(n-p).
    """
    if n < p + 1:
        raise ValueError("need n >= p+1 basis functions")
    ne = n - p
    inner = np.arange(1, ne, dtype=np.float64) / ne
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def gauss_legendre(m):
    """m-point Gauss-Legendre nodes and weights on [-1, 1].

    Newton iteration on P_m(x) = 0 from the Chebyshev-like initial guesses
    cos(pi (k - 1/4) / (m + 1/2)); P_m and P_m' by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; weights 2 / ((1 - x^2) P_m'(x)^2).
    """
    k = np.arange(1, m + 1, dtype=np.float64)
    x = np.cos(np.pi * (k - 0.25) / (m + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for j in range(1, m):
            p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
        dp = m * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for j in range(1, m):
        p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
    dp = m * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def _ratio(num, den):
    """num/den with the B-spline convention 0/0 := 0 (den == 0 only for repeated knots)."""
    out = np.zeros(np.broadcast(num, den).shape)
    nz = den != 0
    np.divide(num, den, out=out, where=nz)
    return out


def bspline_basis(knots, p, x):
    """All B-spline basis functions N_i^p and their first derivatives at points x.

    Returns (N, dN), each of shape (len(x), n) with n = len(knots) - p - 1.
    Degree 0 follows the half-open indicator of Section 2.1, except that the
    last non-empty knot span is closed on the right so that x = xi_end is
    covered.  Higher degrees follow the Cox-de Boor recursion
        N_i^k = (x - xi_i)/(xi_{i+k} - xi_i) N_i^{k-1}
              + (xi_{i+k+1} - x)/(xi_{i+k+1} - xi_{i+1}) N_{i+1}^{k-1},
    and the derivative
        dN_i^p = p/(xi_{i+p} - xi_i) N_i^{p-1} - p/(xi_{i+p+1} - xi_{i+1}) N_{i+1}^{p-1}.
    """
    t = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))[:, None]
    m = len(t) - 1  # number of degree-0 functions
    lo = t[:-1][None, :]
    hi = t[1:][None, :]
    N = ((lo <= x) & (x < hi)).astype(np.float64)
    last = np.max(np.nonzero(t[1:] > t[:-1])[0])  # last non-empty span
    N[:, last] = np.where((x[:, 0] >= t[last]) & (x[:, 0] <= t[last + 1]), 1.0, N[:, last])
    Nprev = N
    for k in range(1, p + 1):
        cnt = m - k
        i = np.arange(cnt)
        a = _ratio(x - t[i][None, :], (t[i + k] - t[i])[None, :])
        b = _ratio(t[i + k + 1][None, :] - x, (t[i + k + 1] - t[i + 1])[None, :])
        Nk = a * Nprev[:, :cnt] + b * Nprev[:, 1:cnt + 1]
        if k == p:
            Nlow = Nprev
        Nprev = Nk
    if p == 0:
        return Nprev, np.zeros_like(Nprev)
    n = m - p
    i = np.arange(n)
    c1 = _ratio(np.full(n, float(p)), t[i + p] - t[i])[None, :]
    c2 = _ratio(np.full(n, float(p)), t[i + p + 1] - t[i + 1])[None, :]
    dN = c1 * Nlow[:, :n] - c2 * Nlow[:, 1:n + 1]
    return Nprev, dN


def nurbs_basis(knots, p, weights, x):
    """Rational basis R_i^p = N_i w_i / W and its quotient-rule derivative (Section 2.3)."""
    N, dN = bspline_basis(knots, p, x)
    w = np.asarray(weights, dtype=np.float64)[None, :]
    W = np.sum(N * w, axis=1, keepdims=True)
    dW = np.sum(dN * w, axis=1, keepdims=True)
    R = N * w / W
    dR = (dN * w * W - N * w * dW) / (W * W)
    return R, dR


def nurbs_curve(knots, p, weights, ctrl, x):
    """NURBS curve C(x) = sum N_i w_i P_i / sum N_i w_i and C'(x) (Section 2.3)."""
    R, dR = nurbs_basis(knots, p, weights, x)
    P = np.asarray(ctrl, dtype=np.float64)
    return R @ P, dR @ P


# The quarter unit arc used by every annulus geometry: quadratic NURBS with
# control points (1,0), (1,1), (0,1) and weights 1, sqrt(2)/2, 1 (the
# single-quadrant piece of the Fig. 1 circle).
QUARTER_ARC_KNOTS = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
QUARTER_ARC_WEIGHTS = np.array([1.0, np.sqrt(0.5), 1.0])
QUARTER_ARC_CTRL = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])


def quarter_arc(x):
    """Point and derivative of the quarter unit arc at parameters x in [0, 1]."""
    return nurbs_curve(QUARTER_ARC_KNOTS, 2, QUARTER_ARC_WEIGHTS, QUARTER_ARC_CTRL, x)
