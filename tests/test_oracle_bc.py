"""Pins of the oracle's non-homogeneous Dirichlet path (Section 4.3): lift vector, partial
restriction, the exactness of linear data on the box, and the ring problem's log solution."""
import math

import numpy as np
import pytest

from oracle import hyperdual as hd
from oracle.geometry import Annulus, Box
from oracle.iga import Space1D, evaluate, l2_error, lift_vector, restrict, restrict_bc, solve, solve_bc
from oracle.manufactured import Manufactured, RingLog

ALL = [True] * 6
RADIAL = [True, True, False, False, False, False]


def test_all_faces_homogeneous_matches_plain_solve():
    sp = [Space1D(7, 2)] * 3
    geom = Annulus()
    src = Manufactured(geom)
    u0, _ = solve(sp, geom, src)
    u1, info = solve_bc(sp, geom, src, ALL, [0.0] * 6)
    assert info["lo"] == [1, 1, 1] and info["hi"] == [1, 1, 1]
    assert np.max(np.abs(u1 - u0)) < 1e-12 * np.max(np.abs(u0))


def test_restrict_bc_with_all_faces_is_restrict():
    sp = [Space1D(6, 2)] * 3
    from oracle.iga import assemble
    Kst, F = assemble(sp, Box(), None)
    a, b = restrict(Kst, F)
    c, d = restrict_bc(Kst, F, [1, 1, 1], [1, 1, 1])
    assert np.array_equal(a, c) and np.array_equal(b, d)


def test_lift_vector_layout():
    g = lift_vector((5, 4, 3), RADIAL, [1.5, 2.5, 0, 0, 0, 0])
    assert np.all(g[0] == 1.5) and np.all(g[-1] == 2.5) and np.all(g[1:-1] == 0.0)
    with pytest.raises(AssertionError):
        lift_vector((5, 4, 3), ALL, [1.0, 2.0, 0, 0, 0, 0])  # data on a direction that meets Dirichlet faces


@pytest.mark.parametrize("p", [1, 2, 3])
def test_linear_data_is_reproduced_exactly_on_the_box(p):
    """u = x solves -Laplace u = 0 with u = 0 on x = 0, u = 1 on x = 1 and zero flux elsewhere,
    and lies in the spline space: the Galerkin solution is exact."""
    n = p + 4
    sp = [Space1D(n, p)] * 3
    u, info = solve_bc(sp, Box(), None, RADIAL, [0.0, 1.0, 0, 0, 0, 0])
    assert info["relres"] < 1e-13
    x = np.linspace(0.0, 1.0, 7)
    uh = evaluate(sp, u, x, x[::2], x[1::3])
    assert np.max(np.abs(uh - x[:, None, None])) < 1e-11


def test_ring_log_solution_is_harmonic_with_the_boundary_values():
    ex = RingLog(1.0, 2.0, 1.0, 2.0)

    def u(x, y, z):
        return ex.u_in + (ex.u_out - ex.u_in) * (0.5 * hd.log(x * x + y * y) - math.log(ex.r_in)) / math.log(2.0)

    rng = np.random.default_rng(3)
    r = rng.uniform(1.0, 2.0, 20)
    t = rng.uniform(0.0, math.pi / 2, 20)
    X = np.stack([r * np.cos(t), r * np.sin(t), rng.uniform(0, 1, 20)], axis=-1)
    assert np.max(np.abs(hd.laplacian(u, X))) < 1e-12
    assert np.allclose(ex.u(X), u(X[:, 0], X[:, 1], X[:, 2]), atol=1e-14)
    for rr, val in ((1.0, 1.0), (2.0, 2.0)):
        assert abs(ex.u(np.array([[rr * 0.6, rr * 0.8, 0.3]]))[0] - val) < 1e-14


def test_ring_converges_at_rate_p_plus_one():
    """Quarter cylinder, u = 1 on rho = 1, u = 2 on rho = 2, natural elsewhere (the ring of
    Exp. 2): the L2 error against the log solution falls like h^(p+1)."""
    geom = Annulus()
    ex = RingLog(1.0, 2.0, 1.0, 2.0)
    p = 2
    errs = []
    ns = [5, 7, 10]
    for n in ns:
        sp = [Space1D(n, p)] * 3
        u, info = solve_bc(sp, geom, None, RADIAL, [1.0, 2.0, 0, 0, 0, 0])
        assert info["relres"] < 1e-12
        errs.append(l2_error(sp, geom, u, ex))
    h = [1.0 / (n - p) for n in ns]
    rate = math.log(errs[0] / errs[-1]) / math.log(h[0] / h[-1])
    assert errs[-1] < 1e-4 and rate > p + 0.6, (errs, rate)
