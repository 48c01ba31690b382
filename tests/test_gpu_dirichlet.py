"""Non-homogeneous Dirichlet data (Section 4.3): the lift g, the right-hand side F - K g and the
partial restriction, against the oracle and against closed forms (linear data on the box, the
log solution of the ring problem)."""
import math

import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding, oracle_geometry

pytestmark = pytest.mark.gpu

RADIAL = [1, 1, 0, 0, 0, 0]


@pytest.fixture(scope="module")
def tt():
    return load_binding()


@pytest.fixture(scope="module")
def ctx(tt):
    import torch
    c = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    yield c
    tt.tt_iga_ctx_destroy(c)


def _solve(tt, ctx, geo, n, p, bc, rhs, tol=1e-12):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=5))
    s = tt.tt_iga_assemble_bc(ctx, g, [rhs], bc, round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=tol))
    return g, s, u, st


def _release(tt, g, s, u):
    tt.tt_iga_solution_destroy(u)
    tt.tt_iga_system_destroy(s)
    tt.tt_iga_geom_destroy(g)


def _eval(tt, ctx, u, pts):
    import torch
    xi = torch.tensor(pts, dtype=torch.float64, device="cuda")
    out = torch.empty(len(pts), dtype=torch.float64, device="cuda")
    tt.tt_iga_eval(ctx, u, xi, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_linear_data_is_exact_on_the_box(tt, ctx, p):
    """u = x on the unit box: 0 on x = 0, 1 on x = 1, zero flux elsewhere, f = 0."""
    g, s, u, st = _solve(tt, ctx, synthetic.UNIT_BOX, p + 5, p, tt.bc_desc(RADIAL, [0.0, 1.0, 0, 0, 0, 0]),
                         tt.rhs_desc(constant=0.0))
    try:
        assert st["converged"] and tt.tt_iga_system_info(s)["modes"] == (p + 3, p + 5, p + 5)
        pts = synthetic.random_points(200, seed=8)
        uh = _eval(tt, ctx, u, pts)
    finally:
        _release(tt, g, s, u)
    assert np.max(np.abs(uh - pts[:, 0])) < 1e-9


@pytest.mark.parametrize("n,p", [(8, 2), (7, 3)])
def test_ring_matches_oracle(tt, ctx, n, p):
    """Quarter cylinder, u = 1 on rho = 1 and 2 on rho = 2: GPU values and L2 error equal the oracle's
    for the same discrete problem."""
    from oracle.iga import Space1D, evaluate, l2_error, solve_bc
    from oracle.manufactured import RingLog
    geo = synthetic.QUARTER_CYLINDER
    g, s, u, st = _solve(tt, ctx, geo, n, p, tt.bc_desc(RADIAL, [1.0, 2.0, 0, 0, 0, 0]), tt.rhs_desc(ring_log=True),
                         tol=1e-13)
    try:
        assert st["converged"] and st["rel_residual"] <= 1e-13
        x = np.linspace(0.0, 1.0, 6)
        pts = np.array([[a, b, c] for c in x[::2] for b in x[1::2] for a in x])
        uh = _eval(tt, ctx, u, pts)
        l2 = tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc(ring_log=True))
    finally:
        _release(tt, g, s, u)
    og = oracle_geometry(geo)
    sp = [Space1D(n, p)] * 3
    uo, info = solve_bc(sp, og, None, [bool(f) for f in RADIAL], [1.0, 2.0, 0, 0, 0, 0], tol=1e-14)
    ref = evaluate(sp, uo, x, x[1::2], x[::2])  # [i1, i2, i3]
    ref = np.array([ref[i, j, k] for k in range(3) for j in range(3) for i in range(6)])
    assert np.max(np.abs(uh - ref)) < 1e-10 * np.max(np.abs(ref))
    lo = l2_error(sp, og, uo, RingLog(1.0, 2.0, 1.0, 2.0))
    assert abs(l2 - lo) <= 1e-6 * lo


def test_ring_converges_at_rate_p_plus_one(tt, ctx):
    p = 3
    errs = []
    ns = [16, 32, 64]
    for n in ns:
        g, s, u, st = _solve(tt, ctx, synthetic.QUARTER_CYLINDER, n, p, tt.bc_desc(RADIAL, [1.0, 2.0, 0, 0, 0, 0]),
                             tt.rhs_desc(ring_log=True), tol=1e-12)
        try:
            assert st["converged"]
            errs.append(tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc(ring_log=True)))
        finally:
            _release(tt, g, s, u)
    rate = math.log(errs[0] / errs[-1]) / math.log((ns[-1] - p) / (ns[0] - p))
    assert rate > p + 0.5 and errs[-1] < 1e-8, (errs, rate)


def test_all_homogeneous_faces_equal_plain_assembly(tt, ctx):
    geo = synthetic.TWISTED_ANNULUS
    desc = tt.geom_desc(geo, 2, 9, cross_tol=1e-14, seed=6)
    g = tt.tt_iga_geometry(ctx, desc)
    rhs = [tt.rhs_desc()]
    s0 = tt.tt_iga_assemble(ctx, g, rhs, round_tol=1e-14)
    s1 = tt.tt_iga_assemble_bc(ctx, g, rhs, tt.bc_desc([1] * 6), round_tol=1e-14)
    try:
        m = tt.tt_iga_system_info(s0)["modes"]
        assert tt.tt_iga_system_info(s1)["modes"] == m == (7, 7, 7)
        f0 = tt.tt_iga_densify_rhs(ctx, s0, 0)
        f1 = tt.tt_iga_densify_rhs(ctx, s1, 0)
    finally:
        tt.tt_iga_system_destroy(s0)
        tt.tt_iga_system_destroy(s1)
        tt.tt_iga_geom_destroy(g)
    assert np.array_equal(f0, f1)


@pytest.mark.parametrize("dirichlet,values", [
    ([0] * 6, [0.0] * 6),                              # no Dirichlet face: singular operator
    ([1, 1, 1, 0, 0, 0], [1.0, 0.0, 2.0, 0, 0, 0]),    # data on two directions
    ([1, 1, 1, 0, 0, 0], [1.0, 2.0, 0.0, 0, 0, 0]),    # data next to Dirichlet faces of another direction
    ([1, 1, 0, 0, 0, 0], [1.0, float("nan"), 0, 0, 0, 0]),
])
def test_rejected_boundary_conditions(tt, ctx, dirichlet, values):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, 2, 6, seed=1))
    try:
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc()], tt.bc_desc(dirichlet, values))
        assert e.value.code == tt.ERR_ARG
    finally:
        tt.tt_iga_geom_destroy(g)
