"""Flux (Neumann) data on natural faces (the surface load vector f_s of Section 3.3): the face load
through the C-ABI against the oracle's surface quadrature, exact linear solutions on the box, the
mixed ring problem against the oracle and its log solution, and the NURBS cylinder patch."""
import math

import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding, oracle_geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    return load_binding()


@pytest.fixture(scope="module")
def ctx(tt):
    import torch
    c = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    yield c
    tt.tt_iga_ctx_destroy(c)


def _eval(tt, ctx, u, pts):
    import torch
    xi = torch.tensor(pts, dtype=torch.float64, device="cuda")
    out = torch.empty(len(pts), dtype=torch.float64, device="cuda")
    tt.tt_iga_eval(ctx, u, xi, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ring_bc(inner, outer):
    """Per-face arrays of the mixed ring problem from ("value", a) / ("flux", q) on the radial faces."""
    dirichlet = [inner[0] == "value", outer[0] == "value", False, False, False, False]
    value = [inner[1] if dirichlet[0] else 0.0, outer[1] if dirichlet[1] else 0.0, 0.0, 0.0, 0.0, 0.0]
    flux = [0.0 if dirichlet[0] else inner[1], 0.0 if dirichlet[1] else outer[1], 0.0, 0.0, 0.0, 0.0]
    return dirichlet, value, flux


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("side", [0, 1])
def test_linear_solution_with_flux_is_exact_on_the_box(tt, ctx, p, side):
    """u = a (x - x_D): u = 0 on x = x_D, outward flux +a on x = Lx (side 1) or -a on x = 0
    (side 0), zero flux elsewhere, f = 0."""
    L, a = 2.0, 1.5
    geo = {"kind": "box", "lx": L, "ly": 1.0, "lz": 1.0}
    flux = [0.0] * 6
    flux[side] = a if side == 1 else -a
    bc = tt.bc_desc([side == 1, side == 0, 0, 0, 0, 0], [0.0] * 6, flux)
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, (p + 5, p + 3, p + 4), cross_tol=1e-14, seed=4))
    s = tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc(constant=0.0)], bc, round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13))
    try:
        assert st["converged"]
        pts = synthetic.random_points(200, seed=12)
        uh = _eval(tt, ctx, u, pts)
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    xd = 0.0 if side == 1 else L
    assert np.max(np.abs(uh - a * (L * pts[:, 0] - xd))) < 1e-9


@pytest.mark.parametrize("geo,faces", [
    (synthetic.TWISTED_ANNULUS, {1: 0.7, 3: -0.4, 5: 1.1}),
    ({"kind": "box", "lx": 2.0, "ly": 3.0, "lz": 0.5}, {0: 0.3, 2: -1.2, 4: 0.9, 5: 0.25}),
])
def test_load_with_flux_matches_oracle(tt, ctx, geo, faces):
    """The restricted load F + F_Gamma (one Dirichlet face, so no lift) equals the oracle's element
    by element on a ragged mesh; the flux faces cover every normal direction and both sides."""
    from oracle.iga import Space1D, assemble, neumann_load, restrict_bc, to_flat
    from oracle.manufactured import ConstantSource
    n, p = (7, 8, 6), 2
    dirichlet = [False, False, False, False, False, False]
    dfree = next(f for f in range(6) if f not in faces)
    dirichlet[dfree] = True
    flux = [faces.get(f, 0.0) for f in range(6)]
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=8))
    s = tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc(constant=1.5)], tt.bc_desc(dirichlet, [0.0] * 6, flux),
                              round_tol=1e-14)
    try:
        Fg = tt.tt_iga_densify_rhs(ctx, s, 0)
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    sp = [Space1D(k, p) for k in n]
    og = oracle_geometry(geo)
    Kst, F = assemble(sp, og, ConstantSource(1.5))
    for f, q in faces.items():
        F = F + neumann_load(sp, og, f, q)
    lo = [1 if dirichlet[2 * d] else 0 for d in range(3)]
    hi = [1 if dirichlet[2 * d + 1] else 0 for d in range(3)]
    _, Fi = restrict_bc(Kst, F, lo, hi)
    ref = to_flat(Fi)
    assert np.max(np.abs(Fg - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("inner,outer", [(("value", 1.0), ("flux", 0.5)), (("flux", -0.75), ("value", 2.0))])
def test_mixed_ring_matches_oracle(tt, ctx, inner, outer):
    """Value on one radial face, flux on the other (with the lift when the value is nonzero):
    GPU values and L2 error equal the oracle's for the same discrete problem."""
    from oracle.iga import Space1D, evaluate, l2_error, solve_bc
    from oracle.manufactured import RingMixed
    n, p = 8, 2
    dirichlet, value, flux = _ring_bc(inner, outer)
    geo = synthetic.QUARTER_CYLINDER
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=5))
    s = tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc(ring_log=True)], tt.bc_desc(dirichlet, value, flux),
                              round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13))
    try:
        assert st["converged"]
        x = np.linspace(0.0, 1.0, 6)
        pts = np.array([[a, b, c] for c in x[::2] for b in x[1::2] for a in x])
        uh = _eval(tt, ctx, u, pts)
        l2 = tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc(ring_log=True))
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    og = oracle_geometry(geo)
    sp = [Space1D(n, p)] * 3
    uo, _ = solve_bc(sp, og, None, dirichlet, value, tol=1e-14, flux=flux)
    ref = evaluate(sp, uo, x, x[1::2], x[::2])
    ref = np.array([ref[i, j, k] for k in range(3) for j in range(3) for i in range(6)])
    assert np.max(np.abs(uh - ref)) < 1e-10 * np.max(np.abs(ref))
    lo = l2_error(sp, og, uo, RingMixed(1.0, 2.0, inner, outer))
    assert abs(l2 - lo) <= 1e-6 * lo


def test_mixed_ring_converges_at_rate_p_plus_one(tt, ctx):
    p, errs, ns = 3, [], [16, 32, 64]
    dirichlet, value, flux = _ring_bc(("value", 1.0), ("flux", 0.5))
    for n in ns:
        g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, p, n, cross_tol=1e-14, seed=5))
        s = tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc(ring_log=True)], tt.bc_desc(dirichlet, value, flux),
                                  round_tol=1e-14)
        u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-12))
        try:
            assert st["converged"]
            errs.append(tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc(ring_log=True)))
        finally:
            tt.tt_iga_solution_destroy(u)
            tt.tt_iga_system_destroy(s)
            tt.tt_iga_geom_destroy(g)
    rate = math.log(errs[0] / errs[-1]) / math.log((ns[-1] - p) / (ns[0] - p))
    assert rate > p + 0.5 and errs[-1] < 1e-8, (errs, rate)


def test_cylinder_patch_flux_equals_the_annulus(tt, ctx):
    """The face area density of the NURBS cylinder net equals the analytic annulus': same loads."""
    n, p = 7, 2
    bc = tt.bc_desc([1, 0, 0, 0, 0, 0], [0.0] * 6, [0.0, 0.8, -0.3, 0.0, 0.0, 0.6])
    rhs = [tt.rhs_desc(constant=1.0)]
    ga = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, p, n, cross_tol=1e-14, seed=3))
    gn = tt.tt_iga_geometry_nurbs(ctx, tt.geom_desc({"kind": "nurbs"}, p, n, cross_tol=1e-14, seed=3),
                                  *synthetic.quarter_cylinder_net())
    sa = tt.tt_iga_assemble_bc(ctx, ga, rhs, bc, round_tol=1e-14)
    sn = tt.tt_iga_assemble_bc(ctx, gn, rhs, bc, round_tol=1e-14)
    try:
        Fa = tt.tt_iga_densify_rhs(ctx, sa, 0)
        Fn = tt.tt_iga_densify_rhs(ctx, sn, 0)
    finally:
        for s in (sa, sn):
            tt.tt_iga_system_destroy(s)
        for g in (ga, gn):
            tt.tt_iga_geom_destroy(g)
    assert np.max(np.abs(Fa - Fn)) < 1e-12 * np.max(np.abs(Fa))


@pytest.mark.parametrize("dirichlet,flux", [
    ([1, 0, 0, 0, 0, 0], [0.5, 0, 0, 0, 0, 0]),             # flux on the Dirichlet face
    ([1, 0, 0, 0, 0, 0], [0, float("inf"), 0, 0, 0, 0]),    # non-finite flux
])
def test_rejected_flux_data(tt, ctx, dirichlet, flux):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, 2, 6, seed=1))
    try:
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc()], tt.bc_desc(dirichlet, [0.0] * 6, flux))
        assert e.value.code == tt.ERR_ARG
    finally:
        tt.tt_iga_geom_destroy(g)


def test_ring_error_rejects_flux_on_an_angular_face(tt, ctx):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, 2, 6, cross_tol=1e-12, seed=1))
    s = tt.tt_iga_assemble_bc(ctx, g, [tt.rhs_desc(ring_log=True)],
                              tt.bc_desc([1, 0, 0, 0, 0, 0], [1.0] + [0.0] * 5, [0, 0.5, 0.2, 0, 0, 0]))
    u, _ = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-10))
    try:
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc(ring_log=True))
        assert e.value.code == tt.ERR_ARG
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
