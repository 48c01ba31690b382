"""Generic single-patch NURBS input (Section 2.2): the quarter cylinder written as a NURBS patch
reproduces the analytic annulus path, and a curved patch matches the oracle's full-grid solve."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding

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


def _cylinder_net():
    from oracle.geometry import quarter_cylinder_patch
    q = quarter_cylinder_patch(1.0, 2.0, 1.0)
    return q.deg, q.knots, q.ctrl, q.w


@pytest.mark.parametrize("n,p", [(6, 2), (7, 3)])
def test_cylinder_patch_equals_the_annulus(tt, ctx, n, p):
    rhs = [tt.rhs_desc(constant=1.0)]
    ga = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, p, n, cross_tol=1e-14, seed=3))
    gn = tt.tt_iga_geometry_nurbs(ctx, tt.geom_desc({"kind": "nurbs"}, p, n, cross_tol=1e-14, seed=3), *_cylinder_net())
    sa = tt.tt_iga_assemble(ctx, ga, rhs, round_tol=1e-14)
    sn = tt.tt_iga_assemble(ctx, gn, rhs, round_tol=1e-14)
    try:
        ra, _ = tt.tt_iga_geom_ranks(ga)
        rn, _ = tt.tt_iga_geom_ranks(gn)
        Ka = tt.tt_iga_densify_operator(ctx, sa)
        Kn = tt.tt_iga_densify_operator(ctx, sn)
        Fa = tt.tt_iga_densify_rhs(ctx, sa, 0)
        Fn = tt.tt_iga_densify_rhs(ctx, sn, 0)
    finally:
        for s in (sa, sn):
            tt.tt_iga_system_destroy(s)
        for g in (ga, gn):
            tt.tt_iga_geom_destroy(g)
    assert ra == rn
    assert np.max(np.abs(Ka - Kn)) < 1e-12 * np.max(np.abs(Ka))
    assert np.max(np.abs(Fa - Fn)) < 1e-12 * np.max(np.abs(Fa))


def test_curved_patch_matches_oracle(tt, ctx):
    from oracle.geometry import NURBSPatch
    from oracle.iga import Space1D, solve, to_flat
    from oracle.manufactured import ConstantSource
    n, p = 7, 2
    net = synthetic.curved_patch(seed=2)
    g = tt.tt_iga_geometry_nurbs(ctx, tt.geom_desc({"kind": "nurbs"}, p, n, cross_tol=1e-14, seed=9), *net)
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc(constant=1.0)], round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13))
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
        assert st["converged"]
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    sp = [Space1D(n, p)] * 3
    uo, _ = solve(sp, NURBSPatch(*net), ConstantSource(1.0), tol=1e-14)
    ref = to_flat(uo[1:-1, 1:-1, 1:-1])
    assert np.max(np.abs(uh - ref)) < 1e-9 * np.max(np.abs(ref))


def _bad(net, what):
    deg, kn, ctrl, w = net
    kn = [np.array(k, dtype=float) for k in kn]
    ctrl, w, deg = ctrl.copy(), w.copy(), list(deg)
    if what == "knots":
        kn[0][1] = 0.3          # not open at the start
    elif what == "order":
        kn[1][3] = 0.9          # interior knots out of order
        kn[1][4] = 0.2
    elif what == "weight":
        w[1, 1, 1] = -0.5
    elif what == "degree":
        deg[2] = 5
    return deg, kn, ctrl, w


@pytest.mark.parametrize("what", ["knots", "order", "weight", "degree"])
def test_malformed_patches_are_rejected(tt, ctx, what):
    with pytest.raises(tt.TTIgaError) as e:
        tt.tt_iga_geometry_nurbs(ctx, tt.geom_desc({"kind": "nurbs"}, 2, 6, seed=1),
                                 *_bad(synthetic.curved_patch(), what))
    assert e.value.code == tt.ERR_ARG


def test_patch_takes_constant_right_hand_sides_only(tt, ctx):
    g = tt.tt_iga_geometry_nurbs(ctx, tt.geom_desc({"kind": "nurbs"}, 2, 6, cross_tol=1e-12, seed=1),
                                 *synthetic.curved_patch())
    try:
        for rhs in (tt.rhs_desc(), tt.rhs_desc(ring_log=True)):
            with pytest.raises(tt.TTIgaError) as e:
                tt.tt_iga_assemble(ctx, g, [rhs])
            assert e.value.code == tt.ERR_ARG
    finally:
        tt.tt_iga_geom_destroy(g)
