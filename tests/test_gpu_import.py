"""Export and import of solution cores (checkpoint and resume), warm-started solves, and the exact
residual of solutions whose residual TT rank is beyond the TT norm's limit.

* A solution exported with tt_iga_solution_cores and rebuilt with tt_iga_import_cores has the same
  coefficients and the same point values.
* tt_iga_solve_from started at an imported converged solution stops after one sweep; started at a
  loose solution it reaches the tight tolerance.
* On a curved NURBS patch (operator TT ranks in the tens) the residual F - K u has TT rank above 256;
  tt_iga_residual then expands F and K u on the device.  At 16^3 unknowns the dense operator fits on
  the host, so the value is checked against numpy's F - K u.
"""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding

pytestmark = pytest.mark.gpu

GEO = synthetic.TWISTED_ANNULUS


@pytest.fixture(scope="module")
def tt():
    return load_binding()


@pytest.fixture(scope="module")
def ctx(tt):
    import torch
    c = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    yield c
    tt.tt_iga_ctx_destroy(c)


@pytest.fixture(scope="module")
def system(tt, ctx):
    n, p = 14, 3
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(GEO, p, n, cross_tol=1e-13, seed=6))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc([(0.2, (1.0, 0.5, 0.0), 0.3)])], round_tol=1e-13)
    yield g, s
    tt.tt_iga_system_destroy(s)
    tt.tt_iga_geom_destroy(g)


def test_export_import_roundtrip(tt, ctx, system):
    import torch
    g, s = system
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-11))
    cores = [c.copy() for c in tt.tt_iga_solution_cores(ctx, u)]
    v = tt.tt_iga_import_cores(ctx, s, cores)
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        assert tt.tt_iga_solution_ranks(v) == tuple(st["ranks"])
        du = tt.tt_iga_densify_solution(ctx, u, m)
        dv = tt.tt_iga_densify_solution(ctx, v, m)
        assert np.array_equal(du, dv)
        xi = torch.as_tensor(synthetic.random_points(500, seed=12), device="cuda")
        a = torch.empty(500, dtype=torch.float64, device="cuda")
        b = torch.empty(500, dtype=torch.float64, device="cuda")
        tt.tt_iga_eval(ctx, u, xi, a)
        tt.tt_iga_eval(ctx, v, xi, b)
        assert torch.equal(a, b)
        assert tt.tt_iga_residual(ctx, s, v, 0) == tt.tt_iga_residual(ctx, s, u, 0)
        again = [c.copy() for c in tt.tt_iga_solution_cores(ctx, v)]
        assert all(np.array_equal(x, y) for x, y in zip(cores, again))
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_solution_destroy(v)


def test_import_rejects_mismatched_cores(tt, ctx, system):
    g, s = system
    m = tt.tt_iga_system_info(s)["modes"]
    good = [np.ones((1, m[0], 2)), np.ones((2, m[1], 2)), np.ones((2, m[2], 1))]
    for bad in ([np.ones((1, m[0] + 1, 2))] + good[1:],          # wrong mode size
                good[:2] + [np.full((2, m[2], 1), np.nan)]):     # non-finite entry
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_import_cores(ctx, s, bad)
        assert e.value.code == tt.ERR_ARG


def test_warm_start_from_imported_cores(tt, ctx, system):
    g, s = system
    tight = tt.solve_opts(tol=1e-11)
    u, st = tt.tt_iga_solve(ctx, s, tight)
    v = tt.tt_iga_import_cores(ctx, s, [c.copy() for c in tt.tt_iga_solution_cores(ctx, u)])
    w, stw = tt.tt_iga_solve_from(ctx, s, tight, v)
    loose, stl = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-4))
    x, stx = tt.tt_iga_solve_from(ctx, s, tight, loose)
    try:
        # resumed at the converged iterate: one sweep, then the exact residual confirms it
        assert stw["converged"] and stw["sweeps"] <= 1 and stw["rel_residual"] <= 1e-11, stw
        # resumed from a loose iterate: reaches the tight tolerance
        assert stx["converged"] and stx["rel_residual"] <= 1e-11, stx
        m = tt.tt_iga_system_info(s)["modes"]
        ref = tt.tt_iga_densify_solution(ctx, u, m)
        for h in (w, x):
            d = tt.tt_iga_densify_solution(ctx, h, m)
            assert np.linalg.norm(d - ref) <= 1e-8 * np.linalg.norm(ref)
    finally:
        for h in (u, v, w, loose, x):
            tt.tt_iga_solution_destroy(h)


def test_dense_residual_beyond_tt_rank_limit(tt, ctx):
    n, p = 18, 3
    net = synthetic.curved_patch(seed=2)
    g = tt.tt_iga_geometry_nurbs(ctx, tt.geom_desc({"kind": "nurbs"}, p, n, cross_tol=1e-8, seed=1), *net,
                                 allow_not_converged=True)
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc(constant=1.0)], round_tol=1e-8)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-6), allow_not_converged=True)
    try:
        info = tt.tt_iga_system_info(s)
        r1, r2 = tt.tt_iga_solution_ranks(u)
        fr = info["rhs_ranks"][0]
        assert info["op_ranks"][0] * r1 + fr[0] > 256 or info["op_ranks"][1] * r2 + fr[1] > 256
        got = tt.tt_iga_residual(ctx, s, u, 0)
        K = tt.tt_iga_densify_operator(ctx, s)
        F = tt.tt_iga_densify_rhs(ctx, s, 0)
        x = tt.tt_iga_densify_solution(ctx, u, info["modes"])
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    ref = np.linalg.norm(F - K @ x) / np.linalg.norm(F)
    assert got > 0.0 and abs(got - ref) <= 1e-6 * ref + 1e-14, (got, ref)
