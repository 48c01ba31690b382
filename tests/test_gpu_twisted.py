"""The non-separable twisted and swollen annulus at p = 3 (the benchmark's geometry) against the oracle,
mixed precision against FP64, and the relative L2 difference call.

* n = 24 and 32: the AMEn solution (FP64 and mixed precision) against the oracle's full-grid FP64 solve,
  compared entry by entry on the coefficient vector (<= 1e-9 FP64, <= 1e-7 mixed, relative).
* n = 128 and 512 (the benchmark size): the mixed solution against the FP64 TT solution of the same
  system, both at relative residual 1e-8, by the relative L2 difference over the mapped domain
  (tt_iga_l2_diff) <= 1e-7.
* tt_iga_l2_diff itself against a plain quadrature written out here with the oracle's basis and
  geometry (both solutions expanded on the tensor Gauss grid, weights times det J).
"""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding, oracle_geometry

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


_ORACLE = {}


def _oracle(n, p):
    """Restricted oracle solution (flat, i1 fastest), computed once per size."""
    if (n, p) not in _ORACLE:
        from oracle.iga import Space1D, solve, to_flat
        from oracle.manufactured import Manufactured
        og = oracle_geometry(GEO)
        u, _ = solve([Space1D(n, p)] * 3, og, Manufactured(og), tol=1e-14)
        _ORACLE[(n, p)] = to_flat(u[1:-1, 1:-1, 1:-1])
    return _ORACLE[(n, p)]


def _solve(tt, ctx, n, p, precision, tol, cross_tol, round_tol, seed=0):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(GEO, p, n, cross_tol=cross_tol, seed=seed))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=round_tol)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=tol, precision=precision))
    return g, s, u, st


def _release(tt, g, s, u):
    tt.tt_iga_solution_destroy(u)
    tt.tt_iga_system_destroy(s)
    tt.tt_iga_geom_destroy(g)


@pytest.mark.parametrize("n", [24, 32])
@pytest.mark.parametrize("precision,tol,bound", [("FP64", 1e-13, 1e-9), ("MIXED_FP32", 1e-10, 1e-7),
                                                 ("MIXED_TF32", 1e-10, 1e-7)])
def test_twisted_p3_matches_oracle(tt, ctx, n, precision, tol, bound):
    p = 3
    g, s, u, st = _solve(tt, ctx, n, p, getattr(tt, precision), tol, 1e-14, 1e-14, seed=4)
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
        res = tt.tt_iga_residual(ctx, s, u, 0)
    finally:
        _release(tt, g, s, u)
    ref = _oracle(n, p)
    assert res <= tol, st
    if precision == "MIXED_TF32":
        assert st["local_matvecs_tensor"] > 0, st
    assert np.linalg.norm(uh - ref) <= bound * np.linalg.norm(ref), (st, np.linalg.norm(uh - ref) / np.linalg.norm(ref))


def _l2_by_quadrature(tt, ctx, g, u, v, s, n, p):
    """sqrt(int (u_h - v_h)^2 / int v_h^2) with the p+1 point Gauss rule, by the oracle's basis and map."""
    from oracle.iga import Space1D, evaluate, from_flat
    m = tt.tt_iga_system_info(s)["modes"]
    full = []
    for h in (u, v):
        c = from_flat(tt.tt_iga_densify_solution(ctx, h, m), m)
        cf = np.zeros((n, n, n))
        cf[1:-1, 1:-1, 1:-1] = c
        full.append(cf)
    sp = [Space1D(n, p)] * 3
    og = oracle_geometry(GEO)
    x = sp[0].flat_points()
    w = sp[0].flat_weights()
    num = den = 0.0
    for k in range(len(x)):
        _, J = og.map(x, x, x[k:k + 1])
        det = np.linalg.det(J)
        uh = evaluate(sp, full[0], x, x, x[k:k + 1])
        vh = evaluate(sp, full[1], x, x, x[k:k + 1])
        wk = w[:, None, None] * w[None, :, None] * w[k] * det
        num += np.sum(wk * (uh - vh) ** 2)
        den += np.sum(wk * vh ** 2)
    return float(np.sqrt(num / den))


def test_l2_diff_matches_quadrature(tt, ctx):
    """Two solutions of the same system that differ visibly (tolerance 1e-3 against 1e-13)."""
    n, p = 10, 3
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(GEO, p, n, cross_tol=1e-14, seed=2))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-14)
    u, _ = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-3, kickrank=-1, max_sweeps=1), allow_not_converged=True)
    v, _ = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13))
    try:
        got = tt.tt_iga_l2_diff(ctx, g, u, v)
        ref = _l2_by_quadrature(tt, ctx, g, u, v, s, n, p)
        same = tt.tt_iga_l2_diff(ctx, g, v, v)
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_solution_destroy(v)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    assert ref > 1e-6  # the two solutions do differ
    assert abs(got - ref) <= 1e-6 * ref, (got, ref)
    assert same <= 1e-14  # a TT minus itself rounds to roundoff, not to an exact zero


@pytest.mark.parametrize("n", [128, 512])
@pytest.mark.parametrize("precision", ["MIXED_FP32", "MIXED_TF32"])
def test_mixed_matches_fp64_tt_at_scale(tt, ctx, n, precision):
    """Benchmark tolerances (cross and rounding 1e-10, residual 1e-8): mixed within 1e-7 of FP64."""
    p = 3
    g, s, u64, st64 = _solve(tt, ctx, n, p, tt.FP64, 1e-8, 1e-10, 1e-10)
    um, stm = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-8, precision=getattr(tt, precision)))
    try:
        d = tt.tt_iga_l2_diff(ctx, g, um, u64)
        rm = tt.tt_iga_residual(ctx, s, um, 0)
    finally:
        tt.tt_iga_solution_destroy(um)
        _release(tt, g, s, u64)
    assert st64["rel_residual"] <= 1e-8 and rm <= 1e-8, (st64, stm)
    assert stm["local_matvecs"] > stm["local_matvecs_fp64"]
    if precision == "MIXED_TF32":
        assert stm["local_matvecs_tensor"] > 0, stm
    assert d <= 1e-7, (d, st64, stm)


def test_inexact_local_solves(tt, ctx):
    """local_rtol: early local systems solved to a fraction of their initial residual.  The exact
    global residual still decides convergence: at n = 24 the result matches the oracle like the
    exact-local-solve path, at n = 512 it is within 1e-7 of the exact-local-solve FP64 solution."""
    p = 3
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(GEO, p, 24, cross_tol=1e-14, seed=4))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13, local_rtol=1e-3))
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
        assert st["converged"] and tt.tt_iga_residual(ctx, s, u, 0) <= 1e-13
    finally:
        _release(tt, g, s, u)
    ref = _oracle(24, p)
    assert np.linalg.norm(uh - ref) <= 1e-9 * np.linalg.norm(ref)
    g, s, u64, st64 = _solve(tt, ctx, 512, p, tt.FP64, 1e-8, 1e-10, 1e-10)
    try:
        for prec in (tt.FP64, tt.MIXED_FP32):
            ui, sti = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-8, precision=prec, local_rtol=1e-3))
            try:
                assert sti["converged"] and tt.tt_iga_residual(ctx, s, ui, 0) <= 1e-8, sti
                assert sti["local_matvecs"] < st64["local_matvecs"] or prec != tt.FP64, (sti, st64)
                assert tt.tt_iga_l2_diff(ctx, g, ui, u64) <= 1e-7
            finally:
                tt.tt_iga_solution_destroy(ui)
    finally:
        _release(tt, g, s, u64)
