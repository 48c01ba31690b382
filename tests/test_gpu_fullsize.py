"""Parity at the benchmark sizes, on outputs the oracle can compute one by one: sampled operator rows and
load entries (oracle: element quadrature over each row's support), sampled residual rows of the TT solution
(oracle rows of K and entries of F applied to the GPU solution), and the L2 convergence rate h^(p+1)."""
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


def _sample_rows(m, count, seed):
    g = synthetic.rng(seed)
    rows = [tuple(int(v) for v in g.integers(0, m, 3)) for _ in range(count)]
    rows += [(0, 0, 0), (m - 1, m - 1, m - 1), (0, m // 2, m - 1)]
    return rows


def _band_pairs(row, p, m):
    """All restricted column multi-indices coupled to `row` (|i_d - j_d| <= p)."""
    cols = []
    for o1 in range(-p, p + 1):
        for o2 in range(-p, p + 1):
            for o3 in range(-p, p + 1):
                c = (row[0] + o1, row[1] + o2, row[2] + o3)
                if all(0 <= v < m for v in c):
                    cols.append(c)
    return cols


def _check_rows(tt, ctx, s, geo, n, p, rows, modes, rel_tol):
    from oracle.iga import Space1D, load_entries, stiffness_rows
    from oracle.manufactured import Manufactured
    og = oracle_geometry(geo)
    sp = [Space1D(n, p)] * 3
    m = n - 2
    full = [(r[0] + 1, r[1] + 1, r[2] + 1) for r in rows]  # restricted -> full basis index
    blocks = stiffness_rows(sp, og, full)
    kmax = 0.0
    worst = 0.0
    for r, blk in zip(rows, blocks):
        cols = _band_pairs(r, p, m)
        got = tt.tt_iga_operator_entries(ctx, s, [r] * len(cols), cols)
        ref = np.array([blk[c[0] - r[0] + p, c[1] - r[1] + p, c[2] - r[2] + p] for c in cols])
        kmax = max(kmax, np.max(np.abs(ref)))
        worst = max(worst, np.max(np.abs(got - ref)))
    assert worst <= rel_tol * kmax, (worst, kmax)
    fo = load_entries(sp, og, Manufactured(og, modes), full)
    fg = tt.tt_iga_vector_entries(ctx, s, None, 0, rows)
    assert np.max(np.abs(fg - fo)) <= rel_tol * np.max(np.abs(fo)) + 1e-300


def test_cylinder_p3_n128_sampled_operator_and_load(tt, ctx):
    """Exact TT ranks (separable geometry): sampled entries agree to roundoff."""
    geo, n, p = synthetic.QUARTER_CYLINDER, 128, 3
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-12, seed=0))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-12)
    try:
        _check_rows(tt, ctx, s, geo, n, p, _sample_rows(n - 2, 12, 1), [], 1e-11)
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)


def test_twisted_p3_n512_sampled_operator_and_load(tt, ctx):
    """Cross and rounding at 1e-10 (Frobenius-relative); an entry can carry up to eps ||K||_F, which
    for this mesh is about 1e5 max|K|, so entries are checked to 1e-10 * 1e5 relative to max|K|."""
    geo, n, p = synthetic.TWISTED_ANNULUS, 512, 3
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-10, seed=0))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-10)
    try:
        _check_rows(tt, ctx, s, geo, n, p, _sample_rows(n - 2, 6, 2), [], 1e-5)
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)


@pytest.mark.parametrize("precision", ["FP64", "MIXED_FP32"])
def test_cylinder_p3_n128_solution_residual_rows(tt, ctx, precision):
    """Exact TT residual <= 1e-8 and oracle-computed residual rows F_a - sum_b K_ab u_b small."""
    from oracle.iga import Space1D, load_entries, stiffness_rows
    from oracle.manufactured import Manufactured
    geo, n, p = synthetic.QUARTER_CYLINDER, 128, 3
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-12, seed=0))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-12)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-8, precision=getattr(tt, precision)))
    try:
        res = tt.tt_iga_residual(ctx, s, u, 0)
        assert res <= 1e-8, st
        m = n - 2
        F = tt.tt_iga_densify_rhs(ctx, s, 0)
        fnorm = np.linalg.norm(F)
        rows = _sample_rows(m, 8, 3)
        og = oracle_geometry(geo)
        sp = [Space1D(n, p)] * 3
        full = [(r[0] + 1, r[1] + 1, r[2] + 1) for r in rows]
        blocks = stiffness_rows(sp, og, full)
        fo = load_entries(sp, og, Manufactured(og), full)
        for r, blk, fa in zip(rows, blocks, fo):
            cols = _band_pairs(r, p, m)
            uv = tt.tt_iga_vector_entries(ctx, None, u, 0, cols)
            ku = sum(blk[c[0] - r[0] + p, c[1] - r[1] + p, c[2] - r[2] + p] * v for c, v in zip(cols, uv))
            assert abs(fa - ku) <= 1e-8 * fnorm
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)


def test_cylinder_p3_refinement_sweep_rate(tt, ctx):
    """L2 error slope ~ h^4 for p = 3 over n = 16, 32, 64, 128 (h = 1/(n-p))."""
    geo, p = synthetic.QUARTER_CYLINDER, 3
    errs, hs = [], []
    for n in (16, 32, 64, 128):
        g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-12, seed=0))
        s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-12)
        u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-10))
        errs.append(tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc()))
        hs.append(1.0 / (n - p))
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(hs[i] / hs[i + 1]) for i in range(3)]
    assert min(rates[1:]) >= 3.7, (errs, rates)
