"""Degenerate and edge cases of the GPU path: the smallest meshes, p = 1, unequal mode sizes, the box
geometry, argument errors and size limits."""
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


def _oracle(geo, n, p, modes=()):
    from oracle.iga import Space1D, solve, to_flat
    from oracle.manufactured import Manufactured
    og = oracle_geometry(geo)
    ns = [n] * 3 if isinstance(n, int) else list(n)
    sp = [Space1D(ns[d], p) for d in range(3)]
    u, _ = solve(sp, og, Manufactured(og, list(modes)), tol=1e-14)
    return to_flat(u[1:-1, 1:-1, 1:-1])


@pytest.mark.parametrize("geo,n,p", [
    (synthetic.QUARTER_CYLINDER, 3, 1),            # one unknown
    (synthetic.TWISTED_ANNULUS, 4, 2),             # one unknown per direction
    (synthetic.TWISTED_ANNULUS, 9, 1),             # linear elements
    ({"kind": "box", "lx": 1.0, "ly": 2.0, "lz": 0.5}, 10, 2),
    (synthetic.TWISTED_ANNULUS, (8, 11, 13), 2),   # unequal mode sizes
])
def test_small_and_degenerate_meshes_match_oracle(tt, ctx, geo, n, p):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=2))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13))
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    ref = _oracle(geo, n, p)
    assert np.linalg.norm(uh - ref) <= 1e-9 * np.linalg.norm(ref), st


def test_argument_errors(tt, ctx):
    bad = [tt.geom_desc(synthetic.QUARTER_CYLINDER, 3, 4),                       # n < p + 2
           tt.geom_desc({**synthetic.QUARTER_CYLINDER, "r_out": 0.5}, 2, 8),     # r_out < r_in
           tt.geom_desc({**synthetic.QUARTER_CYLINDER, "swell": 1.5}, 2, 8),     # swell folds the map
           tt.geom_desc(synthetic.QUARTER_CYLINDER, 8, 16)]                      # p > 7
    for d in bad:
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_geometry(ctx, d)
        assert e.value.code == tt.ERR_ARG
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, 2, 8, cross_tol=1e-12))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-12)
    try:
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_solve(ctx, s, tt.solve_opts(precision=7))  # not a precision mode
        assert e.value.code == tt.ERR_ARG
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_solve(ctx, s, tt.solve_opts(rhs_index=3))
        assert e.value.code == tt.ERR_ARG
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_operator_entries(ctx, s, [(0, 0, 6)], [(0, 0, 0)])  # index beyond n - 2
        assert e.value.code == tt.ERR_ARG
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)


def test_size_limits(tt, ctx):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, 2, 20, cross_tol=1e-12))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc()], round_tol=1e-12)
    try:
        with pytest.raises(tt.TTIgaError) as e:   # 18^3 unknowns > 4096: no dense operator
            tt.tt_iga_densify_operator(ctx, s)
        assert e.value.code == tt.ERR_TOO_LARGE
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)


def test_multiple_right_hand_sides(tt, ctx):
    """One system, several load vectors: each solve matches the oracle for its own source."""
    geo, n, p = synthetic.TWISTED_ANNULUS, 8, 2
    modes = [[], [(0.2, (1.0, 0.5, -1.0), 0.3)], [(-0.25, (0.0, 2.0, 1.0), 1.1), (0.1, (1.0, 1.0, 1.0), 0.0)]]
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=5))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc(m) for m in modes], round_tol=1e-14)
    try:
        info = tt.tt_iga_system_info(s)
        assert info["n_rhs"] == 3
        for k, m in enumerate(modes):
            u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-13, rhs_index=k))
            uh = tt.tt_iga_densify_solution(ctx, u, info["modes"])
            tt.tt_iga_solution_destroy(u)
            ref = _oracle(geo, n, p, m)
            assert np.linalg.norm(uh - ref) <= 1e-9 * np.linalg.norm(ref), (k, st)
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
