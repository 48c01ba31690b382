"""Parity of the AMEn TT solve against the oracle's full-grid PCG solution (FP64 and mixed precision),
plus evaluation and the L2 error."""
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


def _oracle_solution(geo, n, p, modes):
    from oracle.iga import Space1D, solve
    from oracle.manufactured import Manufactured
    og = oracle_geometry(geo)
    sp = [Space1D(n, p)] * 3
    u, info = solve(sp, og, Manufactured(og, modes), tol=1e-14)
    return u, sp, og


def _tt_solve(tt, ctx, geo, n, p, modes, precision, tol):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=4))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc(modes)], round_tol=1e-14)
    u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=tol, precision=precision))
    return g, s, u, st


@pytest.mark.parametrize("geo,n,p,modes", [
    (synthetic.QUARTER_CYLINDER, 8, 2, []),
    (synthetic.TWISTED_ANNULUS, 10, 2, []),
    (synthetic.TWISTED_ANNULUS, 9, 3, [(0.2, (1.0, 1.0, 0.0), 0.7)]),
    (synthetic.QUARTER_CYLINDER, 16, 2, []),
    # degrees 4 and 5: the band block-Jacobi systems (interface blocks above 8) run the
    # warp-scan triangular solves with bandwidths 4 and 5
    (synthetic.TWISTED_ANNULUS, 12, 4, [(0.2, (1.0, 1.0, 0.0), 0.7)]),
    (synthetic.TWISTED_ANNULUS, 11, 5, [(0.2, (1.0, 1.0, 0.0), 0.7)]),
])
def test_fp64_solution_matches_oracle(tt, ctx, geo, n, p, modes):
    from oracle.iga import to_flat
    g, s, u, st = _tt_solve(tt, ctx, geo, n, p, modes, tt.FP64, 1e-13)
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
        res = tt.tt_iga_residual(ctx, s, u, 0)
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    uo, _, _ = _oracle_solution(geo, n, p, modes)
    ref = to_flat(uo[1:-1, 1:-1, 1:-1])
    assert res <= 1e-13
    assert np.linalg.norm(uh - ref) <= 1e-9 * np.linalg.norm(ref), st


@pytest.mark.parametrize("precision", ["MIXED_FP32", "MIXED_TF32"])
def test_mixed_precision_matches_oracle(tt, ctx, precision):
    from oracle.iga import to_flat
    geo, n, p = synthetic.TWISTED_ANNULUS, 12, 3
    g, s, u, st = _tt_solve(tt, ctx, geo, n, p, [], getattr(tt, precision), 1e-10)
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    uo, _, _ = _oracle_solution(geo, n, p, [])
    ref = to_flat(uo[1:-1, 1:-1, 1:-1])
    assert st["rel_residual"] <= 1e-10
    assert st["local_matvecs"] > st["local_matvecs_fp64"]
    if precision == "MIXED_TF32":
        assert st["local_matvecs_tensor"] > 0  # the tensor-core stages ran
    else:
        assert st["local_matvecs_tensor"] == 0
    assert np.linalg.norm(uh - ref) <= 1e-7 * np.linalg.norm(ref)


def test_eval_and_l2_error_match_oracle(tt, ctx):
    import torch
    from oracle.iga import evaluate, l2_error
    from oracle.manufactured import Manufactured
    geo, n, p = synthetic.TWISTED_ANNULUS, 10, 2
    g, s, u, st = _tt_solve(tt, ctx, geo, n, p, [], tt.FP64, 1e-13)
    try:
        xi = synthetic.random_points(300, seed=9)
        xi[:4] = [[0, 0, 0], [1, 1, 1], [0.5, 1.0, 0.0], [1e-12, 0.3, 1 - 1e-12]]
        xt = torch.as_tensor(xi, device="cuda")
        out = torch.empty(len(xi), dtype=torch.float64, device="cuda")
        tt.tt_iga_eval(ctx, u, xt, out)
        got = out.cpu().numpy()
        l2 = tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc())
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    uo, sp, og = _oracle_solution(geo, n, p, [])
    ref = np.array([evaluate(sp, uo, [a], [b], [c])[0, 0, 0] for a, b, c in xi])
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    l2o = l2_error(sp, og, uo, Manufactured(og))
    assert abs(l2 - l2o) <= 1e-6 * l2o


def test_cylinder_p3_n32_matches_oracle(tt, ctx):
    """The refinement sweep's direct-comparison size (n = 32, p = 3)."""
    from oracle.iga import to_flat
    geo, n, p = synthetic.QUARTER_CYLINDER, 32, 3
    g, s, u, st = _tt_solve(tt, ctx, geo, n, p, [], tt.FP64, 1e-12)
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        uh = tt.tt_iga_densify_solution(ctx, u, m)
    finally:
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    uo, _, _ = _oracle_solution(geo, n, p, [])
    ref = to_flat(uo[1:-1, 1:-1, 1:-1])
    assert np.linalg.norm(uh - ref) <= 1e-9 * np.linalg.norm(ref), st
