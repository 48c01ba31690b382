"""End-to-end parity of the TT assembly (TT-cross + contraction + rounding + Dirichlet restriction)
against the oracle's element-loop assembly: densified operator and load vector on tiny meshes."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding, oracle_geometry

pytestmark = pytest.mark.gpu

BOX = {"kind": "box", "lx": 1.0, "ly": 2.0, "lz": 0.5}


@pytest.fixture(scope="module")
def tt():
    return load_binding()


@pytest.fixture(scope="module")
def ctx(tt):
    import torch
    c = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    yield c
    tt.tt_iga_ctx_destroy(c)


CASES = [
    (BOX, 6, 2, []),
    (synthetic.QUARTER_CYLINDER, 6, 2, []),
    (synthetic.QUARTER_CYLINDER, 7, 3, [(0.25, (1.0, 0.0, -1.0), 0.5)]),
    (synthetic.TWISTED_ANNULUS, 6, 2, []),
    (synthetic.TWISTED_ANNULUS, 8, 3, [(-0.2, (0.3, 2.0, 1.0), 0.1)]),
    (synthetic.TWISTED_ANNULUS, 13, 2, []),
]


@pytest.mark.parametrize("geo,n,p,modes", CASES)
def test_operator_and_load_match_oracle(tt, ctx, geo, n, p, modes):
    from oracle.iga import Space1D, assemble, restrict, stencil_to_dense, to_flat
    from oracle.manufactured import Manufactured
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=7))
    s = tt.tt_iga_assemble(ctx, g, [tt.rhs_desc(modes)], round_tol=1e-14)
    try:
        K = tt.tt_iga_densify_operator(ctx, s)
        F = tt.tt_iga_densify_rhs(ctx, s, 0)
    finally:
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    og = oracle_geometry(geo)
    sp = [Space1D(n, p)] * 3
    Kst, Fo = assemble(sp, og, Manufactured(og, modes))
    Ki, Fi = restrict(Kst, Fo)
    ref = stencil_to_dense(Ki, (p, p, p))
    assert np.max(np.abs(K - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(F - to_flat(Fi))) <= 1e-12 * np.max(np.abs(Fi))
    assert np.max(np.abs(K - K.T)) <= 1e-12 * np.max(np.abs(ref))


def test_cylinder_coefficient_ranks_are_exact(tt, ctx):
    """Untwisted cylinder: R11, R22, R33 separable (rank 1), R12, R13, R23 vanish (rank 0)."""
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.QUARTER_CYLINDER, 3, 40, cross_tol=1e-12, seed=1))
    try:
        ranks, err = tt.tt_iga_geom_ranks(g)
    finally:
        tt.tt_iga_geom_destroy(g)
    assert ranks[0] == (1, 1) and ranks[3] == (1, 1) and ranks[5] == (1, 1)
    assert ranks[1] == (0, 0) and ranks[2] == (0, 0) and ranks[4] == (0, 0)
    assert max(err) < 1e-12


def test_twisted_cross_validates(tt, ctx):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(synthetic.TWISTED_ANNULUS, 3, 64, cross_tol=1e-10, seed=2))
    try:
        ranks, err = tt.tt_iga_geom_ranks(g)
    finally:
        tt.tt_iga_geom_destroy(g)
    assert all(r[0] >= 1 for r in ranks)
    assert max(err) <= 1e-9
