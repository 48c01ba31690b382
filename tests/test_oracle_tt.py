"""Pins of oracle.tt: exact rank-1 outer products, TT-SVD bound, Kronecker layout, and the
Section 4.2 contraction against the element-loop assembly."""
import numpy as np
import pytest

from oracle.geometry import Annulus, Box, coefficient_tensor
from oracle.iga import Space1D, assemble, stencil_to_dense
from oracle.tt import load_core, selector, stiffness_core, tt_full, tt_svd, ttm_full
from oracle.manufactured import Manufactured


def test_outer_product_is_rank_one_tt():
    g = np.random.default_rng(0)
    a, b, c = g.standard_normal(5), g.standard_normal(6), g.standard_normal(7)
    X = np.einsum("i,j,k->ijk", a, b, c)
    cores = tt_svd(X, 1e-14)
    assert [G.shape[2] for G in cores[:-1]] == [1, 1]
    assert np.max(np.abs(tt_full(cores) - X)) < 1e-14 * np.max(np.abs(X))


def test_tt_svd_error_bound_and_exact_ranks():
    g = np.random.default_rng(1)
    cores = [g.standard_normal((1, 8, 3)), g.standard_normal((3, 9, 4)), g.standard_normal((4, 10, 1))]
    X = tt_full(cores)
    rc = tt_svd(X, 1e-13)
    assert [G.shape[2] for G in rc[:-1]] == [3, 4]
    Y = X + 1e-3 * g.standard_normal(X.shape)
    eps = 1e-2
    Z = tt_full(tt_svd(Y, eps))
    assert np.linalg.norm(Z - Y) <= eps * np.linalg.norm(Y) * (1 + 1e-12)


def test_ttm_full_is_kronecker_with_first_index_fastest():
    g = np.random.default_rng(2)
    A, B, C = g.standard_normal((3, 3)), g.standard_normal((4, 4)), g.standard_normal((2, 2))
    cores = [A[None, :, :, None], B[None, :, :, None], C[None, :, :, None]]
    assert np.allclose(ttm_full(cores), np.kron(C, np.kron(B, A)))


def test_selector_cases():
    assert selector(1, 1, 1) == ("D", "D")
    assert selector(1, 1, 2) == ("N", "N")
    assert selector(1, 2, 1) == ("D", "N")
    assert selector(1, 2, 2) == ("N", "D")
    assert selector(1, 2, 3) == ("N", "N")


def _tt_operator_dense(spaces, geom, eps=1e-14):
    """K = sum_ij K_ij^TT with R_ij compressed by TT-SVD on the Gauss grid (Section 4.2.1)."""
    pts = [s.flat_points() for s in spaces]
    wts = [s.flat_weights() for s in spaces]
    tabs = [s.full_tables() for s in spaces]
    _, J = geom.map(*pts)
    _, R = coefficient_tensor(J)
    K = 0.0
    for i in range(3):
        for j in range(3):
            field = R[..., i, j]
            if np.max(np.abs(field)) < 1e-14 * np.max(np.abs(R)):
                continue
            G = tt_svd(field, eps)
            M = []
            for d in range(3):
                te, tr = selector(i + 1, j + 1, d + 1)
                A = tabs[d][1] if te == "D" else tabs[d][0]
                B = tabs[d][1] if tr == "D" else tabs[d][0]
                M.append(stiffness_core(G[d], wts[d], A, B))
            K = K + ttm_full(M)
    return K


@pytest.mark.parametrize("geom", [Box(1.0, 2.0, 0.5), Annulus(), Annulus(1.0, 2.0, 1.0, 0.8, 0.2)])
def test_tt_contraction_reproduces_element_assembly(geom):
    sp = [Space1D(6, 2), Space1D(5, 2), Space1D(5, 3)]
    Kst, _ = assemble(sp, geom, None)
    ref = stencil_to_dense(Kst, (2, 2, 3))
    K = _tt_operator_dense(sp, geom)
    assert np.max(np.abs(K - ref)) < 1e-12 * np.max(np.abs(ref))


def test_load_core_reproduces_element_assembly():
    from oracle.tt import tt_svd as svd
    sp = [Space1D(6, 2), Space1D(5, 2), Space1D(5, 3)]
    g = Annulus(1.0, 2.0, 1.0, 0.8, 0.2)
    m = Manufactured(g)
    _, F = assemble(sp, g, m)
    pts = [s.flat_points() for s in sp]
    X, J = g.map(*pts)
    detJ, _ = coefficient_tensor(J)
    G = svd(m.f(X) * detJ, 1e-14)
    cores = [load_core(G[d], sp[d].flat_weights(), sp[d].full_tables()[0]) for d in range(3)]
    assert np.max(np.abs(tt_full(cores) - F)) < 1e-12 * np.max(np.abs(F))
