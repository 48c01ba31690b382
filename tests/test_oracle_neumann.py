"""Pins of the oracle's Neumann (flux) data on natural faces (the surface load vector f_s of
Section 3.3): the face load against closed forms of B-spline integrals and surface areas, exactness of
linear solutions on the box (both signs of the outward normal), and convergence of the mixed
ring problem to its log solution."""
import math

import numpy as np
import pytest

from oracle.geometry import Annulus, Box
from oracle.iga import Space1D, evaluate, l2_error, neumann_load, solve_bc
from oracle.manufactured import RingMixed


def _integral_of_basis(sp):
    """int_0^1 N_i = (t_{i+p+1} - t_i) / (p + 1) for every function of the space."""
    t, p = sp.knots, sp.p
    return (t[p + 1:p + 1 + sp.n] - t[:sp.n]) / (p + 1)


@pytest.mark.parametrize("face", range(6))
def test_box_face_load_is_the_tensor_product_of_basis_integrals(face):
    """On a box the area density is the product of the two tangential side lengths, so
    F_a = flux L_e L_f int N_i int N_j on the face layer and zero elsewhere."""
    L = (2.0, 3.0, 0.5)
    sp = [Space1D(6, 2), Space1D(7, 3), Space1D(5, 1)]
    flux = -1.75
    F = neumann_load(sp, Box(*L), face, flux)
    d, side = divmod(face, 2)
    e, f = [k for k in range(3) if k != d]
    G = flux * L[e] * L[f] * np.outer(_integral_of_basis(sp[e]), _integral_of_basis(sp[f]))
    sel = [slice(None)] * 3
    sel[d] = 0 if side == 0 else sp[d].n - 1
    assert np.max(np.abs(F[tuple(sel)] - G)) < 1e-14
    F[tuple(sel)] = 0.0
    assert not F.any()


@pytest.mark.parametrize("face,radius", [(0, 1.0), (1, 2.0)])
@pytest.mark.parametrize("twist", [0.0, 0.8])
def test_cylinder_face_load_sums_to_flux_times_area(face, radius, twist):
    """Partition of unity: sum_a F_a = flux |face|.  The radial faces of the quarter cylinder
    have area (pi / 2) rho H; a twist about the axis shears each face along itself and leaves
    its area unchanged (|dx/dtheta x dx/dz| = rho theta'(xi_2) H, while |dx/dtheta| |dx/dz|
    grows with the twist)."""
    sp = [Space1D(6, 2), Space1D(14, 3), Space1D(9, 3)]
    F = neumann_load(sp, Annulus(1.0, 2.0, 1.0, twist=twist), face, 0.7)
    assert abs(F.sum() - 0.7 * 0.5 * math.pi * radius) < 1e-9


def test_angular_face_load_of_the_cylinder():
    """Face xi_2 = 0 of the quarter cylinder is the rectangle [r_in, r_out] x [0, H] in the
    plane y = 0: flux (r_out - r_in) H int N_i int N_k."""
    sp = [Space1D(6, 2), Space1D(7, 2), Space1D(5, 3)]
    F = neumann_load(sp, Annulus(1.0, 2.5, 2.0), 2, 1.3)
    G = 1.3 * 1.5 * 2.0 * np.outer(_integral_of_basis(sp[0]), _integral_of_basis(sp[2]))
    assert np.max(np.abs(F[:, 0, :] - G)) < 1e-13 and not F[:, 1:, :].any()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("side", [0, 1])
def test_linear_solution_with_flux_is_exact_on_the_box(p, side):
    """u = a (x - x_D) with u = 0 on the face x = x_D and the outward flux du/dn = +a on the face
    x = Lx (side 1) or -a on x = 0 (side 0); zero flux on the other faces.  u lies in the spline
    space, so the Galerkin solution is exact."""
    L, a = 2.0, 1.5
    sp = [Space1D(p + 4, p), Space1D(p + 2, p), Space1D(p + 3, p)]
    dirichlet = [side == 1, side == 0, False, False, False, False]
    flux = [0.0] * 6
    flux[side] = a if side == 1 else -a
    u, info = solve_bc(sp, Box(L, 1.0, 1.0), None, dirichlet, [0.0] * 6, flux=flux)
    assert info["relres"] < 1e-13
    x = np.linspace(0.0, 1.0, 7)
    uh = evaluate(sp, u, x, x[::2], x[1::3])
    xd = 0.0 if side == 1 else L
    assert np.max(np.abs(uh - a * (L * x[:, None, None] - xd))) < 1e-11


@pytest.mark.parametrize("inner,outer", [(("value", 1.0), ("flux", 0.5)), (("flux", -0.75), ("value", 2.0))])
def test_mixed_ring_converges_at_rate_p_plus_one(inner, outer):
    """The quarter cylinder with a value on one radial face and a flux on the other: the L2
    error to u = A + B ln(rho / r_in) decays like h^(p+1)."""
    p = 2
    geom = Annulus()
    dirichlet = [inner[0] == "value", outer[0] == "value", False, False, False, False]
    value = [inner[1] if dirichlet[0] else 0.0, outer[1] if dirichlet[1] else 0.0, 0, 0, 0, 0]
    flux = [0.0 if dirichlet[0] else inner[1], 0.0 if dirichlet[1] else outer[1], 0, 0, 0, 0]
    ex = RingMixed(1.0, 2.0, inner, outer)
    errs, ns = [], [6, 10]
    for n in ns:
        sp = [Space1D(n, p), Space1D(n, p), Space1D(p + 1, p)]
        u, _ = solve_bc(sp, geom, None, dirichlet, value, flux=flux)
        errs.append(l2_error(sp, geom, u, ex))
    rate = math.log(errs[0] / errs[1]) / math.log((ns[1] - p) / (ns[0] - p))
    assert rate > p + 0.6, (errs, rate)


def test_ring_mixed_solution_meets_its_boundary_data():
    """Values and outward fluxes of u = A + B ln(rho / r_in) on both radial faces, by central
    differences along the radius."""
    for inner, outer in [(("value", 1.0), ("flux", 0.5)), (("flux", -0.75), ("value", 2.0)),
                         (("value", 1.0), ("value", 2.0))]:
        ex = RingMixed(1.0, 2.0, inner, outer)
        h = 1e-6
        for r, data, sign in ((1.0, inner, -1.0), (2.0, outer, 1.0)):
            P = np.array([[r * 0.6, r * 0.8, 0.4]])
            if data[0] == "value":
                assert abs(ex.u(P)[0] - data[1]) < 1e-14
            else:
                du = (ex.u(P * (1 + h / r)) - ex.u(P * (1 - h / r)))[0] / (2 * h)
                assert abs(sign * du - data[1]) < 1e-8
    with pytest.raises(AssertionError):
        RingMixed(1.0, 2.0, ("flux", 1.0), ("flux", 0.5))


def test_flux_on_a_dirichlet_face_is_rejected():
    sp = [Space1D(4, 1)] * 3
    with pytest.raises(AssertionError):
        solve_bc(sp, Box(), None, [True] * 6, [0.0] * 6, flux=[1.0, 0, 0, 0, 0, 0])
