"""Geometry maps x(xi), Jacobian J, det J and the coefficient tensor R (oracle).

TEST INFRASTRUCTURE ONLY. Plain FP64 numpy.

* Section 3.3: the geometry is the exact NURBS map x(xi) = N^T(xi) P, evaluated
  at quadrature points from the nonzero basis functions only.  The paper gives
  no control nets for its shapes, so the two maps here are built from the
  NURBS pieces of ``oracle.spline``:

  - ``Annulus``: a single-patch quarter thick-walled cylinder.  xi_1 is the
    radial direction (degree-1 B-spline with control values r_in, r_out),
    xi_2 the angular direction (the quadratic NURBS quarter arc, weights
    1, sqrt(2)/2, 1) and xi_3 the axial direction (degree-1 B-spline with
    control values 0, H).  The tensor-product NURBS volume with that control
    net is exactly x0 = r(xi_1) C(xi_2), z = H xi_3 because the radial and
    axial weights are 1.  An optional analytic twist about the z axis by
    angle twist*zeta and a radial swell by s = 1 + swell*sin(pi zeta)
    (zeta = z/H) make the coefficient fields non-separable.
  - ``Box``: the identity-like map onto [0,Lx]x[0,Ly]x[0,Lz].

* Section 3.3, change of variables: J = dx/dxi, d Omega = det J d xi (the
  determinant, not an absolute value; det J <= 0 is rejected).
* Eq. (Rxi): R(xi) = J^{-1} J^{-T} det J, six unique entries.

Pins (tests/test_oracle_geometry.py): finite differences of x(xi), the closed
form det J = H s^2 (r_out - r_in) r theta'(xi_2), the diagonal closed form of R
for the untwisted cylinder and the volume of the mapped domain.
"""
import numpy as np

from .spline import bspline_basis, quarter_arc


def _linear(a, b, x):
    """Degree-1 B-spline curve with control values a, b on knots (0,0,1,1): value and derivative."""
    N, dN = bspline_basis(np.array([0.0, 0.0, 1.0, 1.0]), 1, x)
    return N @ np.array([a, b]), dN @ np.array([a, b])


class Annulus:
    """Quarter annulus r_in..r_out, height H, optional twist and swell."""

    def __init__(self, r_in=1.0, r_out=2.0, height=1.0, twist=0.0, swell=0.0):
        self.r_in, self.r_out, self.height = float(r_in), float(r_out), float(height)
        self.twist, self.swell = float(twist), float(swell)

    def map(self, xi1, xi2, xi3):
        """Physical points X[..., 3] and Jacobian J[..., 3, 3] (J[a, b] = dx_a / dxi_b).

        xi1, xi2, xi3 are 1D arrays; the result is on their tensor grid with
        shape (len(xi1), len(xi2), len(xi3), ...).
        """
        r, dr = _linear(self.r_in, self.r_out, xi1)
        C, dC = quarter_arc(xi2)
        z, dz = _linear(0.0, self.height, xi3)
        r, dr = r[:, None, None], dr[:, None, None]
        cx, cy = C[None, :, 0, None], C[None, :, 1, None]
        dcx, dcy = dC[None, :, 0, None], dC[None, :, 1, None]
        zz, dzz = z[None, None, :], dz[None, None, :]
        zeta = zz / self.height
        phi = self.twist * zeta
        dphi = self.twist / self.height
        s = 1.0 + self.swell * np.sin(np.pi * zeta)
        ds = self.swell * np.pi * np.cos(np.pi * zeta) / self.height
        cp, sp = np.cos(phi), np.sin(phi)
        x0, y0 = r * cx, r * cy
        shape = np.broadcast(x0, zz).shape
        X = np.empty(shape + (3,))
        X[..., 0] = s * (cp * x0 - sp * y0)
        X[..., 1] = s * (sp * x0 + cp * y0)
        X[..., 2] = np.broadcast_to(zz, shape)
        J = np.zeros(shape + (3, 3))
        # d/dxi_1 and d/dxi_2 act on (x0, y0) only.
        for b, (ax, ay) in enumerate([(dr * cx, dr * cy), (r * dcx, r * dcy)]):
            J[..., 0, b] = s * (cp * ax - sp * ay)
            J[..., 1, b] = s * (sp * ax + cp * ay)
        # d/dxi_3 acts through z = H xi_3 on s(z) and phi(z).
        J[..., 0, 2] = dzz * (ds * (cp * x0 - sp * y0) + s * dphi * (-sp * x0 - cp * y0))
        J[..., 1, 2] = dzz * (ds * (sp * x0 + cp * y0) + s * dphi * (cp * x0 - sp * y0))
        J[..., 2, 2] = np.broadcast_to(dzz, shape)
        return X, J

    def pullback(self, X):
        """Coordinates (x', y', zeta) of physical points with the twist and swell undone."""
        zeta = X[..., 2] / self.height
        phi = self.twist * zeta
        s = 1.0 + self.swell * np.sin(np.pi * zeta)
        xp = (np.cos(phi) * X[..., 0] + np.sin(phi) * X[..., 1]) / s
        yp = (-np.sin(phi) * X[..., 0] + np.cos(phi) * X[..., 1]) / s
        return xp, yp, zeta


class Box:
    """Map onto the box [0,Lx] x [0,Ly] x [0,Lz] (identity map for unit lengths)."""

    def __init__(self, lx=1.0, ly=1.0, lz=1.0):
        self.L = np.array([lx, ly, lz], dtype=np.float64)

    def map(self, xi1, xi2, xi3):
        shape = (len(xi1), len(xi2), len(xi3))
        X = np.empty(shape + (3,))
        X[..., 0] = self.L[0] * np.asarray(xi1)[:, None, None]
        X[..., 1] = self.L[1] * np.asarray(xi2)[None, :, None]
        X[..., 2] = self.L[2] * np.asarray(xi3)[None, None, :]
        J = np.zeros(shape + (3, 3))
        for a in range(3):
            J[..., a, a] = self.L[a]
        return X, J


def coefficient_tensor(J):
    """det J and R = J^{-1} J^{-T} det J (Eq. Rxi) at every point of J[..., 3, 3]."""
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0):
        raise ValueError("geometry map is not positively oriented (det J <= 0)")
    Jinv = np.linalg.inv(J)
    R = np.einsum("...ab,...cb->...ac", Jinv, Jinv) * detJ[..., None, None]
    return detJ, R


class NURBSPatch:
    """Single-patch trivariate NURBS volume (Section 2.2, the NURBS map of Eq. for x(xi)):

        X(xi) = sum_a w_a P_a N_a(xi) / sum_a w_a N_a(xi),  N_a = N_a1(xi1) N_a2(xi2) N_a3(xi3),

    degrees deg[d], open knot vectors knots[d] on [0, 1], control points ctrl[c1, c2, c3, 3] and
    positive weights w[c1, c2, c3].  The Jacobian follows from the quotient rule with the
    B-spline derivatives of spline.bspline_basis."""

    def __init__(self, degrees, knots, ctrl, weights):
        self.deg = [int(q) for q in degrees]
        self.knots = [np.asarray(k, dtype=np.float64) for k in knots]
        self.ctrl = np.asarray(ctrl, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        for d in range(3):
            assert len(self.knots[d]) == self.ctrl.shape[d] + self.deg[d] + 1

    def map(self, xi1, xi2, xi3):
        from .spline import bspline_basis
        (N1, D1), (N2, D2), (N3, D3) = (bspline_basis(self.knots[d], self.deg[d], x)
                                        for d, x in enumerate((xi1, xi2, xi3)))
        wP = self.w[..., None] * self.ctrl
        W = np.einsum("ia,jb,kc,abc->ijk", N1, N2, N3, self.w, optimize=True)
        A = np.einsum("ia,jb,kc,abcd->ijkd", N1, N2, N3, wP, optimize=True)
        dW = [np.einsum("ia,jb,kc,abc->ijk", *B, self.w, optimize=True)
              for B in ((D1, N2, N3), (N1, D2, N3), (N1, N2, D3))]
        dA = [np.einsum("ia,jb,kc,abcd->ijkd", *B, wP, optimize=True)
              for B in ((D1, N2, N3), (N1, D2, N3), (N1, N2, D3))]
        X = A / W[..., None]
        J = np.empty(X.shape + (3,))
        for b in range(3):
            J[..., :, b] = (dA[b] - X * dW[b][..., None]) / W[..., None]
        return X, J


def quarter_cylinder_patch(r_in=1.0, r_out=2.0, height=1.0):
    """The quarter cylinder of Annulus (no twist, no swell) as a NURBS patch: radial degree 1,
    angular rational quadratic quarter circle (control (1,0), (1,1), (0,1), weights 1, sqrt(2)/2, 1),
    axial degree 1."""
    arc = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    warc = np.array([1.0, np.sqrt(0.5), 1.0])
    ctrl = np.zeros((2, 3, 2, 3))
    w = np.zeros((2, 3, 2))
    for i, r in enumerate((r_in, r_out)):
        for j in range(3):
            for k, z in enumerate((0.0, height)):
                ctrl[i, j, k] = [r * arc[j, 0], r * arc[j, 1], z]
                w[i, j, k] = warc[j]
    knots = [[0, 0, 1, 1], [0, 0, 0, 1, 1, 1], [0, 0, 1, 1]]
    return NURBSPatch((1, 2, 1), knots, ctrl, w)
