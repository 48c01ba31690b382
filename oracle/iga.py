"""Full-grid IGA discretisation of -Laplace(u) = f (oracle, Sections 3.1-3.3).

TEST INFRASTRUCTURE ONLY.  This is the plain definition the TT path
approximates: element-loop quadrature of

    K_ab = int grad_xi N_a^T R(xi) grad_xi N_b d xi          (Eq. Kfinal)
    F_a  = int f N_a det J d xi                               (Eq. ffinal)

with the same per-direction Gauss rule as the TT path (p+1 points per element
unless stated), homogeneous Dirichlet data on all six faces imposed by
dropping the first and last basis function of every direction (the open knot
vector makes the basis interpolatory at the ends) -- or, for the
non-homogeneous Dirichlet problem of Section 4.3 (constant data on some faces,
natural conditions on the others), a lift g carrying the data on the dropped
functions and the right-hand side F - K g, plus, for a constant normal flux on
a natural face, the face load int flux N_a dGamma -- a Jacobi-preconditioned
conjugate-gradient solve of the restricted system, and the relative L2 error
of Eq. (L2norm) read as sqrt(int (u_h - u)^2) / sqrt(int u^2) with p+3 Gauss
points per element.

Data layout: K is held as a stencil array Kst[i1, i2, i3, o1, o2, o3] with
entry K(i, j) at o_d = j_d - i_d + p (tensor-product B-splines of degree p
couple only |i_d - j_d| <= p).  Multi-indices (i1, i2, i3) are arrays with i1
on the first axis; the flattened global index used by the dense helpers is
g = i1 + n1 (i2 + n2 i3) (i1 fastest).

Pins: tests/test_oracle_iga.py (Kronecker structure on the identity map with
textbook 1D matrices, symmetry, K 1 = 0, SPD after restriction, volume, dense
LU on tiny meshes, energy identity, L2 convergence rate h^(p+1));
tests/test_oracle_bc.py (Dirichlet data); tests/test_oracle_neumann.py (face
loads against basis-integral and surface-area closed forms, exact linear
solutions with flux data, the mixed ring problem's convergence).
"""
import numpy as np

from .geometry import coefficient_tensor
from .spline import bspline_basis, gauss_legendre, open_uniform_knots


class Space1D:
    """Open uniform B-spline space of degree p with n functions and its Gauss rule."""

    def __init__(self, n, p, nq=None):
        self.n, self.p = int(n), int(p)
        self.nq = int(nq) if nq is not None else self.p + 1
        self.knots = open_uniform_knots(self.n, self.p)
        self.ne = self.n - self.p
        t, w = gauss_legendre(self.nq)
        h = 1.0 / self.ne
        left = np.arange(self.ne) * h
        # points[e, l] and weights[e, l] of the mapped rule on element e
        self.points = left[:, None] + 0.5 * h * (t[None, :] + 1.0)
        self.weights = np.broadcast_to(0.5 * h * w[None, :], self.points.shape).copy()
        N, dN = bspline_basis(self.knots, self.p, self.points.ravel())
        N = N.reshape(self.ne, self.nq, self.n)
        dN = dN.reshape(self.ne, self.nq, self.n)
        # local tables: the p+1 functions e..e+p that are nonzero on element e
        idx = np.arange(self.ne)[:, None] + np.arange(self.p + 1)[None, :]
        self.N = np.take_along_axis(N, idx[:, None, :], axis=2)
        self.dN = np.take_along_axis(dN, idx[:, None, :], axis=2)
        assert np.allclose(self.N.sum(axis=2), 1.0)

    @property
    def Q(self):
        return self.ne * self.nq

    def flat_points(self):
        return self.points.ravel()

    def flat_weights(self):
        return self.weights.ravel()

    def full_tables(self):
        """N[a, q] and N'[a, q] for all n functions at all Q quadrature points."""
        N, dN = bspline_basis(self.knots, self.p, self.flat_points())
        return N.T.copy(), dN.T.copy()


def _element_block(sp, geom, source, e1, e2, e3):
    """Element matrices and load vectors for the elements (e1[k], e2, e3), k = 0..len(e1)-1.

    Returns Kloc[k, A, B] and Floc[k, A] over the (p+1)^3 local functions
    A = (a1, a2, a3) in C order, following Eq. (Kfinal) and Eq. (ffinal):
    Kloc[k, A, B] = sum_q w_q grad N_A(q)^T R(q) grad N_B(q) and
    Floc[k, A] = sum_q w_q f(x(q)) det J(q) N_A(q).
    """
    s1, s2, s3 = sp
    e1 = np.atleast_1d(e1)
    nel = len(e1)
    nq1, nq2, nq3 = s1.nq, s2.nq, s3.nq
    P1, P2, P3 = s1.p + 1, s2.p + 1, s3.p + 1
    X, J = geom.map(s1.points[e1].ravel(), s2.points[e2], s3.points[e3])
    detJ, R = coefficient_tensor(J)
    w = (s1.weights[e1].reshape(nel, nq1)[:, :, None, None] * s2.weights[e2][None, None, :, None]
         * s3.weights[e3][None, None, None, :])  # [k, l1, l2, l3]
    detJ = detJ.reshape(nel, nq1, nq2, nq3)
    R = R.reshape(nel, nq1, nq2, nq3, 3, 3)
    N1, D1 = s1.N[e1], s1.dN[e1]  # [k, l1, a1]
    N2, D2 = s2.N[e2], s2.dN[e2]  # [l2, a2]
    N3, D3 = s3.N[e3], s3.dN[e3]  # [l3, a3]
    # grad_xi N_A at every quadrature point: G[k, l1, l2, l3, a1, a2, a3, i]
    G = np.empty((nel, nq1, nq2, nq3, P1, P2, P3, 3))
    G[..., 0] = np.einsum("kxa,yb,zc->kxyzabc", D1, N2, N3)
    G[..., 1] = np.einsum("kxa,yb,zc->kxyzabc", N1, D2, N3)
    G[..., 2] = np.einsum("kxa,yb,zc->kxyzabc", N1, N2, D3)
    nqt, nloc = nq1 * nq2 * nq3, P1 * P2 * P3
    G = G.reshape(nel, nqt, nloc, 3)
    Rw = (R * w[..., None, None]).reshape(nel, nqt, 3, 3)
    H = np.einsum("kqai,kqij->kqaj", G, Rw)
    Kloc = np.einsum("kqaj,kqbj->kab", H, G, optimize=True)
    Nv = np.einsum("kxa,yb,zc->kxyzabc", N1, N2, N3).reshape(nel, nqt, nloc)
    if source is not None:
        fw = (source.f(X).reshape(nel, nq1, nq2, nq3) * detJ * w).reshape(nel, nqt)
        Floc = np.einsum("kq,kqa->ka", fw, Nv)
    else:
        Floc = np.zeros((nel, nloc))
    return Kloc, Floc


def assemble(spaces, geom, source):
    """Stencil stiffness Kst[n1, n2, n3, b1, b2, b3] and load F[n1, n2, n3] (b_d = 2 p_d + 1).

    Element loop over every element; each local matrix is scattered to the
    global rows e_d + a_d at stencil offsets b_d - a_d + p_d.
    """
    s1, s2, s3 = spaces
    n = (s1.n, s2.n, s3.n)
    p = (s1.p, s2.p, s3.p)
    b = tuple(2 * q + 1 for q in p)
    Kst = np.zeros(n + b)
    F = np.zeros(n)
    P = tuple(q + 1 for q in p)
    loc = np.array(np.unravel_index(np.arange(P[0] * P[1] * P[2]), P)).T  # [A, 3]
    for e3 in range(s3.ne):
        for e2 in range(s2.ne):
            e1 = np.arange(s1.ne)
            Kloc, Floc = _element_block(spaces, geom, source, e1, e2, e3)
            rows = np.stack([e1[:, None] + loc[None, :, 0], e2 + loc[None, :, 1] + 0 * e1[:, None],
                             e3 + loc[None, :, 2] + 0 * e1[:, None]], axis=-1)  # [k, A, 3]
            off = loc[None, :, :] - loc[:, None, :] + np.array(p)  # [A, B, 3]
            r = np.broadcast_to(rows[:, :, None, :], Kloc.shape + (3,))
            o = np.broadcast_to(off[None], Kloc.shape + (3,))
            np.add.at(Kst, (r[..., 0], r[..., 1], r[..., 2], o[..., 0], o[..., 1], o[..., 2]), Kloc)
            np.add.at(F, (rows[..., 0], rows[..., 1], rows[..., 2]), Floc)
    return Kst, F


def stencil_matvec(Kst, x, p):
    """y(i) = sum_j K(i, j) x(j) for a stencil matrix; x is zero outside its array."""
    n = x.shape
    b = Kst.shape[3:]
    pad = np.pad(x, [(q, q) for q in p])
    y = np.zeros(n)
    for o1 in range(b[0]):
        for o2 in range(b[1]):
            for o3 in range(b[2]):
                y += Kst[..., o1, o2, o3] * pad[o1:o1 + n[0], o2:o2 + n[1], o3:o3 + n[2]]
    return y


def restrict(Kst, F):
    """Homogeneous Dirichlet on all faces: keep interior rows/columns 1..n_d-2."""
    Ki = Kst[1:-1, 1:-1, 1:-1].copy()
    p = tuple((q - 1) // 2 for q in Kst.shape[3:])
    # zero the couplings to the dropped boundary functions
    m = Ki.shape[:3]
    for d in range(3):
        for o in range(Kst.shape[3 + d]):
            shift = o - p[d]
            idx = np.arange(m[d])
            bad = (idx + shift < 0) | (idx + shift >= m[d])
            sl = [slice(None)] * 6
            sl[d] = bad
            sl[3 + d] = o
            Ki[tuple(sl)] = 0.0
    return Ki, F[1:-1, 1:-1, 1:-1].copy()


def bc_ranges(n, dirichlet):
    """Kept functions per direction: a Dirichlet face drops the basis function that is
    interpolatory on it (index 0 on xi_d = 0, n_d - 1 on xi_d = 1).  Face f = 2 d + side."""
    lo = [1 if dirichlet[2 * d] else 0 for d in range(3)]
    hi = [1 if dirichlet[2 * d + 1] else 0 for d in range(3)]
    return lo, hi


def restrict_bc(Kst, F, lo, hi):
    """Rows/columns lo_d .. n_d - 1 - hi_d of the stencil operator and the load vector."""
    n = Kst.shape[:3]
    sl = tuple(slice(lo[d], n[d] - hi[d]) for d in range(3))
    Ki = Kst[sl].copy()
    p = tuple((q - 1) // 2 for q in Kst.shape[3:])
    m = Ki.shape[:3]
    for d in range(3):
        for o in range(Kst.shape[3 + d]):
            shift = o - p[d]
            idx = np.arange(m[d])
            bad = (idx + shift < 0) | (idx + shift >= m[d])
            sel = [slice(None)] * 6
            sel[d] = bad
            sel[3 + d] = o
            Ki[tuple(sel)] = 0.0
    return Ki, F[sl].copy()


def lift_vector(n, dirichlet, value):
    """Coefficients g of the Dirichlet data: the constant face value on the interpolatory
    boundary function of every Dirichlet face, zero elsewhere.  Nonzero data is accepted on
    the faces of one direction only, and the faces of the other two directions must then be
    natural, so that no coefficient belongs to two faces with different data."""
    g = np.zeros(n)
    dirs = [d for d in range(3) if any(dirichlet[2 * d + s] and value[2 * d + s] != 0.0 for s in range(2))]
    assert len(dirs) <= 1, "nonzero Dirichlet data on more than one direction"
    for d in dirs:
        assert not any(dirichlet[2 * e + s] for e in range(3) if e != d for s in range(2)), \
            "nonzero Dirichlet data with Dirichlet faces in another direction"
        for s in range(2):
            if dirichlet[2 * d + s]:
                sel = [slice(None)] * 3
                sel[d] = 0 if s == 0 else n[d] - 1
                g[tuple(sel)] = value[2 * d + s]
    return g


def neumann_load(spaces, geom, face, flux):
    """Surface load vector f_s (Section 3.3) of a constant normal flux du/dn = flux on
    face = 2 d + side (outward normal):
    F_a = int_face flux N_a dGamma, dGamma = |dx/dxi_e x dx/dxi_f| dxi_e dxi_f over the two
    tangential directions e < f, with the per-direction Gauss rules of the spaces.  Only the
    functions that are nonzero on the face (index 0 on side 0, n_d - 1 on side 1) receive load."""
    d, side = divmod(face, 2)
    e, f = [k for k in range(3) if k != d]
    n = tuple(sp.n for sp in spaces)
    xs = [sp.flat_points() for sp in spaces]
    ws = [sp.flat_weights() for sp in spaces]
    xs[d] = np.array([float(side)])
    X, J = geom.map(*xs)
    area = np.linalg.norm(np.cross(J[..., :, e], J[..., :, f]), axis=-1)  # [Q1|1, Q2|1, Q3|1]
    area = np.squeeze(area, axis=d)
    Ne, _ = bspline_basis(spaces[e].knots, spaces[e].p, xs[e])
    Nf, _ = bspline_basis(spaces[f].knots, spaces[f].p, xs[f])
    G = np.einsum("qa,rb,qr,q,r->ab", Ne, Nf, flux * area, ws[e], ws[f], optimize=True)
    F = np.zeros(n)
    sel = [slice(None)] * 3
    sel[d] = 0 if side == 0 else n[d] - 1
    F[tuple(sel)] = G
    return F


def solve_bc(spaces, geom, source, dirichlet, value, tol=1e-14, flux=None):
    """Dirichlet faces with constant data, natural conditions on the others (zero flux, or the
    constant normal flux flux[face] on a natural face): u = g + u_I with
    K_II u_I = F_I + (F_Gamma)_I - (K g)_I; returns the full coefficient array."""
    assert any(dirichlet), "pure natural conditions leave K singular"
    Kst, F = assemble(spaces, geom, source)
    if flux is not None:
        for face in range(6):
            if flux[face] != 0.0:
                assert not dirichlet[face], "flux data on a Dirichlet face"
                F = F + neumann_load(spaces, geom, face, flux[face])
    n = F.shape
    p = tuple(s.p for s in spaces)
    g = lift_vector(n, dirichlet, value)
    lo, hi = bc_ranges(n, dirichlet)
    rhs = F - stencil_matvec(Kst, g, p)
    Ki, Fi = restrict_bc(Kst, rhs, lo, hi)
    ui, it, relres = pcg(Ki, Fi, p, tol=tol)
    u = g.copy()
    u[tuple(slice(lo[d], n[d] - hi[d]) for d in range(3))] += ui
    return u, {"iterations": it, "relres": relres, "Kst": Kst, "F": F, "lo": lo, "hi": hi, "lift": g,
               "Ki": Ki, "Fi": Fi}


def pcg(Kst, F, p, tol=1e-14, maxiter=100000, x0=None):
    """Jacobi-preconditioned conjugate gradients on the stencil system K x = F.

    Stops when ||F - K x||_2 <= tol ||F||_2.  Returns (x, iterations, relres).
    """
    diag = Kst[(...,) + tuple(p)]
    x = np.zeros_like(F) if x0 is None else x0.copy()
    r = F - stencil_matvec(Kst, x, p)
    z = r / diag
    d = z.copy()
    rz = np.vdot(r, z)
    nf = np.linalg.norm(F)
    if nf == 0.0:
        return x, 0, 0.0
    it = 0
    while np.linalg.norm(r) > tol * nf and it < maxiter:
        Kd = stencil_matvec(Kst, d, p)
        alpha = rz / np.vdot(d, Kd)
        x += alpha * d
        r -= alpha * Kd
        z = r / diag
        rz_new = np.vdot(r, z)
        d = z + (rz_new / rz) * d
        rz = rz_new
        it += 1
    relres = np.linalg.norm(F - stencil_matvec(Kst, x, p)) / nf
    return x, it, relres


def stencil_to_dense(Kst, p):
    """Dense N x N matrix of a stencil operator, global index g = i1 + n1 (i2 + n2 i3)."""
    n = Kst.shape[:3]
    N = n[0] * n[1] * n[2]
    A = np.zeros((N, N))
    b = Kst.shape[3:]
    for i3 in range(n[2]):
        for i2 in range(n[1]):
            for i1 in range(n[0]):
                g = i1 + n[0] * (i2 + n[1] * i3)
                for o1 in range(b[0]):
                    for o2 in range(b[1]):
                        for o3 in range(b[2]):
                            j = (i1 + o1 - p[0], i2 + o2 - p[1], i3 + o3 - p[2])
                            if all(0 <= j[d] < n[d] for d in range(3)):
                                A[g, j[0] + n[0] * (j[1] + n[1] * j[2])] += Kst[i1, i2, i3, o1, o2, o3]
    return A


def to_flat(x):
    """Flatten a (n1, n2, n3) array with i1 fastest."""
    return np.asarray(x).transpose(2, 1, 0).ravel()


def from_flat(v, n):
    return np.asarray(v).reshape(n[2], n[1], n[0]).transpose(2, 1, 0)


def solve(spaces, geom, source, tol=1e-14):
    """Assemble, restrict and solve; returns the full coefficient array (zeros on the boundary)."""
    Kst, F = assemble(spaces, geom, source)
    Ki, Fi = restrict(Kst, F)
    p = tuple(s.p for s in spaces)
    ui, it, relres = pcg(Ki, Fi, p, tol=tol)
    u = np.zeros(F.shape)
    u[1:-1, 1:-1, 1:-1] = ui
    return u, {"iterations": it, "relres": relres, "Kst": Kst, "F": F}


def evaluate(spaces, coef, xi1, xi2, xi3):
    """u_h = sum_a c_a N_a on the tensor grid xi1 x xi2 x xi3."""
    N1, _ = bspline_basis(spaces[0].knots, spaces[0].p, xi1)
    N2, _ = bspline_basis(spaces[1].knots, spaces[1].p, xi2)
    N3, _ = bspline_basis(spaces[2].knots, spaces[2].p, xi3)
    return np.einsum("ia,jb,kc,abc->ijk", N1, N2, N3, coef, optimize=True)


def l2_error(spaces, geom, coef, exact):
    """Relative L2 error sqrt(int (u_h - u)^2 dOmega / int u^2 dOmega), p+3 Gauss points per element."""
    fine = [Space1D(s.n, s.p, nq=s.p + 3) for s in spaces]
    x1, x2, x3 = (f.flat_points() for f in fine)
    w1, w2, w3 = (f.flat_weights() for f in fine)
    num = 0.0
    den = 0.0
    for k in range(len(x3)):
        X, J = geom.map(x1, x2, x3[k:k + 1])
        detJ = np.linalg.det(J)
        uh = evaluate(spaces, coef, x1, x2, x3[k:k + 1])
        ue = exact.u(X)
        w = w1[:, None, None] * w2[None, :, None] * w3[k] * detJ
        num += np.sum(w * (uh - ue) ** 2)
        den += np.sum(w * ue ** 2)
    return float(np.sqrt(num / den))


def stiffness_rows(spaces, geom, rows):
    """Rows K(a, .) for multi-indices a (list of triples), each as a stencil block [b1, b2, b3].

    Computes only the element matrices of the elements in the support of N_a.
    """
    p = tuple(s.p for s in spaces)
    P = tuple(q + 1 for q in p)
    out = []
    for a in rows:
        blk = np.zeros(tuple(2 * q + 1 for q in p))
        ranges = [range(max(0, a[d] - p[d]), min(spaces[d].ne - 1, a[d]) + 1) for d in range(3)]
        els = [(x, y, z) for x in ranges[0] for y in ranges[1] for z in ranges[2]]
        Kloc = np.concatenate([_element_block(spaces, geom, None, [e[0]], e[1], e[2])[0] for e in els])
        for k, e in enumerate(els):
            la = tuple(a[d] - e[d] for d in range(3))
            A = np.ravel_multi_index(la, P)
            for B in range(Kloc.shape[2]):
                lb = np.unravel_index(B, P)
                o = tuple(lb[d] - la[d] + p[d] for d in range(3))
                blk[o] += Kloc[k, A, B]
        out.append(blk)
    return out


def load_entries(spaces, geom, source, rows):
    """Entries F(a) for multi-indices a, from the elements in the support of N_a."""
    p = tuple(s.p for s in spaces)
    P = tuple(q + 1 for q in p)
    out = []
    for a in rows:
        ranges = [range(max(0, a[d] - p[d]), min(spaces[d].ne - 1, a[d]) + 1) for d in range(3)]
        els = [(x, y, z) for x in ranges[0] for y in ranges[1] for z in ranges[2]]
        Floc = np.concatenate([_element_block(spaces, geom, source, [e[0]], e[1], e[2])[1] for e in els])
        val = 0.0
        for k, e in enumerate(els):
            val += Floc[k, np.ravel_multi_index(tuple(a[d] - e[d] for d in range(3)), P)]
        out.append(val)
    return np.array(out)
