// 1D tables and the FP64 geometry point evaluator.
//
// * Gauss rule: Golub-Welsch -- nodes are the eigenvalues of the symmetric
//   tridiagonal Jacobi matrix of the Legendre recurrence (off-diagonal
//   k / sqrt(4k^2 - 1)), weights 2 v_0^2 from the normalised eigenvectors;
//   eigenpairs by cyclic Jacobi rotations on the dense m x m matrix (m <= 8),
//   computed once on the host and passed to the table kernel by value.
// * Basis: for element e the nonzero functions are e..e+p (open uniform
//   knots, knot span e+p); values by the Cox-de Boor triangle of Section 2.1
//   and first derivatives by its derivative formula applied to the degree
//   p-1 values.
// * Geometry (Section 3.3): the exact coarse NURBS patch -- radial degree-1
//   B-spline, angular rational quadratic quarter arc with weights 1,
//   sqrt(2)/2, 1, axial degree-1 B-spline -- composed with the analytic twist
//   and swell; J, det J, J^{-1} and R = det J J^{-1} J^{-T} (Eq. Rxi) in FP64.
// * Source: f = -Laplace(u) of the manufactured solution by hyper-dual
//   numbers (exact second derivatives), so f det J is available at any point.
#include "geom_device.cuh"

namespace ttiga {

GeomParams geom_params(const tt_iga_geom_desc &g) {
  GeomParams p{};
  p.kind = g.kind;
  p.r_in = g.r_in; p.r_out = g.r_out; p.height = g.height; p.twist = g.twist; p.swell = g.swell;
  p.lx = g.lx; p.ly = g.ly; p.lz = g.lz;
  return p;
}

RhsParams rhs_params(const tt_iga_rhs_desc *r) {
  RhsParams p;
  memset(&p, 0, sizeof p);
  if (!r) return p;
  p.has = 1;
  p.kind = r->kind;
  p.n_modes = r->n_modes;
  for (int k = 0; k < r->n_modes && k < TT_IGA_MAX_MODES; ++k) {
    p.a[k] = r->a[k];
    p.c[k] = r->c[k];
    for (int d = 0; d < 3; ++d) p.b[k][d] = r->b[k][d];
  }
  p.value = r->value;
  return p;
}

struct GaussRule {
  double x[8], w[8];
};

__global__ void k_basis_tables(int n, int p, int nq, GaussRule rule, double *pts, double *wts, double *N,
                               double *dN) {
  const double *gx = rule.x, *gw = rule.w;
  const int ne = n - p, Q = ne * nq;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    const int e = q / nq, l = q % nq;
    const double h = 1.0 / ne;
    const double x = (e + 0.5 * (gx[l] + 1.0)) * h;
    pts[q] = x;
    wts[q] = 0.5 * h * gw[l];
    double Nv[9], Dv[9];
    local_basis(x, e + p, n, p, Nv, Dv);
    for (int k = 0; k <= p; ++k) {
      N[(long long)q * (p + 1) + k] = Nv[k];
      dN[(long long)q * (p + 1) + k] = Dv[k];
    }
  }
}

void basis_tables(Ctx *c, int n, int p, int nq, double *pts, double *wts, double *N, double *dN) {
  TTI_CHECK_ARG(p >= 1 && p <= 7 && nq >= 1 && nq <= 8 && n >= p + 1, "basis tables: bad n=%d p=%d nq=%d", n, p, nq);
  const int Q = (n - p) * nq;
  // the nq-point rule on [-1, 1] (nq <= 8) is computed once on the host and passed by value
  GaussRule rule{};
  golub_welsch(nq, rule.x, rule.w);
  k_basis_tables<<<grid1d(Q, 128), 128, 0, c->stream>>>(n, p, nq, rule, pts, wts, N, dN);
  TTI_LAUNCH();
}

void build_space(Ctx *c, Space &s, int n, int p, int nq) {
  s.n = n; s.p = p; s.nq = nq; s.ne = n - p; s.Q = s.ne * nq;
  s.pts = DBuf(c, s.Q * sizeof(double));
  s.wts = DBuf(c, s.Q * sizeof(double));
  s.N = DBuf(c, (size_t)s.Q * (p + 1) * sizeof(double));
  s.dN = DBuf(c, (size_t)s.Q * (p + 1) * sizeof(double));
  basis_tables(c, n, p, nq, s.pts.d(), s.wts.d(), s.N.d(), s.dN.d());
}

__global__ void k_geom_points(GeomParams g, RhsParams f, const double *x1, const double *x2, const double *x3, int m,
                              const int *idx, double *out, int *status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int bad = 0;
    double o[8];
    point_outputs(g, f, x1[idx[3 * i]], x2[idx[3 * i + 1]], x3[idx[3 * i + 2]], o, &bad);
    for (int k = 0; k < 8; ++k) out[(long long)i * 8 + k] = o[k];
    if (bad) atomicMax(status, (int)DS_BAD_GEOMETRY);
  }
}

void geom_points(Ctx *c, const GeomParams &g, const RhsParams &f, const double *x1, const double *x2, const double *x3,
                 int m, const int *idx, double *out) {
  if (m <= 0) return;
  k_geom_points<<<grid1d(m, 128), 128, 0, c->stream>>>(g, f, x1, x2, x3, m, idx, out, c->dstatus);
  TTI_LAUNCH();
}

}  // namespace ttiga
