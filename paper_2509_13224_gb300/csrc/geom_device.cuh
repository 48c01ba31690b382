// Device functions of the geometry evaluator shared by the table, cross,
// evaluation and error kernels (Sections 2.1 and 3.3, Eq. Rxi).
#pragma once
#include "geom.cuh"

namespace ttiga {

// ------------------------------------------------------------------ tables

__device__ inline double knot_at(int i, int n, int p) {
  const int ne = n - p;
  if (i <= p) return 0.0;
  if (i >= n) return 1.0;
  return (double)(i - p) / (double)ne;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Golub-Welsch (single thread, m <= 8).
__host__ __device__ inline void golub_welsch(int m, double *x, double *w) {
  double A[8][8], V[8][8];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      A[i][j] = 0.0;
      V[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int k = 1; k < m; ++k) {
    const double b = k / sqrt(4.0 * k * k - 1.0);
    A[k - 1][k] = A[k][k - 1] = b;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) off += A[i][j] * A[i][j];
    if (off < 1e-34) break;
    for (int pp = 0; pp < m; ++pp)
      for (int q = pp + 1; q < m; ++q) {
        if (A[pp][q] == 0.0) continue;
        const double theta = (A[q][q] - A[pp][pp]) / (2.0 * A[pp][q]);
        const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // A <- A G
          const double akp = A[k][pp], akq = A[k][q];
          A[k][pp] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // A <- G^T A
          const double apk = A[pp][k], aqk = A[q][k];
          A[pp][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[k][pp], vkq = V[k][q];
          V[k][pp] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  // sort ascending
  int idx[8];
  for (int i = 0; i < m; ++i) idx[i] = i;
  for (int i = 1; i < m; ++i) {
    int v = idx[i], j = i - 1;
    while (j >= 0 && A[idx[j]][idx[j]] > A[v][v]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = v;
  }
  for (int i = 0; i < m; ++i) {
    x[i] = A[idx[i]][idx[i]];
    const double v0 = V[0][idx[i]];
    w[i] = 2.0 * v0 * v0;
  }
}

// Nonzero basis values N[0..p] (functions s-p..s) and derivatives at x in knot span s.
__device__ inline void local_basis(double x, int s, int n, int p, double *N, double *D) {
  double left[9], right[9], Np[9];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - knot_at(s + 1 - j, n, p);
    right[j] = knot_at(s + j, n, p) - x;
    if (j == p)
      for (int r = 0; r < p; ++r) Np[r] = N[r];  // degree p-1 values
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      const double tmp = N[r] / (right[r + 1] + left[j - r]);
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
  }
  if (p == 0) {
    D[0] = 0.0;
    return;
  }
  // dN_i = p N_i^{p-1}/(xi_{i+p} - xi_i) - p N_{i+1}^{p-1}/(xi_{i+p+1} - xi_{i+1}), i = s-p+j;
  // the degree p-1 functions nonzero in span s are s-p+1..s, held in Np[0..p-1].
  for (int j = 0; j <= p; ++j) {
    const int i = s - p + j;
    double v = 0.0;
    if (j >= 1) {
      const double den = knot_at(i + p, n, p) - knot_at(i, n, p);
      if (den > 0.0) v += p * Np[j - 1] / den;
    }
    if (j <= p - 1) {
      const double den = knot_at(i + p + 1, n, p) - knot_at(i + 1, n, p);
      if (den > 0.0) v -= p * Np[j] / den;
    }
    D[j] = v;
  }
}

// ----------------------------------------------------------- hyper-duals

struct HDual {
  double a, b, c, d;  // value, e1, e2, e1e2
};
__device__ __forceinline__ HDual hd(double a) { return {a, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ HDual operator+(HDual x, HDual y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
__device__ __forceinline__ HDual operator-(HDual x, HDual y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
__device__ __forceinline__ HDual operator*(HDual x, HDual y) {
  return {x.a * y.a, x.a * y.b + x.b * y.a, x.a * y.c + x.c * y.a, x.a * y.d + x.b * y.c + x.c * y.b + x.d * y.a};
}
__device__ __forceinline__ HDual operator*(double s, HDual x) { return {s * x.a, s * x.b, s * x.c, s * x.d}; }
__device__ __forceinline__ HDual operator+(double s, HDual x) { return {s + x.a, x.b, x.c, x.d}; }
__device__ __forceinline__ HDual chain(HDual x, double f0, double f1, double f2) {
  return {f0, f1 * x.b, f1 * x.c, f1 * x.d + f2 * x.b * x.c};
}
__device__ __forceinline__ HDual hsin(HDual x) {
  double s, c;
  sincos(x.a, &s, &c);
  return chain(x, s, c, -s);
}
__device__ __forceinline__ HDual hcos(HDual x) {
  double s, c;
  sincos(x.a, &s, &c);
  return chain(x, c, -s, -c);
}
__device__ __forceinline__ HDual hrecip(HDual x) {
  const double r = 1.0 / x.a;
  return chain(x, r, -r * r, 2.0 * r * r * r);
}

// Manufactured solution at physical point (x, y, z) (hyper-dual arguments).
__device__ inline HDual manufactured_u(const GeomParams &g, const RhsParams &f, HDual x, HDual y, HDual z) {
  const double PI = 3.141592653589793238462643383279502884;
  HDual bubble;
  if (g.kind == TT_IGA_GEOM_ANNULUS) {
    const HDual zeta = (1.0 / g.height) * z;
    const HDual phi = g.twist * zeta;
    const HDual inv_s = hrecip(1.0 + g.swell * hsin(PI * zeta));
    const HDual cp = hcos(phi), sp = hsin(phi);
    const HDual xp = (cp * x + sp * y) * inv_s;
    const HDual yp = (cp * y - sp * x) * inv_s;
    const HDual rho2 = xp * xp + yp * yp;
    bubble = (rho2 - hd(g.r_in * g.r_in)) * (hd(g.r_out * g.r_out) - rho2) * xp * yp * zeta * (hd(1.0) - zeta);
  } else {
    bubble = hsin((PI / g.lx) * x) * hsin((PI / g.ly) * y) * hsin((PI / g.lz) * z);
  }
  HDual mod = hd(1.0);
  for (int k = 0; k < f.n_modes; ++k)
    mod = mod + f.a[k] * hsin(f.b[k][0] * x + f.b[k][1] * y + f.b[k][2] * z + hd(f.c[k]));
  return bubble * mod;
}

__device__ inline double manufactured_value(const GeomParams &g, const RhsParams &f, double x, double y, double z) {
  return manufactured_u(g, f, hd(x), hd(y), hd(z)).a;
}

__device__ inline double source_term(const GeomParams &g, const RhsParams &f, double x, double y, double z) {
  if (!f.has) return 0.0;
  if (f.kind == TT_IGA_RHS_CONSTANT || f.kind == TT_IGA_RHS_RING_LOG) return f.value;
  double lap = 0.0;
  const double X[3] = {x, y, z};
  for (int k = 0; k < 3; ++k) {
    HDual a[3];
    for (int j = 0; j < 3; ++j) a[j] = (j == k) ? HDual{X[j], 1.0, 1.0, 0.0} : hd(X[j]);
    lap += manufactured_u(g, f, a[0], a[1], a[2]).d;
  }
  return -lap;
}

// Physical point and Jacobian J[a][b] = dx_a/dxi_b of the map at parametric xi.
// Nonzero B-spline functions N_{s-q..s} of degree q on a general knot vector t
// (span s: t[s] <= x < t[s+1], the last non-empty span for x = 1) and their first
// derivatives, by the Cox-de Boor triangle of Section 2.1: the row of degree q-1
// gives the derivatives, dN_i = q N_{i,q-1} / (t_{i+q} - t_i) - q N_{i+1,q-1} / (t_{i+q+1} - t_{i+1}).
__device__ inline int nurbs_span(const double *t, int q, int nc, double x) {
  if (x >= t[nc]) return nc - 1;
  int lo = q, hi = nc;  // t[lo] <= x < t[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (x < t[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

__device__ inline void nurbs_basis_ders(const double *t, int q, int s, double x, double N[TT_IGA_NURBS_MAX_DEGREE + 1],
                                        double D[TT_IGA_NURBS_MAX_DEGREE + 1]) {
  double left[TT_IGA_NURBS_MAX_DEGREE + 1], right[TT_IGA_NURBS_MAX_DEGREE + 1];
  double P[TT_IGA_NURBS_MAX_DEGREE + 1];  // degree j values on span s
  P[0] = 1.0;
  double Pm[TT_IGA_NURBS_MAX_DEGREE + 1];  // degree q-1 values
  for (int j = 1; j <= q; ++j) {
    if (j == q)
      for (int r = 0; r < q; ++r) Pm[r] = P[r];
    left[j] = x - t[s + 1 - j];
    right[j] = t[s + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      const double den = right[r + 1] + left[j - r];
      const double tmp = den != 0.0 ? P[r] / den : 0.0;
      P[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    P[j] = saved;
  }
  for (int r = 0; r <= q; ++r) N[r] = P[r];
  // derivative of function i = s - q + r from the degree q-1 functions i and i+1 (r-1 and r in Pm)
  for (int r = 0; r <= q; ++r) {
    const int i = s - q + r;
    double d = 0.0;
    if (r >= 1) {
      const double den = t[i + q] - t[i];
      if (den != 0.0) d += q * Pm[r - 1] / den;
    }
    if (r <= q - 1) {
      const double den = t[i + q + 1] - t[i + 1];
      if (den != 0.0) d -= q * Pm[r] / den;
    }
    D[r] = d;
  }
}

// x(xi) of a NURBS patch and its Jacobian: X = A / W, dX/dxi_d = (dA_d - X dW_d) / W with
// W = sum w N, A = sum w P N over the (q1+1)(q2+1)(q3+1) control points supporting xi.
__device__ inline void nurbs_map(const GeomParams &g, double x1, double x2, double x3, double X[3], double J[3][3]) {
  const double *t[3];
  t[0] = g.nurbs;
  t[1] = t[0] + g.nc[0] + g.nd[0] + 1;
  t[2] = t[1] + g.nc[1] + g.nd[1] + 1;
  const double *w = t[2] + g.nc[2] + g.nd[2] + 1;
  const double *P = w + g.nc[0] * g.nc[1] * g.nc[2];
  const double xs[3] = {fmin(fmax(x1, 0.0), 1.0), fmin(fmax(x2, 0.0), 1.0), fmin(fmax(x3, 0.0), 1.0)};
  double N[3][TT_IGA_NURBS_MAX_DEGREE + 1], D[3][TT_IGA_NURBS_MAX_DEGREE + 1];
  int s[3];
  for (int d = 0; d < 3; ++d) {
    s[d] = nurbs_span(t[d], g.nd[d], g.nc[d], xs[d]);
    nurbs_basis_ders(t[d], g.nd[d], s[d], xs[d], N[d], D[d]);
  }
  double W = 0.0, dW[3] = {0.0, 0.0, 0.0}, A[3] = {0.0, 0.0, 0.0}, dA[3][3] = {};
  for (int c = 0; c <= g.nd[2]; ++c) {
    const int i3 = s[2] - g.nd[2] + c;
    for (int b = 0; b <= g.nd[1]; ++b) {
      const int i2 = s[1] - g.nd[1] + b;
      for (int a = 0; a <= g.nd[0]; ++a) {
        const int i1 = s[0] - g.nd[0] + a;
        const long long idx = ((long long)i3 * g.nc[1] + i2) * g.nc[0] + i1;
        const double wi = w[idx];
        const double v = N[0][a] * N[1][b] * N[2][c];
        const double dv[3] = {D[0][a] * N[1][b] * N[2][c], N[0][a] * D[1][b] * N[2][c], N[0][a] * N[1][b] * D[2][c]};
        W += wi * v;
        for (int e = 0; e < 3; ++e) {
          const double pw = wi * P[3 * idx + e];
          A[e] += pw * v;
          for (int d = 0; d < 3; ++d) dA[e][d] += pw * dv[d];
        }
        for (int d = 0; d < 3; ++d) dW[d] += wi * dv[d];
      }
    }
  }
  for (int e = 0; e < 3; ++e) X[e] = A[e] / W;
  for (int e = 0; e < 3; ++e)
    for (int d = 0; d < 3; ++d) J[e][d] = (dA[e][d] - X[e] * dW[d]) / W;
}

__device__ inline void map_point(const GeomParams &g, double x1, double x2, double x3, double X[3], double J[3][3]) {
  if (g.kind == TT_IGA_GEOM_NURBS) {
    nurbs_map(g, x1, x2, x3, X, J);
    return;
  }
  if (g.kind == TT_IGA_GEOM_BOX) {
    X[0] = g.lx * x1; X[1] = g.ly * x2; X[2] = g.lz * x3;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) J[a][b] = 0.0;
    J[0][0] = g.lx; J[1][1] = g.ly; J[2][2] = g.lz;
    return;
  }
  const double PI = 3.141592653589793238462643383279502884;
  // radial degree-1 B-spline
  const double r = g.r_in * (1.0 - x1) + g.r_out * x1, dr = g.r_out - g.r_in;
  // quarter arc: rational quadratic with control (1,0), (1,1), (0,1), weights 1, sqrt(2)/2, 1
  const double w1 = 0.70710678118654752440;
  const double t = x2, u = 1.0 - t;
  const double B0 = u * u, B1 = 2.0 * t * u, B2 = t * t;
  const double dB0 = -2.0 * u, dB1 = 2.0 * (u - t), dB2 = 2.0 * t;
  const double W = B0 + w1 * B1 + B2, dW = dB0 + w1 * dB1 + dB2;
  const double nx = B0 + w1 * B1, ny = w1 * B1 + B2;
  const double dnx = dB0 + w1 * dB1, dny = w1 * dB1 + dB2;
  const double cx = nx / W, cy = ny / W;
  const double dcx = (dnx * W - nx * dW) / (W * W), dcy = (dny * W - ny * dW) / (W * W);
  // axial degree-1 B-spline
  const double z = g.height * x3, dz = g.height;
  const double zeta = z / g.height;
  const double phi = g.twist * zeta, dphi = g.twist / g.height;
  double sz, cz;
  sincos(PI * zeta, &sz, &cz);
  const double s = 1.0 + g.swell * sz, ds = g.swell * PI * cz / g.height;
  double sp, cp;
  sincos(phi, &sp, &cp);
  const double x0 = r * cx, y0 = r * cy;
  X[0] = s * (cp * x0 - sp * y0);
  X[1] = s * (sp * x0 + cp * y0);
  X[2] = z;
  const double ax[2] = {dr * cx, r * dcx}, ay[2] = {dr * cy, r * dcy};
  for (int b = 0; b < 2; ++b) {
    J[0][b] = s * (cp * ax[b] - sp * ay[b]);
    J[1][b] = s * (sp * ax[b] + cp * ay[b]);
    J[2][b] = 0.0;
  }
  J[0][2] = dz * (ds * (cp * x0 - sp * y0) + s * dphi * (-sp * x0 - cp * y0));
  J[1][2] = dz * (ds * (sp * x0 + cp * y0) + s * dphi * (cp * x0 - sp * y0));
  J[2][2] = dz;
}

// R = det J J^{-1} J^{-T}: with A = adj(J) = det J J^{-1}, R = A A^T / det J.
__device__ inline void point_outputs(const GeomParams &g, const RhsParams &f, double x1, double x2, double x3, double *o,
                              int *bad) {
  double X[3], J[3][3];
  map_point(g, x1, x2, x3, X, J);
  double A[3][3];
  A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
  if (!(det > 0.0)) *bad = 1;
  const double inv = 1.0 / det;
  double R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) R[a][b] = (A[a][0] * A[b][0] + A[a][1] * A[b][1] + A[a][2] * A[b][2]) * inv;
  o[0] = R[0][0]; o[1] = R[0][1]; o[2] = R[0][2];
  o[3] = R[1][1]; o[4] = R[1][2]; o[5] = R[2][2];
  o[6] = det;
  o[7] = f.has ? source_term(g, f, X[0], X[1], X[2]) * det : 0.0;
}

// Cross components beyond the eight point outputs: kFaceComp0 + 2 d + side is the area
// density |dx/dxi_e x dx/dxi_f| of the face xi_d = side (e < f its tangential directions),
// the surface measure of a face integral.  It is evaluated with xi_d replaced by side, so as
// a field on the volume grid it does not vary along direction d.

__device__ inline double face_area_density(const GeomParams &g, int face, double x1, double x2, double x3, int *bad) {
  const int d = face >> 1;
  const double side = (double)(face & 1);
  double X[3], J[3][3];
  map_point(g, d == 0 ? side : x1, d == 1 ? side : x2, d == 2 ? side : x3, X, J);
  const int e = d == 0 ? 1 : 0, h = d == 2 ? 1 : 2;
  const double c0 = J[1][e] * J[2][h] - J[2][e] * J[1][h];
  const double c1 = J[2][e] * J[0][h] - J[0][e] * J[2][h];
  const double c2 = J[0][e] * J[1][h] - J[1][e] * J[0][h];
  const double a = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  if (!(a > 0.0)) *bad = 1;
  return a;
}

// One cross component at a point (0..7: point_outputs, 8..13: face area densities).
__device__ inline double field_value(const GeomParams &g, const RhsParams &f, int comp, double x1, double x2,
                                     double x3, int *bad) {
  if (comp >= kFaceComp0) return face_area_density(g, comp - kFaceComp0, x1, x2, x3, bad);
  double o[8];
  point_outputs(g, f, x1, x2, x3, o, bad);
  return o[comp];
}


}  // namespace ttiga
