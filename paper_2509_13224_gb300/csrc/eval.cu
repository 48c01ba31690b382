// Evaluation of the TT solution u_h(xi) = sum_a u_a N_a(xi) (plus the lift of
// the Dirichlet data, Section 4.3) and the relative L2 error of Eq. (L2norm),
// read as sqrt(int (u_h - u)^2) / sqrt(int u^2) over the mapped domain with p+3
// Gauss points per element and direction.
#include <algorithm>

#include "amen_ops.cuh"
#include "eval.cuh"
#include "geom_device.cuh"
#include "linalg.cuh"
#include "tt.cuh"

namespace ttiga {

// Where the unknowns sit among the basis functions and the lift of the Dirichlet data.
struct EvalLayout {
  int nfull[3], lo[3], m[3];
  int lift_dir;
  double lift_lo, lift_hi;
};

static EvalLayout eval_layout(const tt_iga_solution *u) {
  EvalLayout L;
  for (int d = 0; d < 3; ++d) {
    L.nfull[d] = u->bl.nfull[d];
    L.lo[d] = u->bl.lo[d];
    L.m[d] = u->n[d];
  }
  L.lift_dir = u->bl.lift_dir;
  L.lift_lo = u->bl.lift_lo;
  L.lift_hi = u->bl.lift_hi;
  return L;
}

// u_h at parametric points: the p+1 nonzero functions per direction; function a
// of direction d is restricted TT index a - lo_d when it is an unknown; the lift
// lift_lo N_0 + lift_hi N_{n-1} of the lift direction is added.
__global__ void k_eval_points(const double *__restrict__ U1, const double *__restrict__ U2,
                              const double *__restrict__ U3, EvalLayout L, int p, int r1, int r2, int m,
                              const double *__restrict__ xi, double *__restrict__ out) {
  const int *nf = L.nfull;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    double Nv[3][9], Dv[9];
    int e[3];
    for (int d = 0; d < 3; ++d) {
      const int ne = nf[d] - p;
      double x = xi[3 * t + d];
      x = fmin(fmax(x, 0.0), 1.0);
      int el = (int)floor(x * ne);
      el = min(max(el, 0), ne - 1);
      e[d] = el;
      local_basis(x, el + p, nf[d], p, Nv[d], Dv);
    }
    const int m1 = L.m[0], m2 = L.m[1], m3 = L.m[2];
    double v = 0.0;
    for (int a = 0; a < r1; ++a) {
      double v1 = 0.0;
      for (int k = 0; k <= p; ++k) {
        const int g = e[0] + k - L.lo[0];
        if (g >= 0 && g < m1) v1 += Nv[0][k] * U1[(long long)g * r1 + a];
      }
      if (v1 == 0.0) continue;
      double s = 0.0;
      for (int b = 0; b < r2; ++b) {
        double v2 = 0.0, v3 = 0.0;
        for (int k = 0; k <= p; ++k) {
          const int g2 = e[1] + k - L.lo[1], g3 = e[2] + k - L.lo[2];
          if (g2 >= 0 && g2 < m2) v2 += Nv[1][k] * U2[((long long)a * m2 + g2) * r2 + b];
          if (g3 >= 0 && g3 < m3) v3 += Nv[2][k] * U3[(long long)b * m3 + g3];
        }
        s += v2 * v3;
      }
      v += v1 * s;
    }
    if (L.lift_dir >= 0) {
      const int d = L.lift_dir, ne = nf[d] - p;
      if (e[d] == 0) v += L.lift_lo * Nv[d][0];
      if (e[d] == ne - 1) v += L.lift_hi * Nv[d][p];
    }
    out[t] = v;
  }
}

void eval_points(Ctx *c, const tt_iga_solution *u, int m, const double *xi, double *out) {
  if (m <= 0) return;
  k_eval_points<<<grid1d(m, 128), 128, 0, c->stream>>>(u->u.core[0].d(), u->u.core[1].d(), u->u.core[2].d(),
                                                       eval_layout(u), u->p, u->u.r[1], u->u.r[2], m, xi, out);
  TTI_LAUNCH();
}

// T[q][a][b] = sum_k N[q][k] U[a][e(q)+k-lo][b] over the unknown functions (restricted core U[ra][m][rb]).
__global__ void k_core_table(const double *__restrict__ N, int Q, int nq, int lo, int m, int p,
                             const double *__restrict__ U, int ra, int rb, double *__restrict__ T) {
  const long long tot = (long long)Q * ra * rb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % rb);
    const long long t = e / rb;
    const int a = (int)(t % ra);
    const int q = (int)(t / ra);
    const int el = q / nq;
    double s = 0.0;
    for (int k = 0; k <= p; ++k) {
      const int g = el + k - lo;
      if (g >= 0 && g < m) s += N[(long long)q * (p + 1) + k] * U[((long long)a * m + g) * rb + b];
    }
    T[e] = s;
  }
}

// Lift at the points of the lift direction: lift_lo N_0 (first element) + lift_hi N_{n-1} (last element).
__global__ void k_lift_table(const double *__restrict__ N, int Q, int nq, int ne, int p, double lift_lo,
                             double lift_hi, double *__restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    const int el = q / nq;
    double v = 0.0;
    if (el == 0) v += lift_lo * N[(long long)q * (p + 1)];
    if (el == ne - 1) v += lift_hi * N[(long long)q * (p + 1) + p];
    out[q] = v;
  }
}

__global__ void k_l2_accumulate(GeomParams g, RhsParams f, const double *__restrict__ x1, const double *__restrict__ x2,
                                const double *__restrict__ x3, const double *__restrict__ w1,
                                const double *__restrict__ w2, const double *__restrict__ w3, int Q1, int Q2, int Q3,
                                const double *__restrict__ T1, const double *__restrict__ T2,
                                const double *__restrict__ T3, int r1, int r2, int lift_dir,
                                const double *__restrict__ liftq, double ring_a, double ring_b, double *part) {
  __shared__ double red[2][32];
  double num = 0.0, den = 0.0;
  const long long tot = (long long)Q1 * Q2 * Q3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int q1 = (int)(e % Q1);
    const int q2 = (int)((e / Q1) % Q2);
    const int q3 = (int)(e / ((long long)Q1 * Q2));
    double uh = 0.0;
    for (int a = 0; a < r1; ++a) {
      const double t1 = T1[(long long)q1 * r1 + a];
      double s = 0.0;
      for (int b = 0; b < r2; ++b) s += T2[((long long)q2 * r1 + a) * r2 + b] * T3[(long long)q3 * r2 + b];
      uh += t1 * s;
    }
    if (lift_dir >= 0) uh += liftq[lift_dir == 0 ? q1 : (lift_dir == 1 ? q2 : q3)];
    double X[3], J[3][3];
    map_point(g, x1[q1], x2[q2], x3[q3], X, J);
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    // RING_LOG: the radial solution A + B ln(rho / r_in) of the ring problem (annulus without twist and swell)
    const double ue = (f.kind == TT_IGA_RHS_RING_LOG)
                          ? ring_a + ring_b * log(sqrt(X[0] * X[0] + X[1] * X[1]) / g.r_in)
                          : manufactured_value(g, f, X[0], X[1], X[2]);
    const double w = w1[q1] * w2[q2] * w3[q3] * det;
    num += w * (uh - ue) * (uh - ue);
    den += w * ue * ue;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// Coefficients of the ring problem's exact solution u = A + B ln(rho / r_in) from the radial faces'
// data: a value fixes A + B ln(rho / r_in) there, an outward flux q fixes du/dn = B / r_out
// (outer face) or -B / r_in (inner face, outward normal -rho).
static void ring_solution(const tt_iga_geom *g, const BoundaryLayout &bl, double *A, double *B) {
  const double L = log(g->desc.r_out / g->desc.r_in);
  const double v_in = bl.lift_dir == 0 ? bl.lift_lo : 0.0, v_out = bl.lift_dir == 0 ? bl.lift_hi : 0.0;
  if (bl.lo[0] && bl.hi[0]) {
    *A = v_in;
    *B = (v_out - v_in) / L;
  } else if (bl.lo[0]) {
    *A = v_in;
    *B = bl.flux[1] * g->desc.r_out;
  } else {
    *B = -bl.flux[0] * g->desc.r_in;
    *A = v_out - *B * L;
  }
}

double l2_error(Ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_rhs_desc *rhs) {
  const int p = u->p;
  double ring_a = 0.0, ring_b = 0.0;
  if (rhs->kind == TT_IGA_RHS_RING_LOG) ring_solution(g, u->bl, &ring_a, &ring_b);
  Space fine[3];
  DBuf T[3];
  for (int d = 0; d < 3; ++d) {
    build_space(c, fine[d], u->bl.nfull[d], p, std::min(p + 3, 8));
    const int ra = u->u.r[d], rb = u->u.r[d + 1];
    T[d] = DBuf(c, (size_t)fine[d].Q * ra * rb * sizeof(double));
    const long long tot = (long long)fine[d].Q * ra * rb;
    k_core_table<<<grid1d(tot, 256), 256, 0, c->stream>>>(fine[d].N.d(), fine[d].Q, fine[d].nq, u->bl.lo[d], u->n[d],
                                                          p, u->u.core[d].d(), ra, rb, T[d].d());
    TTI_LAUNCH();
  }
  const int ld = u->bl.lift_dir;
  DBuf liftq(c, ld >= 0 ? (size_t)fine[ld].Q * sizeof(double) : 16);
  if (ld >= 0) {
    k_lift_table<<<grid1d(fine[ld].Q, 128), 128, 0, c->stream>>>(fine[ld].N.d(), fine[ld].Q, fine[ld].nq,
                                                                 fine[ld].ne, p, u->bl.lift_lo, u->bl.lift_hi,
                                                                 liftq.d());
    TTI_LAUNCH();
  }
  RhsParams rp = rhs_params(rhs);
  const int nb = 152 * 8;
  DBuf part(c, 2 * nb * sizeof(double));
  k_l2_accumulate<<<nb, 256, 0, c->stream>>>(g->gp, rp, fine[0].pts.d(), fine[1].pts.d(), fine[2].pts.d(),
                                             fine[0].wts.d(), fine[1].wts.d(), fine[2].wts.d(), fine[0].Q, fine[1].Q,
                                             fine[2].Q, T[0].d(), T[1].d(), T[2].d(), u->u.r[1], u->u.r[2], ld,
                                             liftq.d(), ring_a, ring_b, part.d());
  TTI_LAUNCH();
  std::vector<double> h(2 * nb);
  c->d2h(h.data(), part.d(), h.size() * sizeof(double));
  double num = 0.0, den = 0.0;
  for (int i = 0; i < nb; ++i) { num += h[2 * i]; den += h[2 * i + 1]; }
  return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

// w^T M w of a TT vector w and a band TT-matrix M by the left interface
// recursion of the AMEn contractions (PhiL of a 1 x 1 x 1 start, three cores).
static double quadratic_form(Ctx *c, const TT3 &M, const int n[3], int p, const TT3 &w) {
  Work<double> wk{c};
  DBuf phi(c, sizeof(double));
  const double one = 1.0;
  c->h2d(phi.get(), &one, sizeof one);
  for (int k = 0; k < 3; ++k) {
    BandCore A{M.core[k].d(), nullptr, M.r[k], n[k], 2 * p + 1, p, M.r[k + 1]};
    DBuf next(c, (size_t)w.r[k + 1] * M.r[k + 1] * w.r[k + 1] * sizeof(double));
    left_update(c, wk, w.core[k].d(), w.r[k], w.r[k + 1], phi.d(), A, w.core[k].d(), w.r[k], w.r[k + 1], next.d());
    phi = std::move(next);
  }
  double v = 0.0;
  c->d2h(&v, phi.get(), sizeof v);
  return v;
}

double l2_diff(Ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_solution *v) {
  TT3 M;
  mass_matrix(c, g, v->bl, M);
  // w = u - v, rounded first: the rounding's orthogonalisation resolves the difference of two
  // nearly equal TTs to FP64 accuracy relative to ||u||, so the quadratic form of w carries no
  // cancellation between the two solutions
  TT3 w;
  tt_sum(c, u->u, 1.0, v->u, -1.0, w);
  const double wn = tt_round(c, w, 1e-13, 0);
  const double den = quadratic_form(c, M, v->n, v->p, v->u);
  if (!(wn > 0.0)) return 0.0;
  const double num = quadratic_form(c, M, v->n, v->p, w);
  if (!(den > 0.0)) return -1.0;
  return sqrt(std::max(num, 0.0) / den);
}

}  // namespace ttiga
