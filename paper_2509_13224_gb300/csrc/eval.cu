// Evaluation of the TT solution u_h(xi) = sum_a u_a N_a(xi) and the relative
// L2 error of Eq. (L2norm), read as sqrt(int (u_h - u)^2) / sqrt(int u^2) over
// the mapped domain with p+3 Gauss points per element and direction.
#include <algorithm>

#include "eval.cuh"
#include "geom_device.cuh"
#include "linalg.cuh"

namespace ttiga {

// u_h at parametric points: the p+1 nonzero functions per direction, interior
// functions 1..n-2 map to restricted TT index a-1.
__global__ void k_eval_points(const double *__restrict__ U1, const double *__restrict__ U2,
                              const double *__restrict__ U3, int n1, int n2, int n3, int p, int r1, int r2, int m,
                              const double *__restrict__ xi, double *__restrict__ out) {
  const int nf[3] = {n1, n2, n3};
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
    const int m1 = n1 - 2, m2 = n2 - 2, m3 = n3 - 2;
    double v = 0.0;
    for (int a = 0; a < r1; ++a) {
      double v1 = 0.0;
      for (int k = 0; k <= p; ++k) {
        const int g = e[0] + k - 1;
        if (g >= 0 && g < m1) v1 += Nv[0][k] * U1[(long long)g * r1 + a];
      }
      if (v1 == 0.0) continue;
      double s = 0.0;
      for (int b = 0; b < r2; ++b) {
        double v2 = 0.0, v3 = 0.0;
        for (int k = 0; k <= p; ++k) {
          const int g2 = e[1] + k - 1, g3 = e[2] + k - 1;
          if (g2 >= 0 && g2 < m2) v2 += Nv[1][k] * U2[((long long)a * m2 + g2) * r2 + b];
          if (g3 >= 0 && g3 < m3) v3 += Nv[2][k] * U3[(long long)b * m3 + g3];
        }
        s += v2 * v3;
      }
      v += v1 * s;
    }
    out[t] = v;
  }
}

void eval_points(Ctx *c, const tt_iga_solution *u, int m, const double *xi, double *out) {
  if (m <= 0) return;
  k_eval_points<<<grid1d(m, 128), 128, 0, c->stream>>>(u->u.core[0].d(), u->u.core[1].d(), u->u.core[2].d(),
                                                       u->n[0] + 2, u->n[1] + 2, u->n[2] + 2, u->p, u->u.r[1],
                                                       u->u.r[2], m, xi, out);
  TTI_LAUNCH();
}

// T[q][a][b] = sum_k N[q][k] U[a][e(q)+k-1][b] over interior functions (restricted core U[ra][n-2][rb]).
__global__ void k_core_table(const double *__restrict__ N, int Q, int nq, int n, int p, const double *__restrict__ U,
                             int ra, int rb, double *__restrict__ T) {
  const long long tot = (long long)Q * ra * rb;
  const int m = n - 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % rb);
    const long long t = e / rb;
    const int a = (int)(t % ra);
    const int q = (int)(t / ra);
    const int el = q / nq;
    double s = 0.0;
    for (int k = 0; k <= p; ++k) {
      const int g = el + k - 1;
      if (g >= 0 && g < m) s += N[(long long)q * (p + 1) + k] * U[((long long)a * m + g) * rb + b];
    }
    T[e] = s;
  }
}

__global__ void k_l2_accumulate(GeomParams g, RhsParams f, const double *__restrict__ x1, const double *__restrict__ x2,
                                const double *__restrict__ x3, const double *__restrict__ w1,
                                const double *__restrict__ w2, const double *__restrict__ w3, int Q1, int Q2, int Q3,
                                const double *__restrict__ T1, const double *__restrict__ T2,
                                const double *__restrict__ T3, int r1, int r2, double *part) {
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
    double X[3], J[3][3];
    map_point(g, x1[q1], x2[q2], x3[q3], X, J);
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double ue = manufactured_value(g, f, X[0], X[1], X[2]);
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

double l2_error(Ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_rhs_desc *rhs) {
  const int p = u->p;
  Space fine[3];
  DBuf T[3];
  for (int d = 0; d < 3; ++d) {
    build_space(c, fine[d], u->n[d] + 2, p, std::min(p + 3, 8));
    const int ra = u->u.r[d], rb = u->u.r[d + 1];
    T[d] = DBuf(c, (size_t)fine[d].Q * ra * rb * sizeof(double));
    const long long tot = (long long)fine[d].Q * ra * rb;
    k_core_table<<<grid1d(tot, 256), 256, 0, c->stream>>>(fine[d].N.d(), fine[d].Q, fine[d].nq, u->n[d] + 2, p,
                                                          u->u.core[d].d(), ra, rb, T[d].d());
    TTI_LAUNCH();
  }
  RhsParams rp = rhs_params(rhs);
  const int nb = 152 * 8;
  DBuf part(c, 2 * nb * sizeof(double));
  k_l2_accumulate<<<nb, 256, 0, c->stream>>>(g->gp, rp, fine[0].pts.d(), fine[1].pts.d(), fine[2].pts.d(),
                                             fine[0].wts.d(), fine[1].wts.d(), fine[2].wts.d(), fine[0].Q, fine[1].Q,
                                             fine[2].Q, T[0].d(), T[1].d(), T[2].d(), u->u.r[1], u->u.r[2], part.d());
  TTI_LAUNCH();
  std::vector<double> h(2 * nb);
  c->d2h(h.data(), part.d(), h.size() * sizeof(double));
  double num = 0.0, den = 0.0;
  for (int i = 0; i < nb; ++i) { num += h[2 * i]; den += h[2 * i + 1]; }
  return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

}  // namespace ttiga
