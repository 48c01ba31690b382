// Order-3 TT operations: block sums, rounding by QR + SVD (FP64), point
// evaluation and densification.
#include <algorithm>
#include <cmath>
#include <vector>

#include "linalg.cuh"

#include "tt.cuh"

namespace ttiga {

__global__ void k_transpose(const double *__restrict__ in, double *__restrict__ out, long long rows, long long cols) {
  __shared__ double tile[32][33];
  const long long bx = blockIdx.x * 32LL, by = blockIdx.y * 32LL;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const long long r = by + k, cc = bx + threadIdx.x;
    if (r < rows && cc < cols) tile[k][threadIdx.x] = in[r * cols + cc];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const long long r = bx + k, cc = by + threadIdx.x;  // out is cols x rows
    if (r < cols && cc < rows) out[r * rows + cc] = tile[threadIdx.x][k];
  }
}

void transpose(Ctx *c, const double *in, double *out, long long rows, long long cols) {
  if (rows <= 0 || cols <= 0) return;
  long long gx = (cols + 31) / 32, gy = (rows + 31) / 32;
  TTI_CHECK_ARG(gy <= 65535, "transpose: too many rows (%lld)", rows);
  k_transpose<<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, c->stream>>>(in, out, rows, cols);
  TTI_LAUNCH();
}

// dst[RA][m][RB] block (oa.., ob..) = s * src[ra][m][rb]
__global__ void k_embed(double *dst, int RA, int m, int RB, const double *src, int ra, int rb, int oa, int ob, double s) {
  const long long tot = (long long)ra * m * rb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long b = e % rb, t = e / rb;
    const long long i = t % m, a = t / m;
    dst[((a + oa) * m + i) * RB + b + ob] = s * src[e];
  }
}

static void embed(Ctx *c, double *dst, int RA, int m, int RB, const double *src, int ra, int rb, int oa, int ob,
                  double s) {
  long long tot = (long long)ra * m * rb;
  if (tot <= 0) return;
  k_embed<<<grid1d(tot, 256), 256, 0, c->stream>>>(dst, RA, m, RB, src, ra, rb, oa, ob, s);
  TTI_LAUNCH();
}

void tt_copy(Ctx *c, const TT3 &x, TT3 &y) {
  for (int k = 0; k < 3; ++k) y.m[k] = x.m[k];
  for (int k = 0; k < 4; ++k) y.r[k] = x.r[k];
  y.alloc(c);
  for (int k = 0; k < 3; ++k)
    TTI_CUDA(cudaMemcpyAsync(y.core[k].get(), x.core[k].get(), x.core_elems(k) * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
}

void tt_sum(Ctx *c, const TT3 &x, double a, const TT3 &y, double b, TT3 &out) {
  for (int k = 0; k < 3; ++k) TTI_CHECK_ARG(x.m[k] == y.m[k], "tt_sum: mode sizes differ");
  TT3 o;
  for (int k = 0; k < 3; ++k) o.m[k] = x.m[k];
  o.r[0] = 1; o.r[3] = 1;
  o.r[1] = x.r[1] + y.r[1];
  o.r[2] = x.r[2] + y.r[2];
  o.alloc(c);
  for (int k = 0; k < 3; ++k) c->zero(o.core[k].get(), o.core_elems(k) * sizeof(double));
  embed(c, o.core[0].d(), 1, o.m[0], o.r[1], x.core[0].d(), 1, x.r[1], 0, 0, a);
  embed(c, o.core[0].d(), 1, o.m[0], o.r[1], y.core[0].d(), 1, y.r[1], 0, x.r[1], b);
  embed(c, o.core[1].d(), o.r[1], o.m[1], o.r[2], x.core[1].d(), x.r[1], x.r[2], 0, 0, 1.0);
  embed(c, o.core[1].d(), o.r[1], o.m[1], o.r[2], y.core[1].d(), y.r[1], y.r[2], x.r[1], x.r[2], 1.0);
  embed(c, o.core[2].d(), o.r[2], o.m[2], 1, x.core[2].d(), x.r[2], 1, 0, 0, 1.0);
  embed(c, o.core[2].d(), o.r[2], o.m[2], 1, y.core[2].d(), y.r[2], 1, x.r[2], 0, 1.0);
  out = std::move(o);
}

void tt_sum_many(Ctx *c, const std::vector<const TT3 *> &xs, TT3 &out) {
  TTI_CHECK_ARG(!xs.empty(), "tt_sum_many: no terms");
  TT3 o;
  for (int k = 0; k < 3; ++k) o.m[k] = xs[0]->m[k];
  o.r[0] = 1;
  o.r[3] = 1;
  o.r[1] = o.r[2] = 0;
  for (const TT3 *x : xs) {
    for (int k = 0; k < 3; ++k) TTI_CHECK_ARG(x->m[k] == o.m[k], "tt_sum_many: mode sizes differ");
    o.r[1] += x->r[1];
    o.r[2] += x->r[2];
  }
  o.alloc(c);
  for (int k = 0; k < 3; ++k) c->zero(o.core[k].get(), o.core_elems(k) * sizeof(double));
  int off1 = 0, off2 = 0;
  for (const TT3 *x : xs) {
    embed(c, o.core[0].d(), 1, o.m[0], o.r[1], x->core[0].d(), 1, x->r[1], 0, off1, 1.0);
    embed(c, o.core[1].d(), o.r[1], o.m[1], o.r[2], x->core[1].d(), x->r[1], x->r[2], off1, off2, 1.0);
    embed(c, o.core[2].d(), o.r[2], o.m[2], 1, x->core[2].d(), x->r[2], 1, off2, 0, 1.0);
    off1 += x->r[1];
    off2 += x->r[2];
  }
  out = std::move(o);
}

// W[j][l] = S[j] * V[l][j] for j < r (rows of diag(S) V^T)
__global__ void k_svt(const double *S, const double *V, int k, int r, double *W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * k; e += gridDim.x * blockDim.x) {
    const int j = e / k, l = e % k;
    W[e] = S[j] * V[(long long)l * k + j];
  }
}

void svt(Ctx *c, const double *S, const double *V, int k, int r, double *W) {
  if (r <= 0 || k <= 0) return;
  k_svt<<<grid1d((long long)r * k, 256), 256, 0, c->stream>>>(S, V, k, r, W);
  TTI_LAUNCH();
}

// Orthogonalise core k (k = 2 or 1, 0-based 2 / 1) from the right: core_k = L Q
// with Q orthonormal rows; L merged into core_{k-1}.
void orth_right_step(Ctx *c, TT3 &x, int k) {
  const int ra = x.r[k], m = x.m[k], rb = x.r[k + 1];
  const long long cols = (long long)m * rb;
  DBuf T(c, (size_t)cols * ra * sizeof(double)), Qt(c, (size_t)cols * ra * sizeof(double)),
      R(c, (size_t)ra * ra * sizeof(double));
  transpose(c, x.core[k].d(), T.d(), ra, cols);           // (m rb) x ra
  qr(c, (int)cols, ra, T.d(), ra, Qt.d(), R.d());          // T = Q R
  transpose(c, Qt.d(), x.core[k].d(), cols, ra);          // core_k = Q^T (ra x m rb)
  // core_{k-1} <- core_{k-1} R^T : ((r_{k-1} m_{k-1}) x ra) (ra x ra)
  const int rows = x.r[k - 1] * x.m[k - 1];
  DBuf out(c, (size_t)rows * ra * sizeof(double));
  gemm<double>(c, false, true, rows, ra, ra, 1.0, x.core[k - 1].d(), ra, 0, R.d(), ra, 0, 0.0, out.d(), ra, 0, 1);
  x.core[k - 1] = std::move(out);
}

double tt_orth_rl(Ctx *c, TT3 &x) {
  orth_right_step(c, x, 2);
  orth_right_step(c, x, 1);
  return host_nrm2(c, x.core[0].d(), (long long)x.core_elems(0));
}

// ||X||_F by a right-to-left sweep of R factors only: core 3 = L3 Q3 (R of the
// transposed core), core 2 <- core 2 L3, core 2 = L2 Q2, core 1 <- core 1 L2,
// ||X|| = ||core 1||.  The orthogonal factors are never formed.
double tt_norm(Ctx *c, const TT3 &x) {
  const int m1 = x.m[0], m2 = x.m[1], m3 = x.m[2], r1 = x.r[1], r2 = x.r[2];
  // core 3 is r2 x m3: QR of its transpose (m3 x r2) gives R3; core 3 = R3^T Q3^T
  DBuf T3(c, (size_t)m3 * r2 * sizeof(double)), R3(c, (size_t)r2 * r2 * sizeof(double));
  transpose(c, x.core[2].d(), T3.d(), r2, m3);
  qr(c, m3, r2, T3.d(), r2, nullptr, R3.d());
  // core 2 (r1 m2 x r2) times R3^T
  DBuf C2(c, (size_t)r1 * m2 * r2 * sizeof(double));
  gemm<double>(c, false, true, r1 * m2, r2, r2, 1.0, x.core[1].d(), r2, 0, R3.d(), r2, 0, 0.0, C2.d(), r2, 0, 1);
  DBuf T2(c, (size_t)m2 * r2 * r1 * sizeof(double)), R2(c, (size_t)r1 * r1 * sizeof(double));
  transpose(c, C2.d(), T2.d(), r1, (long long)m2 * r2);
  qr(c, m2 * r2, r1, T2.d(), r1, nullptr, R2.d());
  DBuf C1(c, (size_t)m1 * r1 * sizeof(double));
  gemm<double>(c, false, true, m1, r1, r1, 1.0, x.core[0].d(), r1, 0, R2.d(), r1, 0, 0.0, C1.d(), r1, 0, 1);
  return host_nrm2(c, C1.d(), (long long)m1 * r1);
}

// Left-to-right truncation step at core k (0 or 1) with absolute threshold delta.
// Returns the retained rank; fills sv with the singular values when requested.
static int trunc_left_step(Ctx *c, TT3 &x, int k, double delta_or_eps, bool delta_is_rel, int max_rank,
                           double *norm_out) {
  const int ra = x.r[k], m = x.m[k], rb = x.r[k + 1];
  const int rows = ra * m;
  DBuf Q(c, (size_t)rows * rb * sizeof(double)), R(c, (size_t)rb * rb * sizeof(double));
  qr(c, rows, rb, x.core[k].d(), rb, Q.d(), R.d());
  DBuf U(c, (size_t)rb * rb * sizeof(double)), S(c, (size_t)rb * sizeof(double)), V(c, (size_t)rb * rb * sizeof(double));
  svd_small(c, rb, R.d(), U.d(), S.d(), V.d());
  std::vector<double> s(rb);
  c->d2h(s.data(), S.d(), rb * sizeof(double));
  double nrm2 = 0.0;
  for (double v : s) nrm2 += v * v;
  if (norm_out) *norm_out = sqrt(nrm2);
  const double delta = delta_is_rel ? delta_or_eps * sqrt(nrm2) / sqrt(2.0) : delta_or_eps;
  // smallest r with ||s[r:]|| <= delta
  int r = rb;
  double tail = 0.0;
  while (r > 1) {
    const double t = tail + s[r - 1] * s[r - 1];
    if (sqrt(t) > delta) break;
    tail = t;
    --r;
  }
  if (max_rank > 0 && r > max_rank) r = max_rank;
  // core_k <- Q U[:, :r]
  DBuf nk(c, (size_t)rows * r * sizeof(double));
  gemm<double>(c, false, false, rows, r, rb, 1.0, Q.d(), rb, 0, U.d(), rb, 0, 0.0, nk.d(), r, 0, 1);
  // core_{k+1} <- (diag(S) V^T)[:r] core_{k+1}
  DBuf W(c, (size_t)r * rb * sizeof(double));
  k_svt<<<grid1d((long long)r * rb, 256), 256, 0, c->stream>>>(S.d(), V.d(), rb, r, W.d());
  TTI_LAUNCH();
  const long long cols = (long long)x.m[k + 1] * x.r[k + 2];
  DBuf nn(c, (size_t)r * cols * sizeof(double));
  gemm<double>(c, false, false, r, (int)cols, rb, 1.0, W.d(), rb, 0, x.core[k + 1].d(), cols, 0, 0.0, nn.d(), cols, 0, 1);
  x.core[k] = std::move(nk);
  x.core[k + 1] = std::move(nn);
  x.r[k + 1] = r;
  return r;
}

double tt_round(Ctx *c, TT3 &x, double eps, int max_rank) {
  tt_orth_rl(c, x);
  double nrm = 0.0;
  // The first SVD sees the whole norm; delta = eps ||X|| / sqrt(d - 1) with d = 3.
  trunc_left_step(c, x, 0, eps, true, max_rank, &nrm);
  const double delta = eps * nrm / sqrt(2.0);
  trunc_left_step(c, x, 1, delta, false, max_rank, nullptr);
  return nrm;
}

__global__ void k_tt_eval(const double *G1, const double *G2, const double *G3, int m1, int m2, int m3, int r1, int r2,
                          int m, const int *idx, double *out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    const int i1 = idx[3 * t], i2 = idx[3 * t + 1], i3 = idx[3 * t + 2];
    double v = 0.0;
    for (int a = 0; a < r1; ++a) {
      const double g1 = G1[(long long)i1 * r1 + a];
      if (g1 == 0.0) continue;
      double s = 0.0;
      const double *g2 = G2 + ((long long)a * m2 + i2) * r2;
      for (int b = 0; b < r2; ++b) s += g2[b] * G3[(long long)b * m3 + i3];
      v += g1 * s;
    }
    out[t] = v;
  }
}

void tt_eval_points(Ctx *c, const TT3 &x, int m, const int *idx, double *out) {
  if (m <= 0) return;
  k_tt_eval<<<grid1d(m, 128), 128, 0, c->stream>>>(x.core[0].d(), x.core[1].d(), x.core[2].d(), x.m[0], x.m[1],
                                                   x.m[2], x.r[1], x.r[2], m, idx, out);
  TTI_LAUNCH();
}

__global__ void k_tt_full(const double *G1, const double *G2, const double *G3, int m1, int m2, int m3, int r1, int r2,
                          double *out) {
  const long long tot = (long long)m1 * m2 * m3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(e % m1);
    const int i2 = (int)((e / m1) % m2);
    const int i3 = (int)(e / ((long long)m1 * m2));
    double v = 0.0;
    for (int a = 0; a < r1; ++a) {
      double s = 0.0;
      for (int b = 0; b < r2; ++b) s += G2[((long long)a * m2 + i2) * r2 + b] * G3[(long long)b * m3 + i3];
      v += G1[(long long)i1 * r1 + a] * s;
    }
    out[e] = v;
  }
}

void tt_dense(Ctx *c, const TT3 &x, double *out) {
  // T[i1][(i2, b)] = G1[i1][a] G2[a][(i2, b)];  out[(i1, i2)][i3] = T[(i1, i2)][b] G3[b][i3]
  const int m1 = x.m[0], m2 = x.m[1], m3 = x.m[2], r1 = x.r[1], r2 = x.r[2];
  DBuf T(c, (size_t)m1 * m2 * r2 * sizeof(double));
  gemm<double>(c, false, false, m1, m2 * r2, r1, 1.0, x.core[0].d(), r1, 0, x.core[1].d(), (long long)m2 * r2, 0, 0.0,
               T.d(), (long long)m2 * r2, 0, 1);
  gemm<double>(c, false, false, m1 * m2, m3, r2, 1.0, T.d(), r2, 0, x.core[2].d(), m3, 0, 0.0, out, m3, 0, 1);
}

void tt_full(Ctx *c, const TT3 &x, double *out) {
  long long tot = (long long)x.m[0] * x.m[1] * x.m[2];
  k_tt_full<<<grid1d(tot, 256), 256, 0, c->stream>>>(x.core[0].d(), x.core[1].d(), x.core[2].d(), x.m[0], x.m[1],
                                                     x.m[2], x.r[1], x.r[2], out);
  TTI_LAUNCH();
}

}  // namespace ttiga
