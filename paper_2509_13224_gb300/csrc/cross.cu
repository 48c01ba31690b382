// Rank-adaptive TT-cross for order-3 fields sampled on the tensor Gauss grid.
//
// The paper builds the coefficient TT cores with TT-Toolbox's amen_cross
// (Section 4.1.2): maxvol-guided sampling of the function at selected
// multi-indices to a tolerance eps.  This is a GPU formulation of the same
// idea for d = 3, one mode at a time:
//   1. mode 1: sample k random fibres A(:, j2, j3); the truncated SVD (QR +
//      Jacobi SVD) of the Q1 x k fibre matrix gives the column basis U1 and
//      rank r1; maxvol picks r1 rows I1 and the interpolation core
//      G1 = U1 U1[I1]^{-1};
//   2. mode 2: sample the (r1 Q2) x k matrix A(I1, :, j3) over random j3,
//      truncate, maxvol -> rows I2 of (alpha, i2) and G2 = U2 U2[I2]^{-1};
//   3. mode 3: G3 = A(I2, :) evaluated on all Q3 points;
//   4. validate max |TT - f| on random points; if the sampled ranks saturate
//      or the check fails, double the number of fibres and repeat.
// Every sample is an FP64 evaluation of the exact geometry (Section 3.3).
#include <algorithm>
#include <cmath>
#include <unordered_set>

#include "cross.cuh"
#include "geom_device.cuh"
#include "linalg.cuh"
#include "tt.cuh"

namespace ttiga {

namespace {

struct SplitMix {
  uint64_t s;
  explicit SplitMix(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  long long below(long long n) { return (long long)(next() % (uint64_t)n); }
};

// k distinct integers from [0, n) (all of them, shuffled, when k >= n)
std::vector<long long> distinct(SplitMix &rng, long long n, int k, const std::vector<long long> &keep) {
  std::vector<long long> out(keep.begin(), keep.end());
  std::unordered_set<long long> seen(out.begin(), out.end());
  if (k >= n) {
    for (long long i = 0; i < n; ++i)
      if (!seen.count(i)) out.push_back(i);
    return out;
  }
  while ((int)out.size() < k) {
    long long v = rng.below(n);
    if (seen.insert(v).second) out.push_back(v);
  }
  return out;
}

}  // namespace

// Y[row][col] = f(point(row, col)), see the row modes in cross3.
__global__ void k_fibers(GeomParams g, RhsParams f, int comp, const double *x1, const double *x2, const double *x3,
                         int rows, int cols, int rowmode, int Q2, const int *rowA, const int *rowB, const int *colA,
                         const int *colB, double *Y, int *status) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(e / cols), col = (int)(e % cols);
    int i1, i2, i3;
    if (rowmode == 0) {
      i1 = row; i2 = colA[col]; i3 = colB[col];
    } else if (rowmode == 1) {
      i1 = rowA[row / Q2]; i2 = row % Q2; i3 = colB[col];
    } else {
      i1 = rowA[row]; i2 = rowB[row]; i3 = col;
    }
    int bad = 0;
    Y[e] = field_value(g, f, comp, x1[i1], x2[i2], x3[i3], &bad);
    if (bad) atomicMax(status, (int)DS_BAD_GEOMETRY);
  }
}

__global__ void k_field_points(GeomParams g, RhsParams f, int comp, const double *x1, const double *x2,
                               const double *x3, int m, const int *idx, double *out, int *status) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    int bad = 0;
    out[t] = field_value(g, f, comp, x1[idx[3 * t]], x2[idx[3 * t + 1]], x3[idx[3 * t + 2]], &bad);
    if (bad) atomicMax(status, (int)DS_BAD_GEOMETRY);
  }
}

__global__ void k_maxabs_diff(const double *a, const double *b, long long n, double *out) {
  __shared__ double red[32];
  double v = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) v = fmax(v, fabs(a[i] - (b ? b[i] : 0.0)));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    *out = m;
  }
}

static double host_maxabs(Ctx *c, const double *a, const double *b, long long n) {
  k_maxabs_diff<<<1, 1024, 0, c->stream>>>(a, b, n, c->dscratch);
  TTI_LAUNCH();
  double v;
  c->d2h(&v, c->dscratch, sizeof v);
  return v;
}

void field_points(Ctx *c, const Space *s, const GeomParams &g, const RhsParams &f, int comp, int m, const int *idx,
                  double *out) {
  if (m <= 0) return;
  RhsParams ff = f;
  if (comp != 7) ff.has = 0;
  k_field_points<<<grid1d(m, 128), 128, 0, c->stream>>>(g, ff, comp, s[0].pts.d(), s[1].pts.d(), s[2].pts.d(), m, idx,
                                                         out, c->dstatus);
  TTI_LAUNCH();
}

namespace {

struct Sampler {
  Ctx *c;
  const Space *s;
  GeomParams g;
  RhsParams f;
  int comp;
  long long evals = 0;
  void fibers(int rows, int cols, int rowmode, const std::vector<int> &rowA, const std::vector<int> &rowB,
              const std::vector<int> &colA, const std::vector<int> &colB, double *Y) {
    DBuf dra(c, std::max<size_t>(1, rowA.size()) * sizeof(int)), drb(c, std::max<size_t>(1, rowB.size()) * sizeof(int));
    DBuf dca(c, std::max<size_t>(1, colA.size()) * sizeof(int)), dcb(c, std::max<size_t>(1, colB.size()) * sizeof(int));
    if (!rowA.empty()) c->h2d(dra.get(), rowA.data(), rowA.size() * sizeof(int));
    if (!rowB.empty()) c->h2d(drb.get(), rowB.data(), rowB.size() * sizeof(int));
    if (!colA.empty()) c->h2d(dca.get(), colA.data(), colA.size() * sizeof(int));
    if (!colB.empty()) c->h2d(dcb.get(), colB.data(), colB.size() * sizeof(int));
    long long tot = (long long)rows * cols;
    k_fibers<<<grid1d(tot, 128, 152 * 64), 128, 0, c->stream>>>(g, f, comp, s[0].pts.d(), s[1].pts.d(), s[2].pts.d(),
                                                               rows, cols, rowmode, s[1].Q, dra.as<int>(),
                                                               drb.as<int>(), dca.as<int>(), dcb.as<int>(), Y,
                                                               c->dstatus);
    TTI_LAUNCH();
    evals += tot;
    // the index buffers are released stream-ordered after the kernel
  }
};

// Truncated column basis of Y (rows x k): returns rank and U (rows x rank).
int skeleton(Ctx *c, const double *Y, int rows, int k, double rel, DBuf &U) {
  DBuf Q(c, (size_t)rows * k * sizeof(double)), R(c, (size_t)k * k * sizeof(double));
  qr(c, rows, k, Y, k, Q.d(), R.d());
  DBuf Ur(c, (size_t)k * k * sizeof(double)), S(c, (size_t)k * sizeof(double)), V(c, (size_t)k * k * sizeof(double));
  svd_small(c, k, R.d(), Ur.d(), S.d(), V.d());
  std::vector<double> sv(k);
  c->d2h(sv.data(), S.d(), k * sizeof(double));
  int r = 0;
  if (sv[0] > 0.0)
    while (r < k && r < rows && sv[r] > rel * sv[0]) ++r;
  if (r == 0) return 0;
  U = DBuf(c, (size_t)rows * r * sizeof(double));
  gemm<double>(c, false, false, rows, r, k, 1.0, Q.d(), k, 0, Ur.d(), k, 0, 0.0, U.d(), r, 0, 1);
  return r;
}

}  // namespace

void cross3(Ctx *c, const Space *s, const GeomParams &g, const RhsParams &f, int comp, double eps, int max_rank,
            uint64_t seed, double zero_scale, CrossResult &out, const std::function<double(double)> *zero_ref) {
  bool ref_asked = false;
  const int Q1 = s[0].Q, Q2 = s[1].Q, Q3 = s[2].Q;
  if (max_rank <= 0) max_rank = 64;
  max_rank = std::min(max_rank, 240);
  Sampler sm{c, s, g, f, comp};
  if (comp != 7) sm.f.has = 0;
  SplitMix rng(seed * 0x100000001B3ULL + 0x9E37ULL * (uint64_t)(comp + 1));
  const double rel = std::max(eps * 0.1, 1e-15);
  int k = 8;
  out = CrossResult();
  for (int attempt = 0; attempt < 4; ++attempt) {
    // ---- mode 1
    DBuf U1;
    int r1 = 0;
    std::vector<long long> cols1;
    double scale = 0.0;
    for (;;) {
      const long long space = (long long)Q2 * Q3;
      cols1 = distinct(rng, space, (int)std::min<long long>(k, space), cols1);
      const int k1 = (int)cols1.size();
      std::vector<int> ca(k1), cb(k1);
      for (int j = 0; j < k1; ++j) { ca[j] = (int)(cols1[j] % Q2); cb[j] = (int)(cols1[j] / Q2); }
      DBuf Y(c, (size_t)Q1 * k1 * sizeof(double));
      sm.fibers(Q1, k1, 0, {}, {}, ca, cb, Y.d());
      scale = host_maxabs(c, Y.d(), nullptr, (long long)Q1 * k1);
      if (zero_ref && !ref_asked) {
        zero_scale = (*zero_ref)(scale);
        ref_asked = true;
      }
      const double zs = zero_scale > 0 ? zero_scale : scale;
      if (scale <= 1e-13 * zs || scale == 0.0) {
        out.zero = true;
        out.scale = scale;
        out.evaluations = sm.evals;
        return;
      }
      r1 = skeleton(c, Y.d(), Q1, k1, rel, U1);
      if (r1 >= k1 - 1 && k1 < space && k1 < Q1 && k1 < max_rank + 8) {
        k = std::min<long long>(2 * k1, std::min<long long>(space, max_rank + 8));
        continue;
      }
      break;
    }
    r1 = std::min(r1, max_rank);
    DBuf G1(c, (size_t)Q1 * r1 * sizeof(double)), I1d(c, r1 * sizeof(int));
    {
      int mm = Q1, rr = r1;
      long long off = 0, roff = 0;
      maxvol_batched(c, 1, &mm, &rr, &off, U1.d(), G1.d(), I1d.as<int>(), &roff, 1e-2, 4 * r1 + 16);
    }
    std::vector<int> I1(r1);
    c->d2h(I1.data(), I1d.get(), r1 * sizeof(int));
    // ---- mode 2
    DBuf U2;
    int r2 = 0;
    std::vector<long long> cols2;
    const int rows2 = r1 * Q2;
    int kk = k;
    for (;;) {
      cols2 = distinct(rng, Q3, std::min(kk, Q3), cols2);
      const int k2 = (int)cols2.size();
      std::vector<int> cb(k2);
      for (int j = 0; j < k2; ++j) cb[j] = (int)cols2[j];
      DBuf Y(c, (size_t)rows2 * k2 * sizeof(double));
      sm.fibers(rows2, k2, 1, I1, {}, {}, cb, Y.d());
      r2 = skeleton(c, Y.d(), rows2, k2, rel, U2);
      if (r2 >= k2 - 1 && k2 < Q3 && k2 < rows2 && k2 < max_rank + 8) {
        kk = std::min(2 * k2, std::min(Q3, max_rank + 8));
        continue;
      }
      break;
    }
    if (r2 == 0) {  // the sampled slab vanished: treat the field as zero
      out.zero = true;
      out.scale = scale;
      out.evaluations = sm.evals;
      return;
    }
    r2 = std::min(r2, max_rank);
    DBuf G2(c, (size_t)rows2 * r2 * sizeof(double)), I2d(c, r2 * sizeof(int));
    {
      int mm = rows2, rr = r2;
      long long off = 0, roff = 0;
      maxvol_batched(c, 1, &mm, &rr, &off, U2.d(), G2.d(), I2d.as<int>(), &roff, 1e-2, 4 * r2 + 16);
    }
    std::vector<int> I2(r2);
    c->d2h(I2.data(), I2d.get(), r2 * sizeof(int));
    // ---- mode 3
    std::vector<int> P1(r2), P2(r2);
    for (int b = 0; b < r2; ++b) { P1[b] = I1[I2[b] / Q2]; P2[b] = I2[b] % Q2; }
    TT3 tt;
    tt.m[0] = Q1; tt.m[1] = Q2; tt.m[2] = Q3;
    tt.r[0] = 1; tt.r[1] = r1; tt.r[2] = r2; tt.r[3] = 1;
    tt.core[0] = std::move(G1);
    tt.core[1] = std::move(G2);
    tt.core[2] = DBuf(c, (size_t)r2 * Q3 * sizeof(double));
    sm.fibers(r2, Q3, 2, P1, P2, {}, {}, tt.core[2].d());
    // ---- validation on random grid points
    const int nv = 4096;
    std::vector<int> pts(3 * nv);
    for (int t = 0; t < nv; ++t) {
      pts[3 * t] = (int)rng.below(Q1);
      pts[3 * t + 1] = (int)rng.below(Q2);
      pts[3 * t + 2] = (int)rng.below(Q3);
    }
    DBuf dp(c, pts.size() * sizeof(int)), ex(c, nv * sizeof(double)), ap(c, nv * sizeof(double));
    c->h2d(dp.get(), pts.data(), pts.size() * sizeof(int));
    field_points(c, s, g, f, comp, nv, dp.as<int>(), ex.d());
    sm.evals += nv;
    tt_eval_points(c, tt, nv, dp.as<int>(), ap.d());
    const double err = host_maxabs(c, ex.d(), ap.d(), nv);
    const double ref = std::max(scale, zero_scale);
    out.tt = std::move(tt);
    out.scale = scale;
    out.max_rel_err = err / ref;
    out.evaluations = sm.evals;
    if (out.max_rel_err <= std::max(10.0 * eps, 1e-13)) {
      out.converged = true;
      return;
    }
    out.converged = false;
    k = std::min(2 * std::max(k, r1 + 8), max_rank + 8);
  }
}

}  // namespace ttiga
