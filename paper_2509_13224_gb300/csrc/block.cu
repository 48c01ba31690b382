// Multiple right-hand sides as one block-TT solve.  The right-hand-side index
// is one more tensor mode; merged into one of the three modes it leaves an
// ordinary order-3 TT system, so the AMEn solver, its local PCG, the
// preconditioners, the TT sums and the rounding all apply unchanged: the
// operator is I (x) K, i.e. that core of K repeated on the diagonal blocks of
// the merged mode, and the block solution carries all solutions in one TT
// whose ranks span all of them.  The interfaces, the local operators and
// their preconditioner factors are built once per step for all right-hand
// sides, and every local PCG works on all of them at once.
#include <algorithm>
#include <cmath>

#include "block.cuh"
#include "linalg.cuh"
#include "tt.cuh"

namespace ttiga {

// dst[R0][nb m][b][R1] block-diagonal in the merged mode: entry (k m + i, o) is
// src[R0][m][b][R1] entry (i, o) when column i + o - p lies in block k, else 0.
__global__ void k_block_band(const double *__restrict__ src, double *__restrict__ dst, int R0, int m, int b, int p,
                             int R1, int nb) {
  const long long tot = (long long)R0 * nb * m * b * R1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(e % R1);
    long long t = e / R1;
    const int o = (int)(t % b);
    t /= b;
    const int g = (int)(t % ((long long)nb * m));
    const int alpha = (int)(t / ((long long)nb * m));
    const int i = g % m, j = i + o - p;
    dst[e] = (j >= 0 && j < m) ? src[(((long long)alpha * m + i) * b + o) * R1 + beta] : 0.0;
  }
}

// dst[RA][M][RB] at rank offsets (oa, ob) and mode offset io = s * src[ra][m][rb].
__global__ void k_embed_mode(double *dst, int M, int RB, const double *src, int ra, int m, int rb, int oa, int io,
                             int ob, double s) {
  const long long tot = (long long)ra * m * rb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % rb);
    const long long t = e / rb;
    const int i = (int)(t % m), a = (int)(t / m);
    dst[(((long long)a + oa) * M + i + io) * RB + b + ob] = s * src[e];
  }
}

// dst[ra][m][rb] = s * src[ra][M][rb] rows io .. io + m - 1 of the mode.
__global__ void k_slice_mode(double *dst, const double *src, int ra, int m, int rb, int M, int io, double s) {
  const long long tot = (long long)ra * m * rb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % rb);
    const long long t = e / rb;
    const int i = (int)(t % m), a = (int)(t / m);
    dst[e] = s * src[(((long long)a * M) + i + io) * rb + b];
  }
}

void stack_system(Ctx *c, const tt_iga_system *s, int mode, double eps, tt_iga_system *out,
                  std::vector<double> &scale) {
  const int nb = (int)s->F.size();
  TTI_CHECK_ARG(nb >= 1, "stack: the system has no right-hand side");
  TTI_CHECK_ARG(s->stacked == 1, "stack: the system is already a block system");
  TTI_CHECK_ARG(mode >= 0 && mode < 3, "stack: mode %d out of range (0, 1, 2)", mode);
  const int m = s->n[mode], b = s->b, p = s->p;
  TTI_CHECK_ARG((long long)nb * m <= (1LL << 30), "stack: merged mode too large");
  scale.assign(nb, 0.0);
  for (int k = 0; k < nb; ++k) {
    scale[k] = s->F_norm[k];
    TTI_CHECK_ARG(scale[k] > 0.0, "stack: right-hand side %d is zero", k);
  }
  out->ctx = c;
  for (int d = 0; d < 3; ++d) out->n[d] = s->n[d];
  out->n[mode] = nb * m;
  out->p = p;
  out->b = b;
  out->bl = s->bl;
  out->stacked = nb;
  out->stack_mode = mode;
  // operator: core `mode` on every diagonal block of the merged mode, the others shared
  TT3 &K = out->K;
  for (int k = 0; k < 4; ++k) K.r[k] = s->K.r[k];
  for (int d = 0; d < 3; ++d) K.m[d] = s->K.m[d];
  K.m[mode] = nb * m * b;
  K.alloc(c);
  for (int d = 0; d < 3; ++d) {
    if (d == mode) {
      const long long tot = (long long)K.r[d] * nb * m * b * K.r[d + 1];
      k_block_band<<<grid1d(tot, 256), 256, 0, c->stream>>>(s->K.core[d].d(), K.core[d].d(), K.r[d], m, b, p,
                                                            K.r[d + 1], nb);
      TTI_LAUNCH();
    } else {
      TTI_CUDA(cudaMemcpyAsync(K.core[d].get(), s->K.core[d].get(), s->K.core_elems(d) * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  // load: F_b = sum_k e_k (x) F_k / ||F_k|| in the merged mode, a TT whose ranks add up
  // (block-diagonal inner cores, core 1 side by side, core 3 stacked), then one rounding
  TT3 Fb;
  for (int d = 0; d < 3; ++d) Fb.m[d] = s->n[d];
  Fb.m[mode] = nb * m;
  Fb.r[0] = Fb.r[3] = 1;
  Fb.r[1] = Fb.r[2] = 0;
  for (int k = 0; k < nb; ++k) {
    Fb.r[1] += s->F[k].r[1];
    Fb.r[2] += s->F[k].r[2];
  }
  Fb.alloc(c);
  for (int d = 0; d < 3; ++d) c->zero(Fb.core[d].get(), Fb.core_elems(d) * sizeof(double));
  int off[4] = {0, 0, 0, 0};
  for (int k = 0; k < nb; ++k) {
    const TT3 &Fk = s->F[k];
    for (int d = 0; d < 3; ++d) {
      const long long tot = (long long)Fk.r[d] * Fk.m[d] * Fk.r[d + 1];
      k_embed_mode<<<grid1d(tot, 256), 256, 0, c->stream>>>(Fb.core[d].d(), Fb.m[d], Fb.r[d + 1], Fk.core[d].d(),
                                                            Fk.r[d], Fk.m[d], Fk.r[d + 1], off[d],
                                                            d == mode ? k * m : 0, off[d + 1],
                                                            d == 0 ? 1.0 / scale[k] : 1.0);
      TTI_LAUNCH();
    }
    off[1] += Fk.r[1];
    off[2] += Fk.r[2];
  }
  const double nrm = tt_round(c, Fb, eps, 0);
  out->F.clear();
  out->F_norm.clear();
  out->F.push_back(std::move(Fb));
  out->F_norm.push_back(nrm);
}

constexpr double kSliceRoundTol = 1e-14;

void unstack_solution(Ctx *c, const tt_iga_solution *ub, int k, double scale, tt_iga_solution *out) {
  const int nb = ub->stacked, mode = ub->stack_mode;
  TTI_CHECK_ARG(nb > 1 || k == 0, "unstack: block %d of a plain solution", k);
  TTI_CHECK_ARG(k >= 0 && k < nb, "unstack: block %d out of range (%d blocks)", k, nb);
  const int m = ub->n[mode] / nb;
  out->ctx = c;
  for (int d = 0; d < 3; ++d) out->n[d] = ub->n[d];
  out->n[mode] = m;
  out->p = ub->p;
  out->bl = ub->bl;
  out->stacked = 1;
  TT3 &u = out->u;
  for (int d = 0; d < 3; ++d) u.m[d] = ub->u.m[d];
  u.m[mode] = m;
  for (int d = 0; d < 4; ++d) u.r[d] = ub->u.r[d];
  u.alloc(c);
  for (int d = 0; d < 3; ++d) {
    const double sd = d == 0 ? scale : 1.0;
    const long long tot = (long long)u.core_elems(d);
    k_slice_mode<<<grid1d(tot, 256), 256, 0, c->stream>>>(u.core[d].d(), ub->u.core[d].d(), u.r[d], u.m[d],
                                                          u.r[d + 1], ub->u.m[d], d == mode ? k * m : 0, sd);
    TTI_LAUNCH();
  }
  // The slice inherits the block solution's ranks, which span the subspaces of every right-hand
  // side; rounding to 1e-14 relative accuracy keeps its own numerical rank only, so evaluation,
  // L2 errors and residuals of the slice do not pay for the other right-hand sides.
  if (u.r[1] > 1 || u.r[2] > 1) tt_round(c, u, kSliceRoundTol, 0);
}

}  // namespace ttiga
