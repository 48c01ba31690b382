// TT-IGA assembly on the device (Sections 4.2.1, 4.2.2, 4.3).
//
// Per-direction quadrature contraction: for a coefficient core G[r0][Q][r1]
//   M[alpha][i][o][beta] = sum_q w_q G[alpha][q][beta] A_i(q) B_{i+o-p}(q)
// where (A, B) are (N', N'), (N, N), (N', N) or (N, N') by the a_ij^(d)
// selector.  Basis functions i and j = i+o-p overlap only on the elements
// max(i, j) - p .. min(i, j), so each band output sums at most (p+1) nq terms.
// One thread per band output, consecutive threads on consecutive beta so
// reads of G and writes of M are coalesced along the rank.
#include <algorithm>
#include <utility>
#include <cmath>

#include "amen_ops.cuh"
#include "handles.cuh"
#include "linalg.cuh"
#include "tt.cuh"

namespace ttiga {

__global__ void k_stiffness_core(int n, int p, int nq, const double *__restrict__ wts, const double *__restrict__ TA,
                                 const double *__restrict__ TB, const double *__restrict__ G, int r0, int r1,
                                 double *__restrict__ M) {
  const int b = 2 * p + 1, ne = n - p, Q = ne * nq, P = p + 1;
  const long long tot = (long long)r0 * n * b * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(e % r1);
    long long t = e / r1;
    const int o = (int)(t % b);
    t /= b;
    const int i = (int)(t % n);
    const int alpha = (int)(t / n);
    const int j = i + o - p;
    double acc = 0.0;
    if (j >= 0 && j < n) {
      const int elo = max(max(i, j) - p, 0), ehi = min(min(i, j), ne - 1);
      for (int el = elo; el <= ehi; ++el) {
        for (int l = 0; l < nq; ++l) {
          const int q = el * nq + l;
          acc += wts[q] * G[((long long)alpha * Q + q) * r1 + beta] * TA[(long long)q * P + (i - el)] *
                 TB[(long long)q * P + (j - el)];
        }
      }
    }
    M[e] = acc;
  }
}

__global__ void k_load_core(int n, int p, int nq, const double *__restrict__ wts, const double *__restrict__ TN,
                            const double *__restrict__ G, int r0, int r1, double *__restrict__ F) {
  const int ne = n - p, Q = ne * nq, P = p + 1;
  const long long tot = (long long)r0 * n * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(e % r1);
    const long long t = e / r1;
    const int i = (int)(t % n);
    const int alpha = (int)(t / n);
    const int elo = max(i - p, 0), ehi = min(i, ne - 1);
    double acc = 0.0;
    for (int el = elo; el <= ehi; ++el)
      for (int l = 0; l < nq; ++l) {
        const int q = el * nq + l;
        acc += wts[q] * G[((long long)alpha * Q + q) * r1 + beta] * TN[(long long)q * P + (i - el)];
      }
    F[e] = acc;
  }
}

void stiffness_core(Ctx *c, int n, int p, int nq, const double *wts, const double *N, const double *dN, const double *G,
                    int r0, int r1, int test_deriv, int trial_deriv, double *M) {
  TTI_CHECK_ARG(n > p && p >= 1 && nq >= 1 && r0 >= 1 && r1 >= 1, "stiffness_core: bad sizes");
  const long long tot = (long long)r0 * n * (2 * p + 1) * r1;
  k_stiffness_core<<<grid1d(tot, 256, 152 * 32), 256, 0, c->stream>>>(n, p, nq, wts, test_deriv ? dN : N,
                                                                     trial_deriv ? dN : N, G, r0, r1, M);
  TTI_LAUNCH();
}

void load_core(Ctx *c, int n, int p, int nq, const double *wts, const double *N, const double *G, int r0, int r1,
               double *F) {
  TTI_CHECK_ARG(n > p && p >= 1 && nq >= 1 && r0 >= 1 && r1 >= 1, "load_core: bad sizes");
  const long long tot = (long long)r0 * n * r1;
  k_load_core<<<grid1d(tot, 256, 152 * 32), 256, 0, c->stream>>>(n, p, nq, wts, N, G, r0, r1, F);
  TTI_LAUNCH();
}

// Normal-direction core of a face load: the area density's core G[r0][Q][r1] does not vary
// along the mode (the field is evaluated on the face), so its first slice, scaled by the flux
// q, sits on basis function idx (0 or n - 1, the only one nonzero on the face); the others are 0.
__global__ void k_face_core(const double *G, int r0, int Q, int r1, int n, int idx, double q, double *F) {
  const long long tot = (long long)r0 * n * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(e % r1);
    const long long t = e / r1;
    const int i = (int)(t % n), alpha = (int)(t / n);
    F[e] = (i == idx) ? q * G[(long long)alpha * Q * r1 + beta] : 0.0;
  }
}

// Drop basis functions 0 and n-1 (homogeneous Dirichlet, Section 4.3):
// band core [r0][n][b][r1] -> [r0][n-2][b][r1], zeroing couplings to the dropped functions.
// Keep functions lo .. lo + nr - 1 of a band core (couplings to dropped functions zeroed).
__global__ void k_restrict_band(const double *src, double *dst, int r0, int n, int p, int r1, int lo, int nr) {
  const int b = 2 * p + 1;
  const long long tot = (long long)r0 * nr * b * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(e % r1);
    long long t = e / r1;
    const int o = (int)(t % b);
    t /= b;
    const int ir = (int)(t % nr);
    const int alpha = (int)(t / nr);
    const int jr = ir + o - p;
    dst[e] = (jr >= 0 && jr < nr) ? src[(((long long)alpha * n + ir + lo) * b + o) * r1 + beta] : 0.0;
  }
}

__global__ void k_restrict_vec(const double *src, double *dst, int r0, int n, int r1, int lo, int nr) {
  const long long tot = (long long)r0 * nr * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(e % r1);
    const long long t = e / r1;
    const int ir = (int)(t % nr), alpha = (int)(t / nr);
    dst[e] = src[((long long)alpha * n + ir + lo) * r1 + beta];
  }
}

static void restrict_tt(Ctx *c, TT3 &x, const BoundaryLayout &bl, int p, bool band) {
  for (int k = 0; k < 3; ++k) {
    const int r0 = x.r[k], r1 = x.r[k + 1];
    const int n = bl.nfull[k], nr = n - bl.lo[k] - bl.hi[k];
    const int bw = band ? 2 * p + 1 : 1;
    DBuf out(c, (size_t)r0 * nr * bw * r1 * sizeof(double));
    const long long tot = (long long)r0 * nr * bw * r1;
    if (band)
      k_restrict_band<<<grid1d(tot, 256), 256, 0, c->stream>>>(x.core[k].d(), out.d(), r0, n, p, r1, bl.lo[k], nr);
    else
      k_restrict_vec<<<grid1d(tot, 256), 256, 0, c->stream>>>(x.core[k].d(), out.d(), r0, n, r1, bl.lo[k], nr);
    TTI_LAUNCH();
    x.core[k] = std::move(out);
    x.m[k] = nr * bw;
  }
}

static TT3 clone_tt(Ctx *c, const TT3 &x) {
  TT3 y;
  for (int k = 0; k < 3; ++k) y.m[k] = x.m[k];
  for (int k = 0; k < 4; ++k) y.r[k] = x.r[k];
  y.alloc(c);
  for (int k = 0; k < 3; ++k)
    TTI_CUDA(cudaMemcpyAsync(y.core[k].get(), x.core[k].get(), x.core_elems(k) * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
  return y;
}

BoundaryLayout boundary_layout(const tt_iga_bc_desc *bc, const int nfull[3]) {
  BoundaryLayout bl;
  for (int d = 0; d < 3; ++d) bl.nfull[d] = nfull[d];
  if (!bc) return bl;
  bool any = false;
  int dir = -1;
  for (int d = 0; d < 3; ++d) {
    bl.lo[d] = bc->dirichlet[2 * d] ? 1 : 0;
    bl.hi[d] = bc->dirichlet[2 * d + 1] ? 1 : 0;
    any = any || bl.lo[d] || bl.hi[d];
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * d + side;
      TTI_CHECK_ARG(std::isfinite(bc->value[f]), "bc: value of face %d is not finite", f);
      TTI_CHECK_ARG(std::isfinite(bc->flux[f]), "bc: flux of face %d is not finite", f);
      TTI_CHECK_ARG(bc->flux[f] == 0.0 || !bc->dirichlet[f], "bc: flux on the Dirichlet face %d", f);
      bl.flux[f] = bc->flux[f];
      if (bc->dirichlet[2 * d + side] && bc->value[2 * d + side] != 0.0) {
        TTI_CHECK_ARG(dir < 0 || dir == d, "bc: nonzero Dirichlet data on more than one direction");
        dir = d;
      }
    }
  }
  TTI_CHECK_ARG(any, "bc: no Dirichlet face (the operator would be singular)");
  if (dir >= 0) {
    for (int e = 0; e < 3; ++e)
      TTI_CHECK_ARG(e == dir || (!bl.lo[e] && !bl.hi[e]),
                    "bc: nonzero data on direction %d needs natural faces in direction %d", dir, e);
    bl.lift_dir = dir;
    bl.lift_lo = bc->dirichlet[2 * dir] ? bc->value[2 * dir] : 0.0;
    bl.lift_hi = bc->dirichlet[2 * dir + 1] ? bc->value[2 * dir + 1] : 0.0;
  }
  for (int d = 0; d < 3; ++d)
    TTI_CHECK_ARG(nfull[d] - bl.lo[d] - bl.hi[d] >= 1, "bc: no unknowns left in direction %d", d);
  return bl;
}

// The operator (sum of the K_ab terms, rounded after every addition) and each
// load vector are independent and are built concurrently on helper contexts.
void assemble_system(Ctx *c, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int n_rhs, double round_tol,
                     const BoundaryLayout &bl, tt_iga_system *out) {
  const int p = g->desc.p;
  const int b = 2 * p + 1;
  int n[3];
  for (int d = 0; d < 3; ++d) n[d] = g->s[d].n;
  const bool lift = bl.lift_dir >= 0;
  const bool flux = bl.has_flux();
  TT3 K, Kfull;  // Kfull: the operator before restriction, kept for F - K g
  TT3 Fn;        // sum of the face loads of the flux data
  std::vector<TT3> F(n_rhs);
  std::vector<double> F_norm(n_rhs, 0.0);

  // K = sum of the K_ab terms, rounded after every summation step (Section 4.2.1), which
  // keeps the ranks from inflating.  A step sums as many consecutive terms as keep the
  // summed ranks within kSumRankCap (at least two), since rounding a sum of ranks up to
  // that cap costs about what rounding a pair does, and the groups of a level run
  // concurrently; with the low-rank coefficient fields of smooth geometries one step
  // takes all terms, one rounding instead of a tree of them.
  auto build_operator = [&](Ctx *h) {
    std::vector<TT3> terms;
    static const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (auto &pr : pairs) {
      const int i = pr[0], j = pr[1];
      const CrossResult &R = g->R[field_of(i, j)];
      if (R.zero) continue;
      const int nterms = (i == j) ? 1 : 2;
      for (int t = 0; t < nterms; ++t) {
        const int a = t == 0 ? i : j, bb = t == 0 ? j : i;  // K_ab: derivative on test index in direction a
        TT3 T;
        for (int d = 0; d < 3; ++d) T.m[d] = n[d] * b;
        for (int k = 0; k < 4; ++k) T.r[k] = R.tt.r[k];
        T.alloc(h);
        for (int d = 0; d < 3; ++d)
          stiffness_core(h, n[d], p, g->s[d].nq, g->s[d].wts.d(), g->s[d].N.d(), g->s[d].dN.d(), R.tt.core[d].d(),
                         R.tt.r[d], R.tt.r[d + 1], d == a, d == bb, T.core[d].d());
        terms.push_back(std::move(T));
      }
    }
    TTI_CHECK_ARG(!terms.empty(), "assemble: every coefficient field vanished");
    constexpr int kSumRankCap = 32;
    bool restricted = false;
    while (terms.size() > 1) {
      std::vector<std::pair<int, int>> groups;  // [begin, end) of consecutive terms
      const int nt = (int)terms.size();
      for (int i0 = 0; i0 < nt;) {
        int r1 = terms[i0].r[1], r2 = terms[i0].r[2], i1 = i0 + 1;
        while (i1 < nt && r1 + terms[i1].r[1] <= kSumRankCap && r2 + terms[i1].r[2] <= kSumRankCap) {
          r1 += terms[i1].r[1];
          r2 += terms[i1].r[2];
          ++i1;
        }
        if (i1 == i0 + 1 && i1 < nt) ++i1;  // at least a pair: every level shrinks
        groups.emplace_back(i0, i1);
        i0 = i1;
      }
      // the level that leaves one term makes the operator: without a lift its Dirichlet
      // restriction (linear) goes before that rounding, which then serves both
      const bool last = groups.size() == 1;
      std::vector<TT3> next(groups.size());
      std::vector<int> sums;  // groups that are summed and rounded (a lone last term moves on)
      for (int q = 0; q < (int)groups.size(); ++q) {
        if (groups[q].second - groups[q].first == 1) next[q] = std::move(terms[groups[q].first]);
        else sums.push_back(q);
      }
      run_concurrent(h, (int)sums.size(), [&](int t, Ctx *hh) {
        const int q = sums[t];
        std::vector<const TT3 *> xs;
        for (int i = groups[q].first; i < groups[q].second; ++i) xs.push_back(&terms[i]);
        tt_sum_many(hh, xs, next[q]);
        if (last && !lift) restrict_tt(hh, next[q], bl, p, true);
        tt_round(hh, next[q], round_tol, 0);
        for (int d = 0; d < 3; ++d) next[q].core[d].rehome(h);
      });
      terms = std::move(next);  // the consumed terms are freed on h, after the helpers (ordered by the join)
      if (last && !lift) restricted = true;
    }
    K = std::move(terms[0]);
    if (lift) {
      Kfull = clone_tt(h, K);
      for (int d = 0; d < 3; ++d) Kfull.core[d].rehome(c);
    }
    if (!restricted) {
      restrict_tt(h, K, bl, p, true);
      tt_round(h, K, round_tol, 0);
    }
    for (int d = 0; d < 3; ++d) K.core[d].rehome(c);
  };

  auto build_load = [&](int k, Ctx *h) {
    RhsParams rp = rhs_params(&rhs[k]);
    CrossResult fj;
    cross3(h, g->s, g->gp, rp, 7, g->desc.cross_tol, g->desc.max_rank, g->desc.seed + 7919ULL * (k + 1), 0.0, fj);
    TT3 &Fk = F[k];
    for (int d = 0; d < 3; ++d) Fk.m[d] = n[d];
    if (fj.zero) {
      Fk.r[1] = Fk.r[2] = 1;
      Fk.alloc(h);
      for (int d = 0; d < 3; ++d) h->zero(Fk.core[d].get(), Fk.core_elems(d) * sizeof(double));
    } else {
      for (int q = 0; q < 4; ++q) Fk.r[q] = fj.tt.r[q];
      Fk.alloc(h);
      for (int d = 0; d < 3; ++d)
        load_core(h, n[d], p, g->s[d].nq, g->s[d].wts.d(), g->s[d].N.d(), fj.tt.core[d].d(), fj.tt.r[d],
                  fj.tt.r[d + 1], Fk.core[d].d());
    }
    if (!lift && !flux) {
      restrict_tt(h, Fk, bl, p, false);
      F_norm[k] = tt_round(h, Fk, round_tol, 0);
    }
    for (int d = 0; d < 3; ++d) Fk.core[d].rehome(c);
  };

  // Surface load vector of the flux data (f_s of Section 3.3, the boundary term of the weak
  // form of Section 3.2), F_a = q int_face N_a dGamma: the area density of each face with a
  // flux by TT-cross, contracted with the tangential quadrature, summed over the faces.
  auto build_faces = [&](Ctx *h) {
    std::vector<TT3> terms;
    RhsParams none = rhs_params(nullptr);
    for (int f = 0; f < 6; ++f) {
      const double q = bl.flux[f];
      if (q == 0.0) continue;
      const int d = f >> 1;
      CrossResult a;
      cross3(h, g->s, g->gp, none, kFaceComp0 + f, g->desc.cross_tol, g->desc.max_rank,
             g->desc.seed + 104729ULL * (f + 1), 0.0, a);
      TTI_CHECK_ARG(!a.zero, "bc: face %d has zero area", f);
      if (!a.converged) fail(TT_IGA_ERR_NOT_CONVERGED, "bc: TT-cross of the area of face %d did not validate", f);
      TT3 T;
      for (int k = 0; k < 3; ++k) T.m[k] = n[k];
      for (int k = 0; k < 4; ++k) T.r[k] = a.tt.r[k];
      T.alloc(h);
      for (int k = 0; k < 3; ++k) {
        if (k == d) {
          const long long tot = (long long)T.r[k] * n[k] * T.r[k + 1];
          k_face_core<<<grid1d(tot, 256), 256, 0, h->stream>>>(a.tt.core[k].d(), T.r[k], g->s[k].Q, T.r[k + 1], n[k],
                                                                (f & 1) ? n[k] - 1 : 0, q, T.core[k].d());
          TTI_LAUNCH();
        } else {
          load_core(h, n[k], p, g->s[k].nq, g->s[k].wts.d(), g->s[k].N.d(), a.tt.core[k].d(), T.r[k], T.r[k + 1],
                    T.core[k].d());
        }
      }
      if (!terms.empty()) {
        TT3 S;
        tt_sum(h, terms.back(), 1.0, T, 1.0, S);
        tt_round(h, S, round_tol, 0);
        terms.back() = std::move(S);
      } else {
        terms.push_back(std::move(T));
      }
    }
    Fn = std::move(terms.back());
    for (int k = 0; k < 3; ++k) Fn.core[k].rehome(c);
  };

  run_concurrent(c, 1 + n_rhs + (flux ? 1 : 0), [&](int task, Ctx *h) {
    if (task == 0) build_operator(h);
    else if (task <= n_rhs) build_load(task - 1, h);
    else build_faces(h);
  });

  if (flux && !lift) {
    for (int k = 0; k < n_rhs; ++k) {
      TT3 S;
      tt_sum(c, F[k], 1.0, Fn, 1.0, S);
      restrict_tt(c, S, bl, p, false);
      F_norm[k] = tt_round(c, S, round_tol, 0);
      F[k] = std::move(S);
    }
  }
  if (lift) {
    // g = (lift_lo e_0 + lift_hi e_{n-1}) in direction lift_dir, ones in the others (rank 1);
    // K g by band TT-matrix times TT vector, then F_k <- F_k - K g, restricted and rounded
    TT3 G;
    for (int d = 0; d < 3; ++d) G.m[d] = n[d];
    G.r[1] = G.r[2] = 1;
    G.alloc(c);
    for (int d = 0; d < 3; ++d) {
      std::vector<double> v(n[d], d == bl.lift_dir ? 0.0 : 1.0);
      if (d == bl.lift_dir) {
        v[0] = bl.lift_lo;
        v[n[d] - 1] = bl.lift_hi;
      }
      c->h2d(G.core[d].get(), v.data(), v.size() * sizeof(double));
    }
    TT3 Kg;
    for (int d = 0; d < 3; ++d) Kg.m[d] = n[d];
    for (int k = 0; k < 4; ++k) Kg.r[k] = Kfull.r[k];
    Kg.alloc(c);
    for (int d = 0; d < 3; ++d) {
      BandCore A{Kfull.core[d].d(), nullptr, Kfull.r[d], n[d], b, p, Kfull.r[d + 1]};
      tt_matvec_core(c, A, G.core[d].d(), 1, 1, Kg.core[d].d());
    }
    c->sync();  // the host vectors above are released at scope end
    for (int k = 0; k < n_rhs; ++k) {
      if (flux) {
        TT3 T;
        tt_sum(c, F[k], 1.0, Fn, 1.0, T);
        F[k] = std::move(T);
      }
      TT3 S;
      tt_sum(c, F[k], 1.0, Kg, -1.0, S);
      restrict_tt(c, S, bl, p, false);
      F_norm[k] = tt_round(c, S, round_tol, 0);
      F[k] = std::move(S);
    }
  }

  out->ctx = c;
  out->p = p;
  out->b = b;
  out->bl = bl;
  for (int d = 0; d < 3; ++d) out->n[d] = n[d] - bl.lo[d] - bl.hi[d];
  out->K = std::move(K);
  out->F.clear();
  out->F_norm.clear();
  for (int k = 0; k < n_rhs; ++k) {
    out->F.push_back(std::move(F[k]));
    out->F_norm.push_back(F_norm[k]);
  }
}

// Mass matrix on the mapped domain, M_ab = int N_a N_b det J dxi, restricted to the
// unknowns of bl: det J on the tensor Gauss grid by TT-cross (component 6 of the
// point evaluator) to the geometry's cross tolerance, then the per-direction
// quadrature contraction of Section 4.2.1 with the selector (N, N) in every
// direction (no derivative), the same Gauss rule as the stiffness.
void mass_matrix(Ctx *c, const tt_iga_geom *g, const BoundaryLayout &bl, TT3 &M) {
  const int p = g->desc.p, b = 2 * p + 1;
  CrossResult dj;
  cross3(c, g->s, g->gp, rhs_params(nullptr), 6, g->desc.cross_tol, g->desc.max_rank, g->desc.seed + 15485863ULL, 0.0,
         dj);
  TTI_CHECK_ARG(!dj.zero, "mass matrix: det J vanishes on the sampled grid");
  if (!dj.converged) fail(TT_IGA_ERR_NOT_CONVERGED, "mass matrix: TT-cross of det J did not validate");
  for (int d = 0; d < 3; ++d) M.m[d] = g->s[d].n * b;
  for (int k = 0; k < 4; ++k) M.r[k] = dj.tt.r[k];
  M.alloc(c);
  for (int d = 0; d < 3; ++d)
    stiffness_core(c, g->s[d].n, p, g->s[d].nq, g->s[d].wts.d(), g->s[d].N.d(), g->s[d].dN.d(), dj.tt.core[d].d(),
                   dj.tt.r[d], dj.tt.r[d + 1], 0, 0, M.core[d].d());
  restrict_tt(c, M, bl, p, true);
}

// K(row, col) of the restricted band TT operator at index pairs.
__global__ void k_op_entries(const double *M1, const double *M2, const double *M3, int n1, int n2, int n3, int p,
                             int r1, int r2, int m, const int *rows, const int *cols, double *out) {
  const int b = 2 * p + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    const int i1 = rows[3 * t], i2 = rows[3 * t + 1], i3 = rows[3 * t + 2];
    const int o1 = cols[3 * t] - i1 + p, o2 = cols[3 * t + 1] - i2 + p, o3 = cols[3 * t + 2] - i3 + p;
    double v = 0.0;
    if (o1 >= 0 && o1 < b && o2 >= 0 && o2 < b && o3 >= 0 && o3 < b) {
      for (int a = 0; a < r1; ++a) {
        const double x = M1[((long long)i1 * b + o1) * r1 + a];
        if (x == 0.0) continue;
        double s = 0.0;
        for (int c2 = 0; c2 < r2; ++c2)
          s += M2[(((long long)a * n2 + i2) * b + o2) * r2 + c2] * M3[((long long)c2 * n3 + i3) * b + o3];
        v += x * s;
      }
    }
    out[t] = v;
  }
}

void operator_entries(Ctx *c, const tt_iga_system *s, int m, const int *rows, const int *cols, double *out) {
  if (m <= 0) return;
  k_op_entries<<<grid1d(m, 128), 128, 0, c->stream>>>(s->K.core[0].d(), s->K.core[1].d(), s->K.core[2].d(), s->n[0],
                                                       s->n[1], s->n[2], s->p, s->K.r[1], s->K.r[2], m, rows, cols, out);
  TTI_LAUNCH();
}

}  // namespace ttiga
