// extern "C" entry points of the TT-IGA library (include/tt_iga.h).
#include <algorithm>
#include <future>
#include <cmath>

#include "amen.cuh"
#include "amen_ops.cuh"
#include "block.cuh"
#include "eval.cuh"
#include "handles.cuh"
#include "bbprec.cuh"
#include "linalg.cuh"
#include "pcg_fused.cuh"
#include "tt.cuh"

namespace ttiga {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_live_contexts{0};

// Read and clear the device status word; map it to a status code.
static int device_status(Ctx *c) {
  int s = 0;
  c->d2h(&s, c->dstatus, sizeof s);
  if (s != 0) c->zero(c->dstatus, sizeof(int));
  switch (s) {
    case DS_OK: return TT_IGA_OK;
    case DS_BAD_GEOMETRY: return TT_IGA_ERR_BAD_GEOMETRY;
    default: return TT_IGA_ERR_NOT_CONVERGED;
  }
}

__global__ void k_op_dense(const double *M1, const double *M2, const double *M3, int n1, int n2, int n3, int p, int r1,
                           int r2, double *out) {
  const long long N = (long long)n1 * n2 * n3;
  const int b = 2 * p + 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * N; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / N, col = e % N;
    const int i1 = (int)(row % n1), i2 = (int)((row / n1) % n2), i3 = (int)(row / ((long long)n1 * n2));
    const int j1 = (int)(col % n1), j2 = (int)((col / n1) % n2), j3 = (int)(col / ((long long)n1 * n2));
    const int o1 = j1 - i1 + p, o2 = j2 - i2 + p, o3 = j3 - i3 + p;
    double v = 0.0;
    if (o1 >= 0 && o1 < b && o2 >= 0 && o2 < b && o3 >= 0 && o3 < b) {
      for (int a = 0; a < r1; ++a) {
        double s = 0.0;
        for (int c2 = 0; c2 < r2; ++c2)
          s += M2[(((long long)a * n2 + i2) * b + o2) * r2 + c2] * M3[((long long)c2 * n3 + i3) * b + o3];
        v += M1[((long long)i1 * b + o1) * r1 + a] * s;
      }
    }
    out[e] = v;
  }
}

}  // namespace ttiga

using namespace ttiga;

#define API_TRY try {
#define API_CATCH(ctxp)                                                   \
  }                                                                       \
  catch (const ttiga::Error &e) {                                         \
    if (ctxp) (ctxp)->last_error = e.what();                              \
    return e.code;                                                        \
  }                                                                       \
  catch (const std::exception &e) {                                       \
    if (ctxp) (ctxp)->last_error = e.what();                              \
    return TT_IGA_ERR_CUDA;                                               \
  }

extern "C" {

int tt_iga_ctx_create(tt_iga_ctx **out, const tt_iga_ctx_opts *o) {
  if (!out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  tt_iga_ctx *c = new tt_iga_ctx();
  API_TRY
  c->device = o ? o->device : 0;
  TTI_CUDA(cudaSetDevice(c->device));
  if (o && (o->alloc_fn != nullptr) != (o->free_fn != nullptr)) fail(TT_IGA_ERR_ARG, "alloc_fn and free_fn go together");
  if (o && o->stream) {
    c->stream = (cudaStream_t)o->stream;
  } else {
    TTI_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  if (o) {
    c->alloc_fn = o->alloc_fn;
    c->free_fn = o->free_fn;
    c->alloc_user = o->alloc_user;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  TTI_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  TTI_CUDA(cudaMalloc(&c->dstatus, 64));
  TTI_CUDA(cudaMemset(c->dstatus, 0, 64));
  TTI_CUDA(cudaMalloc(&c->dscratch, Ctx::kScratchDoubles * sizeof(double)));
  *out = c;
  g_live_contexts.fetch_add(1, std::memory_order_relaxed);
  return TT_IGA_OK;
  }
  catch (const ttiga::Error &e) {
    int code = e.code;
    delete c;
    return code;
  }
}

void tt_iga_ctx_destroy(tt_iga_ctx *c) {
  if (!c) return;
  g_live_contexts.fetch_sub(1, std::memory_order_relaxed);
  cudaStreamSynchronize(c->stream);
  c->release_subs();
  if (c->dstatus) cudaFree(c->dstatus);
  if (c->dscratch) cudaFree(c->dscratch);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  for (auto &e : c->prof_events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  delete c;
}

const char *tt_iga_last_error(const tt_iga_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

int tt_iga_ctx_memory(const tt_iga_ctx *c, size_t *in_use, size_t *peak) {
  if (!c) return TT_IGA_ERR_ARG;
  if (in_use) *in_use = c->in_use;
  if (peak) *peak = c->peak;
  return TT_IGA_OK;
}

unsigned long long tt_iga_launch_count(void) { return ttiga::g_launches.load(); }

int tt_iga_ctx_set_sm_limit(tt_iga_ctx *c, int max_sms) {
  if (!c || max_sms < 0) return TT_IGA_ERR_ARG;
  c->coop_sms = max_sms;
  for (auto &s : c->subs) s->coop_sms = max_sms;
  return TT_IGA_OK;
}

int tt_iga_profile_enable(tt_iga_ctx *c, int family) {
  if (!c || family < 0 || family > 6) return TT_IGA_ERR_ARG;
  API_TRY
  c->sync();
  c->prof_family = family;
  c->prof_used = 0;
  c->prof_work.clear();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_profile_read(tt_iga_ctx *c, double *ms_total, long long *launches, double *flops_total) {
  if (!c) return TT_IGA_ERR_ARG;
  API_TRY
  c->sync();
  double ms = 0.0, work = 0.0;
  for (size_t i = 0; i < c->prof_used; ++i) {
    float t = 0.f;
    TTI_CUDA(cudaEventElapsedTime(&t, c->prof_events[i].first, c->prof_events[i].second));
    ms += t;
    work += c->prof_work[i];
  }
  if (ms_total) *ms_total = ms;
  if (launches) *launches = (long long)c->prof_used;
  if (flops_total) *flops_total = work;
  return TT_IGA_OK;
  API_CATCH(c)
}

// ------------------------------------------------------------------ geometry

namespace {

void check_discretisation(const tt_iga_geom_desc *g) {
  TTI_CHECK_ARG(g->p >= 1 && g->p <= 7, "geometry: degree p=%d outside 1..7", g->p);
  for (int d = 0; d < 3; ++d)
    TTI_CHECK_ARG(g->n[d] >= g->p + 2, "geometry: n[%d]=%d needs >= p+2", d, g->n[d]);
  const int nq = g->nq > 0 ? g->nq : g->p + 1;
  TTI_CHECK_ARG(nq <= 8, "geometry: nq=%d above 8", nq);
}

// Tables of the three directions and the TT-cross of the six fields of R (shared by
// the analytic maps and the NURBS patch); G->desc and G->gp are set by the caller.
int build_geometry(tt_iga_ctx *c, tt_iga_geom *G, const tt_iga_geom_desc *g) {
  const int nq = G->desc.nq;
  for (int d = 0; d < 3; ++d) build_space(c, G->s[d], g->n[d], g->p, nq);
  RhsParams none = rhs_params(nullptr);
  const int diag[3] = {0, 3, 5}, off[3] = {1, 2, 4};
  // All six fields run concurrently.  An off-diagonal field is rank 0 when its
  // magnitude is below 1e-13 of the largest diagonal magnitude; the diagonal
  // fields publish theirs after their first fibre sample and the off-diagonal
  // ones wait for them there.  Every field has its own seed, so the result
  // does not depend on the order in which the fields run.
  std::promise<double> diag_scale[3];
  std::shared_future<double> diag_ref[3];
  for (int i = 0; i < 3; ++i) diag_ref[i] = diag_scale[i].get_future().share();
  run_concurrent(c, 6, [&](int i, Ctx *h) {
    const int f = i < 3 ? diag[i] : off[i - 3];
    bool published = false;
    std::function<double(double)> ref;
    if (i < 3)
      ref = [&, i](double own) {
        diag_scale[i].set_value(own);
        published = true;
        return 0.0;
      };
    else
      ref = [&](double) {
        double m = 0.0;
        for (auto &r : diag_ref) m = std::max(m, r.get());
        return m;  // 0 when every diagonal field vanished: the field's own scale decides
      };
    try {
      cross3(h, G->s, G->gp, none, f, G->desc.cross_tol, G->desc.max_rank, G->desc.seed + 101ULL * (f + 1), 0.0,
             G->R[f], &ref);
    } catch (...) {
      if (i < 3 && !published) diag_scale[i].set_exception(std::current_exception());
      throw;
    }
    for (int k = 0; k < 3; ++k) G->R[f].tt.core[k].rehome(c);
  });
  bool conv = true;
  for (int f = 0; f < 6; ++f) conv = conv && G->R[f].converged;
  const int st = device_status(c);
  if (st == TT_IGA_ERR_BAD_GEOMETRY) {
    c->last_error = "geometry: det J <= 0 at a sampled quadrature point";
    return st;
  }
  if (!conv) {
    c->last_error = "geometry: TT-cross did not validate within max_rank";
    return TT_IGA_ERR_NOT_CONVERGED;
  }
  return TT_IGA_OK;
}

tt_iga_geom *new_geometry(tt_iga_ctx *c, const tt_iga_geom_desc *g) {
  auto *G = new tt_iga_geom();
  G->ctx = c;
  G->desc = *g;
  G->desc.nq = g->nq > 0 ? g->nq : g->p + 1;
  if (G->desc.cross_tol <= 0) G->desc.cross_tol = 1e-10;
  if (G->desc.max_rank <= 0) G->desc.max_rank = 64;
  G->gp = geom_params(G->desc);
  return G;
}

}  // namespace

int tt_iga_geometry(tt_iga_ctx *c, const tt_iga_geom_desc *g, tt_iga_geom **out) {
  if (!c || !g || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  TTI_CHECK_ARG(g->kind == TT_IGA_GEOM_BOX || g->kind == TT_IGA_GEOM_ANNULUS,
                "geometry: unknown kind %d (NURBS patches go through tt_iga_geometry_nurbs)", g->kind);
  check_discretisation(g);
  if (g->kind == TT_IGA_GEOM_ANNULUS)
    TTI_CHECK_ARG(g->r_in > 0 && g->r_out > g->r_in && g->height > 0 && fabs(g->swell) < 1.0,
                  "geometry: bad annulus parameters");
  else
    TTI_CHECK_ARG(g->lx > 0 && g->ly > 0 && g->lz > 0, "geometry: bad box lengths");
  std::unique_ptr<tt_iga_geom> guard(new_geometry(c, g));
  const int st = build_geometry(c, guard.get(), g);
  *out = guard.release();
  return st;
  API_CATCH(c)
}

int tt_iga_geometry_nurbs(tt_iga_ctx *c, const tt_iga_geom_desc *g, const tt_iga_nurbs_patch *patch,
                          tt_iga_geom **out) {
  if (!c || !g || !patch || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  TTI_CHECK_ARG(g->kind == TT_IGA_GEOM_NURBS, "geometry_nurbs: desc kind must be TT_IGA_GEOM_NURBS");
  check_discretisation(g);
  TTI_CHECK_ARG(patch->ctrl && patch->weights, "geometry_nurbs: null control points or weights");
  std::vector<double> packed;
  long long ncp = 1;
  for (int d = 0; d < 3; ++d) {
    const int q = patch->deg[d], m = patch->ncp[d];
    TTI_CHECK_ARG(q >= 1 && q <= TT_IGA_NURBS_MAX_DEGREE, "geometry_nurbs: degree %d of direction %d", q, d);
    TTI_CHECK_ARG(m >= q + 1 && m <= TT_IGA_NURBS_MAX_CP, "geometry_nurbs: %d control points in direction %d", m, d);
    TTI_CHECK_ARG(patch->knots[d], "geometry_nurbs: null knot vector %d", d);
    const double *t = patch->knots[d];
    const int len = m + q + 1;
    for (int k = 0; k < len; ++k) {
      TTI_CHECK_ARG(std::isfinite(t[k]) && (k == 0 || t[k] >= t[k - 1]), "geometry_nurbs: knots %d not nondecreasing",
                    d);
      if (k <= q) TTI_CHECK_ARG(t[k] == 0.0, "geometry_nurbs: knots %d must start with %d zeros", d, q + 1);
      if (k >= len - q - 1) TTI_CHECK_ARG(t[k] == 1.0, "geometry_nurbs: knots %d must end with %d ones", d, q + 1);
      packed.push_back(t[k]);
    }
    ncp *= m;
  }
  for (long long i = 0; i < ncp; ++i) {
    TTI_CHECK_ARG(patch->weights[i] > 0.0 && std::isfinite(patch->weights[i]), "geometry_nurbs: weight %lld", i);
    packed.push_back(patch->weights[i]);
  }
  for (long long i = 0; i < 3 * ncp; ++i) {
    TTI_CHECK_ARG(std::isfinite(patch->ctrl[i]), "geometry_nurbs: control point value %lld", i);
    packed.push_back(patch->ctrl[i]);
  }
  std::unique_ptr<tt_iga_geom> guard(new_geometry(c, g));
  tt_iga_geom *G = guard.get();
  G->nurbs = DBuf(c, packed.size() * sizeof(double));
  c->h2d(G->nurbs.get(), packed.data(), packed.size() * sizeof(double));
  for (int d = 0; d < 3; ++d) {
    G->gp.nd[d] = patch->deg[d];
    G->gp.nc[d] = patch->ncp[d];
  }
  G->gp.nurbs = G->nurbs.d();
  c->sync();  // the packed host copy is released at scope end
  const int st = build_geometry(c, G, g);
  *out = guard.release();
  return st;
  API_CATCH(c)
}

void tt_iga_geom_destroy(tt_iga_geom *g) { delete g; }

int tt_iga_geom_ranks(const tt_iga_geom *g, int ranks[6][2], double max_rel_err[6]) {
  if (!g) return TT_IGA_ERR_ARG;
  for (int f = 0; f < 6; ++f) {
    if (ranks) {
      ranks[f][0] = g->R[f].zero ? 0 : g->R[f].tt.r[1];
      ranks[f][1] = g->R[f].zero ? 0 : g->R[f].tt.r[2];
    }
    if (max_rel_err) max_rel_err[f] = g->R[f].zero ? 0.0 : g->R[f].max_rel_err;
  }
  return TT_IGA_OK;
}

// ------------------------------------------------------------------ assembly

int tt_iga_assemble(tt_iga_ctx *c, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int n_rhs, double round_tol,
                    tt_iga_system **out) {
  return tt_iga_assemble_bc(c, g, rhs, n_rhs, round_tol, nullptr, out);
}

int tt_iga_assemble_bc(tt_iga_ctx *c, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int n_rhs,
                       double round_tol, const tt_iga_bc_desc *bc, tt_iga_system **out) {
  if (!c || !g || !out || (n_rhs > 0 && !rhs) || n_rhs < 1) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  if (g->ctx != c) fail(TT_IGA_ERR_STATE, "assemble: geometry belongs to another context");
  for (int k = 0; k < n_rhs; ++k) {
    TTI_CHECK_ARG(rhs[k].n_modes >= 0 && rhs[k].n_modes <= TT_IGA_MAX_MODES, "assemble: n_modes out of range");
    TTI_CHECK_ARG(rhs[k].kind >= TT_IGA_RHS_MANUFACTURED && rhs[k].kind <= TT_IGA_RHS_RING_LOG,
                  "assemble: unknown right-hand side kind %d", rhs[k].kind);
    TTI_CHECK_ARG(g->desc.kind != TT_IGA_GEOM_NURBS || rhs[k].kind == TT_IGA_RHS_CONSTANT,
                  "assemble: a NURBS patch takes CONSTANT right-hand sides only");
  }
  if (round_tol <= 0) round_tol = 1e-12;
  const int nfull[3] = {g->s[0].n, g->s[1].n, g->s[2].n};
  const BoundaryLayout bl = boundary_layout(bc, nfull);
  auto *S = new tt_iga_system();
  std::unique_ptr<tt_iga_system> guard(S);
  assemble_system(c, g, rhs, n_rhs, round_tol, bl, S);
  const int st = device_status(c);
  *out = guard.release();
  if (st != TT_IGA_OK) {
    c->last_error = "assemble: device-side check failed";
    return st;
  }
  return TT_IGA_OK;
  API_CATCH(c)
}

void tt_iga_system_destroy(tt_iga_system *s) { delete s; }

int tt_iga_system_info(const tt_iga_system *s, int op_ranks[2], int n_rhs_max, int (*rhs_ranks)[2], int modes[3]) {
  if (!s) return TT_IGA_ERR_ARG;
  if (op_ranks) { op_ranks[0] = s->K.r[1]; op_ranks[1] = s->K.r[2]; }
  if (rhs_ranks)
    for (int k = 0; k < n_rhs_max && k < (int)s->F.size(); ++k) {
      rhs_ranks[k][0] = s->F[k].r[1];
      rhs_ranks[k][1] = s->F[k].r[2];
    }
  if (modes)
    for (int d = 0; d < 3; ++d) modes[d] = s->n[d];
  return (int)s->F.size();
}

// --------------------------------------------------------------------- solve

// Solve options with the defaults of tt_iga_solve_opts filled in.
// Default forcing term of the inexact local solves (tt_iga_solve_opts.local_rtol).
constexpr double kDefaultLocalRtol = -1.0;

static tt_iga_solve_opts solve_defaults(const tt_iga_solve_opts *opts) {
  tt_iga_solve_opts o{};
  if (opts) o = *opts;
  if (o.tol <= 0) o.tol = 1e-8;
  if (o.max_sweeps <= 0) o.max_sweeps = 30;
  if (!opts || opts->kickrank == 0) o.kickrank = 4;
  else if (o.kickrank < 0) o.kickrank = 0;
  if (o.max_rank <= 0) o.max_rank = 256;
  o.max_rank = std::min(o.max_rank, 240);
  if (o.local_maxit <= 0) o.local_maxit = 500;
  if (o.local_rtol == 0.0) o.local_rtol = kDefaultLocalRtol;
  TTI_CHECK_ARG(std::isfinite(o.local_rtol) && o.local_rtol < 1.0, "solve: local_rtol %g is not below 1",
                o.local_rtol);
  TTI_CHECK_ARG(o.precision == TT_IGA_FP64 || o.precision == TT_IGA_MIXED_FP32 || o.precision == TT_IGA_MIXED_TF32,
                "solve: precision %d is not one of FP64, MIXED_FP32, MIXED_TF32", o.precision);
  return o;
}

int tt_iga_solve(tt_iga_ctx *c, const tt_iga_system *s, const tt_iga_solve_opts *opts, tt_iga_solution **out,
                 tt_iga_stats *st) {
  if (!c || !s || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  if (s->ctx != c) fail(TT_IGA_ERR_STATE, "solve: system belongs to another context");
  const tt_iga_solve_opts o = solve_defaults(opts);
  TTI_CHECK_ARG(o.rhs_index >= 0 && o.rhs_index < (int)s->F.size(), "solve: rhs_index %d out of range", o.rhs_index);
  auto *U = new tt_iga_solution();
  U->bl = s->bl;
  U->stacked = s->stacked;
  U->stack_mode = s->stack_mode;
  std::unique_ptr<tt_iga_solution> guard(U);
  int status = amen_solve(c, s, o, U, st);
  const int ds = device_status(c);
  *out = guard.release();
  if (ds != TT_IGA_OK && status == TT_IGA_OK) {
    c->last_error = "solve: device-side breakdown flag raised";
    return ds;
  }
  if (status != TT_IGA_OK) c->last_error = "solve: AMEn did not reach the tolerance within max_sweeps";
  return status;
  API_CATCH(c)
}

void tt_iga_solution_destroy(tt_iga_solution *u) { delete u; }

int tt_iga_system_stack(tt_iga_ctx *c, const tt_iga_system *s, int mode, double eps, tt_iga_system **out,
                        double *scales) {
  if (!c || !s || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  if (s->ctx != c) fail(TT_IGA_ERR_STATE, "stack: system belongs to another context");
  auto *B = new tt_iga_system();
  std::unique_ptr<tt_iga_system> guard(B);
  std::vector<double> sc;
  stack_system(c, s, mode, eps > 0 ? eps : 1e-14, B, sc);
  if (scales) std::copy(sc.begin(), sc.end(), scales);
  *out = guard.release();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_solution_unstack(tt_iga_ctx *c, const tt_iga_solution *ub, int k, double scale, tt_iga_solution **out) {
  if (!c || !ub || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  TTI_CHECK_ARG(std::isfinite(scale), "unstack: scale is not finite");
  auto *U = new tt_iga_solution();
  std::unique_ptr<tt_iga_solution> guard(U);
  unstack_solution(c, ub, k, scale, U);
  *out = guard.release();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_solve_block(tt_iga_ctx *c, const tt_iga_system *s, const tt_iga_solve_opts *opts, int mode,
                       tt_iga_solution **out, tt_iga_stats *st, double *rel_res) {
  if (!c || !s || !out) return TT_IGA_ERR_ARG;
  const int nb = (int)s->F.size();
  for (int k = 0; k < nb; ++k) out[k] = nullptr;
  API_TRY
  if (s->ctx != c) fail(TT_IGA_ERR_STATE, "solve_block: system belongs to another context");
  tt_iga_solve_opts o = solve_defaults(opts);
  o.rhs_index = 0;
  o.tol /= sqrt((double)nb);  // block residual = rms of the per-right-hand-side relative residuals
  tt_iga_system B;
  std::vector<double> scale;
  if (mode < 0) mode = kDefaultStackMode;
  stack_system(c, s, mode, 1e-3 * o.tol, &B, scale);
  tt_iga_solution ub;
  ub.bl = s->bl;
  ub.stacked = nb;
  ub.stack_mode = mode;
  int status = amen_solve(c, &B, o, &ub, st);
  const int ds = device_status(c);
  std::vector<std::unique_ptr<tt_iga_solution>> sols(nb);
  for (int k = 0; k < nb; ++k) {
    sols[k].reset(new tt_iga_solution());
    unstack_solution(c, &ub, k, scale[k], sols[k].get());
    if (rel_res) {
      rel_res[k] = exact_residual(c, s, sols[k].get(), k);
    }
  }
  for (int k = 0; k < nb; ++k) out[k] = sols[k].release();
  if (ds != TT_IGA_OK && status == TT_IGA_OK) {
    c->last_error = "solve_block: device-side breakdown flag raised";
    return ds;
  }
  if (status != TT_IGA_OK) c->last_error = "solve_block: AMEn did not reach the tolerance within max_sweeps";
  return status;
  API_CATCH(c)
}

int tt_iga_solution_ranks(const tt_iga_solution *u, int ranks[2]) {
  if (!u || !ranks) return TT_IGA_ERR_ARG;
  ranks[0] = u->u.r[1];
  ranks[1] = u->u.r[2];
  return TT_IGA_OK;
}

int tt_iga_residual(tt_iga_ctx *c, const tt_iga_system *s, const tt_iga_solution *u, int k, double *rel) {
  if (!c || !s || !u || !rel) return TT_IGA_ERR_ARG;
  API_TRY
  TTI_CHECK_ARG(k >= 0 && k < (int)s->F.size(), "residual: rhs %d out of range", k);
  *rel = exact_residual(c, s, u, k);
  if (*rel < 0.0)
    fail(TT_IGA_ERR_TOO_LARGE, "residual: the TT rank of F - K u is above 256 and the problem too large to expand");
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_solution_cores(tt_iga_ctx *c, const tt_iga_solution *u, double *out, size_t cap, int modes[3],
                          int ranks[4]) {
  if (!c || !u) return TT_IGA_ERR_ARG;
  API_TRY
  size_t tot = 0;
  for (int k = 0; k < 3; ++k) tot += u->u.core_elems(k);
  if (modes)
    for (int k = 0; k < 3; ++k) modes[k] = u->u.m[k];
  if (ranks)
    for (int k = 0; k < 4; ++k) ranks[k] = u->u.r[k];
  if (!out) return TT_IGA_OK;
  if (cap < tot) fail(TT_IGA_ERR_TOO_LARGE, "solution_cores: need %zu doubles, got %zu", tot, cap);
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    TTI_CUDA(cudaMemcpyAsync(out + off, u->u.core[k].get(), u->u.core_elems(k) * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
    off += u->u.core_elems(k);
  }
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_import_cores(tt_iga_ctx *c, const tt_iga_system *s, const double *cores, const int modes[3],
                        const int ranks[4], tt_iga_solution **out) {
  if (!c || !s || !cores || !modes || !ranks || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  if (s->ctx != c) fail(TT_IGA_ERR_STATE, "import_cores: system belongs to another context");
  TTI_CHECK_ARG(ranks[0] == 1 && ranks[3] == 1, "import_cores: ranks[0] and ranks[3] must be 1");
  for (int d = 0; d < 3; ++d)
    TTI_CHECK_ARG(modes[d] == s->n[d], "import_cores: mode %d has size %d, the system %d", d, modes[d], s->n[d]);
  for (int k = 1; k <= 2; ++k)
    TTI_CHECK_ARG(ranks[k] >= 1 && ranks[k] <= 256, "import_cores: rank %d = %d outside 1..256", k, ranks[k]);
  auto *U = new tt_iga_solution();
  std::unique_ptr<tt_iga_solution> guard(U);
  U->ctx = c;
  U->p = s->p;
  U->bl = s->bl;
  U->stacked = s->stacked;
  U->stack_mode = s->stack_mode;
  for (int d = 0; d < 3; ++d) U->n[d] = U->u.m[d] = modes[d];
  for (int k = 0; k < 4; ++k) U->u.r[k] = ranks[k];
  U->u.alloc(c);
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    const size_t ne = U->u.core_elems(k);
    for (size_t i = 0; i < ne; ++i)
      TTI_CHECK_ARG(std::isfinite(cores[off + i]), "import_cores: core %d holds a non-finite value", k);
    TTI_CUDA(cudaMemcpyAsync(U->u.core[k].get(), cores + off, ne * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    off += ne;
  }
  c->sync();  // the host array may be released when the call returns
  *out = guard.release();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_solve_from(tt_iga_ctx *c, const tt_iga_system *s, const tt_iga_solve_opts *opts, const tt_iga_solution *u0,
                      tt_iga_solution **out, tt_iga_stats *st) {
  if (!c || !s || !u0 || !out) return TT_IGA_ERR_ARG;
  *out = nullptr;
  API_TRY
  if (s->ctx != c || u0->ctx != c) fail(TT_IGA_ERR_STATE, "solve_from: handles belong to another context");
  const tt_iga_solve_opts o = solve_defaults(opts);
  TTI_CHECK_ARG(o.rhs_index >= 0 && o.rhs_index < (int)s->F.size(), "solve_from: rhs_index %d out of range",
                o.rhs_index);
  for (int d = 0; d < 3; ++d)
    TTI_CHECK_ARG(u0->u.m[d] == s->n[d], "solve_from: the initial iterate's mode %d has size %d, the system %d", d,
                  u0->u.m[d], s->n[d]);
  TTI_CHECK_ARG(u0->stacked == s->stacked, "solve_from: block layouts differ");
  auto *U = new tt_iga_solution();
  U->bl = s->bl;
  U->stacked = s->stacked;
  U->stack_mode = s->stack_mode;
  std::unique_ptr<tt_iga_solution> guard(U);
  int status = amen_solve(c, s, o, U, st, u0);
  const int ds = device_status(c);
  *out = guard.release();
  if (ds != TT_IGA_OK && status == TT_IGA_OK) {
    c->last_error = "solve_from: device-side breakdown flag raised";
    return ds;
  }
  if (status != TT_IGA_OK) c->last_error = "solve_from: AMEn did not reach the tolerance within max_sweeps";
  return status;
  API_CATCH(c)
}

// ---------------------------------------------------------------- evaluation

int tt_iga_eval(tt_iga_ctx *c, const tt_iga_solution *u, int m, const double *xi, double *u_out) {
  if (!c || !u || m < 0 || (m > 0 && (!xi || !u_out))) return TT_IGA_ERR_ARG;
  API_TRY
  TTI_CHECK_ARG(u->stacked == 1, "eval: block solution (slice it with tt_iga_solution_unstack first)");
  eval_points(c, u, m, xi, u_out);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_l2_error(tt_iga_ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_rhs_desc *rhs,
                    double *rel) {
  if (!c || !g || !u || !rhs || !rel) return TT_IGA_ERR_ARG;
  API_TRY
  TTI_CHECK_ARG(u->stacked == 1, "l2_error: block solution (slice it with tt_iga_solution_unstack first)");
  TTI_CHECK_ARG(rhs->kind == TT_IGA_RHS_MANUFACTURED || rhs->kind == TT_IGA_RHS_RING_LOG,
                "l2_error: needs a right-hand side with an exact solution (MANUFACTURED or RING_LOG)");
  TTI_CHECK_ARG(g->desc.kind != TT_IGA_GEOM_NURBS, "l2_error: no exact solution is defined on a NURBS patch");
  if (rhs->kind == TT_IGA_RHS_RING_LOG) {
    const BoundaryLayout &bl = u->bl;
    bool radial_only = bl.lift_dir <= 0 && (bl.lo[0] || bl.hi[0]);
    for (int d = 1; d < 3; ++d)
      radial_only = radial_only && !bl.lo[d] && !bl.hi[d] && bl.flux[2 * d] == 0.0 && bl.flux[2 * d + 1] == 0.0;
    TTI_CHECK_ARG(g->desc.kind == TT_IGA_GEOM_ANNULUS && g->desc.twist == 0.0 && g->desc.swell == 0.0 && radial_only,
                  "l2_error: the ring solution needs the annulus without twist and swell, data on the radial faces "
                  "only and at least one radial Dirichlet face");
  }
  *rel = l2_error(c, g, u, rhs);
  return TT_IGA_OK;
  API_CATCH(c)
}

static bool same_layout(const BoundaryLayout &a, const BoundaryLayout &b) {
  for (int d = 0; d < 3; ++d)
    if (a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d] || a.nfull[d] != b.nfull[d]) return false;
  return a.lift_dir == b.lift_dir && a.lift_lo == b.lift_lo && a.lift_hi == b.lift_hi;
}

int tt_iga_l2_diff(tt_iga_ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_solution *v,
                   double *rel) {
  if (!c || !g || !u || !v || !rel) return TT_IGA_ERR_ARG;
  API_TRY
  TTI_CHECK_ARG(u->stacked == 1 && v->stacked == 1, "l2_diff: block solution (slice it first)");
  TTI_CHECK_ARG(u->p == v->p && u->p == g->desc.p, "l2_diff: degrees differ");
  for (int d = 0; d < 3; ++d)
    TTI_CHECK_ARG(u->n[d] == v->n[d] && v->bl.nfull[d] == g->s[d].n, "l2_diff: discretisations differ");
  TTI_CHECK_ARG(same_layout(u->bl, v->bl), "l2_diff: boundary layouts differ");
  TTI_CHECK_ARG(v->bl.lift_dir < 0, "l2_diff: solutions with a Dirichlet lift are not supported");
  const double r = l2_diff(c, g, u, v);
  if (r < 0.0) fail(TT_IGA_ERR_ARG, "l2_diff: the reference solution v is zero");
  *rel = r;
  return TT_IGA_OK;
  API_CATCH(c)
}

// ------------------------------------------------------------ dense hooks

int tt_iga_densify_operator(tt_iga_ctx *c, const tt_iga_system *s, double *out, size_t cap) {
  if (!c || !s || !out) return TT_IGA_ERR_ARG;
  API_TRY
  const long long N = (long long)s->n[0] * s->n[1] * s->n[2];
  if (N > 4096 || (size_t)(N * N) > cap) fail(TT_IGA_ERR_TOO_LARGE, "densify_operator: N=%lld too large", N);
  DBuf d(c, (size_t)N * N * sizeof(double));
  k_op_dense<<<grid1d(N * N, 256), 256, 0, c->stream>>>(s->K.core[0].d(), s->K.core[1].d(), s->K.core[2].d(), s->n[0],
                                                        s->n[1], s->n[2], s->p, s->K.r[1], s->K.r[2], d.d());
  TTI_LAUNCH();
  c->d2h(out, d.get(), (size_t)N * N * sizeof(double));
  return TT_IGA_OK;
  API_CATCH(c)
}

static int densify_tt(Ctx *c, const TT3 &x, double *out, size_t cap) {
  const long long N = (long long)x.m[0] * x.m[1] * x.m[2];
  if (N > (1LL << 22) || (size_t)N > cap) fail(TT_IGA_ERR_TOO_LARGE, "densify: N=%lld too large", N);
  DBuf d(c, (size_t)N * sizeof(double));
  tt_full(c, x, d.d());
  c->d2h(out, d.get(), (size_t)N * sizeof(double));
  return TT_IGA_OK;
}

int tt_iga_densify_rhs(tt_iga_ctx *c, const tt_iga_system *s, int k, double *out, size_t cap) {
  if (!c || !s || !out) return TT_IGA_ERR_ARG;
  API_TRY
  TTI_CHECK_ARG(k >= 0 && k < (int)s->F.size(), "densify_rhs: rhs %d out of range", k);
  return densify_tt(c, s->F[k], out, cap);
  API_CATCH(c)
}

int tt_iga_densify_solution(tt_iga_ctx *c, const tt_iga_solution *u, double *out, size_t cap) {
  if (!c || !u || !out) return TT_IGA_ERR_ARG;
  API_TRY
  return densify_tt(c, u->u, out, cap);
  API_CATCH(c)
}

int tt_iga_operator_entries(tt_iga_ctx *c, const tt_iga_system *s, int m, const int *rows, const int *cols,
                            double *out) {
  if (!c || !s || m < 0 || (m > 0 && (!rows || !cols || !out))) return TT_IGA_ERR_ARG;
  API_TRY
  if (m == 0) return TT_IGA_OK;
  for (int t = 0; t < m; ++t)
    for (int d = 0; d < 3; ++d)
      TTI_CHECK_ARG(rows[3 * t + d] >= 0 && rows[3 * t + d] < s->n[d] && cols[3 * t + d] >= 0 &&
                        cols[3 * t + d] < s->n[d],
                    "operator_entries: index out of range");
  DBuf dr(c, (size_t)m * 3 * sizeof(int)), dc(c, (size_t)m * 3 * sizeof(int)), dout(c, (size_t)m * sizeof(double));
  c->h2d(dr.get(), rows, (size_t)m * 3 * sizeof(int));
  c->h2d(dc.get(), cols, (size_t)m * 3 * sizeof(int));
  operator_entries(c, s, m, dr.as<int>(), dc.as<int>(), dout.d());
  c->d2h(out, dout.get(), (size_t)m * sizeof(double));
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_vector_entries(tt_iga_ctx *c, const tt_iga_system *s, const tt_iga_solution *u, int k, int m,
                          const int *idx, double *out) {
  if (!c || (!s && !u) || m < 0 || (m > 0 && (!idx || !out))) return TT_IGA_ERR_ARG;
  API_TRY
  if (m == 0) return TT_IGA_OK;
  const TT3 *x;
  if (u) {
    x = &u->u;
  } else {
    TTI_CHECK_ARG(k >= 0 && k < (int)s->F.size(), "vector_entries: rhs %d out of range", k);
    x = &s->F[k];
  }
  for (int t = 0; t < m; ++t)
    for (int d = 0; d < 3; ++d)
      TTI_CHECK_ARG(idx[3 * t + d] >= 0 && idx[3 * t + d] < x->m[d], "vector_entries: index out of range");
  DBuf di(c, (size_t)m * 3 * sizeof(int)), dout(c, (size_t)m * sizeof(double));
  c->h2d(di.get(), idx, (size_t)m * 3 * sizeof(int));
  tt_eval_points(c, *x, m, di.as<int>(), dout.d());
  c->d2h(out, dout.get(), (size_t)m * sizeof(double));
  return TT_IGA_OK;
  API_CATCH(c)
}

// ------------------------------------------------------- kernel-level calls

int tt_iga_basis_tables(tt_iga_ctx *c, int n, int p, int nq, double *pts, double *wts, double *N, double *dN) {
  if (!c || !pts || !wts || !N || !dN) return TT_IGA_ERR_ARG;
  API_TRY
  basis_tables(c, n, p, nq, pts, wts, N, dN);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_geom_points(tt_iga_ctx *c, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int m, const int *idx,
                       double *out, long long *bad) {
  if (!c || !g || m < 0 || (m > 0 && (!idx || !out))) return TT_IGA_ERR_ARG;
  API_TRY
  geom_points(c, g->gp, rhs_params(rhs), g->s[0].pts.d(), g->s[1].pts.d(), g->s[2].pts.d(), m, idx, out);
  const int st = device_status(c);
  if (bad) *bad = (st == TT_IGA_ERR_BAD_GEOMETRY) ? 1 : 0;
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_stiffness_core(tt_iga_ctx *c, int n, int p, int nq, const double *wts, const double *N, const double *dN,
                          const double *G, int r0, int r1, int test_deriv, int trial_deriv, double *M) {
  if (!c || !wts || !N || !dN || !G || !M) return TT_IGA_ERR_ARG;
  API_TRY
  stiffness_core(c, n, p, nq, wts, N, dN, G, r0, r1, test_deriv, trial_deriv, M);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_load_core(tt_iga_ctx *c, int n, int p, int nq, const double *wts, const double *N, const double *G, int r0,
                     int r1, double *F) {
  if (!c || !wts || !N || !G || !F) return TT_IGA_ERR_ARG;
  API_TRY
  load_core(c, n, p, nq, wts, N, G, r0, r1, F);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_round(tt_iga_ctx *c, const int nm[3], const int r[4], const double *const cores[3], double eps,
                 int max_rank, double *const out_cores[3], int out_r[4]) {
  if (!c || !nm || !r || !cores || !out_cores || !out_r) return TT_IGA_ERR_ARG;
  API_TRY
  TTI_CHECK_ARG(r[0] == 1 && r[3] == 1 && r[1] >= 1 && r[2] >= 1 && r[1] <= 256 && r[2] <= 256,
                "round: ranks must be 1, r1, r2, 1 with r <= 256");
  TT3 x;
  for (int k = 0; k < 3; ++k) {
    TTI_CHECK_ARG(nm[k] >= 1 && cores[k] && out_cores[k], "round: bad mode size or core pointer");
    x.m[k] = nm[k];
  }
  for (int k = 0; k < 4; ++k) x.r[k] = r[k];
  x.alloc(c);
  for (int k = 0; k < 3; ++k)
    TTI_CUDA(cudaMemcpyAsync(x.core[k].get(), cores[k], x.core_elems(k) * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  tt_round(c, x, eps, max_rank);
  for (int k = 0; k < 3; ++k)
    TTI_CUDA(cudaMemcpyAsync(out_cores[k], x.core[k].get(), x.core_elems(k) * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
  for (int k = 0; k < 4; ++k) out_r[k] = x.r[k];
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_gemm_f64(tt_iga_ctx *c, int ta, int tb, int m, int n, int k, double alpha, const double *A, int lda,
                    const double *B, int ldb, double beta, double *C, int ldc) {
  if (!c || !C || (k > 0 && (!A || !B)) || m < 0 || n < 0 || k < 0 || ldc < n) return TT_IGA_ERR_ARG;
  API_TRY
  gemm<double>(c, ta != 0, tb != 0, m, n, k, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_qr(tt_iga_ctx *c, int m, int k, const double *A, int lda, double *Q, double *R) {
  if (!c || !A || !Q || !R || lda < k) return TT_IGA_ERR_ARG;
  API_TRY
  qr(c, m, k, A, lda, Q, R);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_blockband_solve(tt_iga_ctx *c, int rl, int rr, int Rl, int Rr, int n, int p, const double *PhiL,
                           const double *A, const double *PhiR, const double *r, double *z) {
  if (!c || !PhiL || !A || !PhiR || !r || !z || rl < 1 || rr < 1 || Rl < 1 || Rr < 1) return TT_IGA_ERR_ARG;
  if (!ttiga::bb_eligible(rl * rr, n, p)) return TT_IGA_ERR_TOO_LARGE;
  API_TRY
  ttiga::BandCore core{A, nullptr, Rl, n, 2 * p + 1, p, Rr};
  ttiga::BBPrec P;
  ttiga::bb_prec_build(c, PhiL, rl, core, PhiR, rr, P);
  ttiga::bb_solve_once<double>(c, P, rl, rr, n, p, r, z);
  c->sync();
  return TT_IGA_OK;
  API_CATCH(c)
}

int tt_iga_svd_small(tt_iga_ctx *c, int k, const double *A, double *U, double *s, double *V) {
  if (!c || !A || !U || !s || !V) return TT_IGA_ERR_ARG;
  API_TRY
  svd_small(c, k, A, U, s, V);
  return device_status(c);
  API_CATCH(c)
}

int tt_iga_svd_small_noalloc(void *stream, int k, const double *A, double *U, double *s, double *V, int *info) {
  try {
    return svd_small_noalloc(static_cast<cudaStream_t>(stream), k, A, U, s, V, info);
  } catch (...) {
    return TT_IGA_ERR_CUDA;
  }
}

int tt_iga_maxvol(tt_iga_ctx *c, int m, int r, const double *U, double delta, int maxit, int *rows, double *B) {
  if (!c || !U || !rows || !B) return TT_IGA_ERR_ARG;
  API_TRY
  long long off = 0, roff = 0;
  maxvol_batched(c, 1, &m, &r, &off, U, B, rows, &roff, delta, maxit);
  return device_status(c);
  API_CATCH(c)
}

}  // extern "C"
