// AMEn TT linear solver for the SPD system K u = F (Section 4.1.2).
//
// The paper solves with TT-Toolbox's amen_solve: one TT core of u is updated
// at a time by minimising the residual over it, and an enrichment step with a
// low-rank approximation of the residual controls rank growth.  This is a GPU
// implementation of that scheme (Dolgov and Savostyanov 2014) for d = 3:
//
//   forward sweep k = 1, 2, 3:
//     local system  B_k = PhiL_k (x) A_k (x) PhiR_k, rhs_k = PsiL_k F_k PsiR_k
//     local solve   PCG with a band block-Jacobi preconditioner (FP64), or
//                   FP32 PCG inside FP64 iterative refinement (mixed)
//     truncation    QR + SVD of the (r_{k-1} n_k) x r_k solution, smallest rank
//                   whose local residual stays below the truncation tolerance
//     enrichment    append the residual projected onto the right interface of
//                   a rank-rho residual approximation z, re-orthogonalise (QR)
//     z update      core k of z = residual projected on z's own interfaces
//     interfaces    left interfaces of u and z for core k + 1
//   backward pass: right-orthogonalise cores 3, 2 of u and z, refresh the
//   right interfaces.
//   stop:  exact ||F - K u|| / ||F|| <= tol (TT arithmetic with QR
//   orthogonalisation) when the residual's rank allows it, otherwise the
//   largest relative local residual of the sweep.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "amen.cuh"
#include "amen_ops.cuh"
#include "bbprec.cuh"
#include "linalg.cuh"
#include "pcg_fused.cuh"
#include "tt.cuh"

namespace ttiga {

namespace {

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; }
};

void random_tt(Ctx *c, TT3 &x, const int m[3], int r1, int r2, uint64_t seed) {
  SplitMix64 rng{seed};
  for (int k = 0; k < 3; ++k) x.m[k] = m[k];
  x.r[0] = 1; x.r[1] = r1; x.r[2] = r2; x.r[3] = 1;
  x.alloc(c);
  for (int k = 0; k < 3; ++k) {
    std::vector<double> h(x.core_elems(k));
    for (auto &v : h) v = rng.uniform();
    c->h2d(x.core[k].get(), h.data(), h.size() * sizeof(double));
  }
}

DBuf ones(Ctx *c) {
  DBuf d(c, sizeof(double));
  const double one = 1.0;
  c->h2d(d.get(), &one, sizeof one);
  return d;
}

__global__ void k_sub(const double *a, double *b, long long n) {  // b = a - b
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i] - b[i];
}

template <typename T>
__global__ void k_pcg_xr(T *x, T *r, const T *p, const T *q, const double *rz, const double *pq, long long n) {
  const double alpha = (*pq != 0.0) ? *rz / *pq : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] += (T)alpha * p[i];
    r[i] -= (T)alpha * q[i];
  }
}

template <typename T>
__global__ void k_pcg_p(T *p, const T *z, const double *rz_new, const double *rz_old, long long n) {
  const double beta = (*rz_old != 0.0) ? *rz_new / *rz_old : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + (T)beta * p[i];
}

// Deterministic dot product of FP32 or FP64 vectors accumulated in FP64.
template <typename T>
__global__ void k_dot_part(const T *x, const T *y, long long n, double *part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += (double)x[i] * (double)y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
__global__ void k_dot_final(const double *part, int np, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < np; ++i) t += part[i];
    *out = t;
  }
}

template <typename T> void dot_dev(Ctx *c, const T *x, const T *y, long long n, double *out, double *part) {
  const int nb = (int)std::min<long long>(128, std::max<long long>(1, (n + 255) / 256));
  k_dot_part<T><<<nb, 256, 0, c->stream>>>(x, y, n, part);
  TTI_LAUNCH();
  k_dot_final<<<1, 32, 0, c->stream>>>(part, nb, out);
  TTI_LAUNCH();
}

// ||F - K u|| / Fnorm for the band TT operator K (cores Kc, ranks R) and a TT u.
// The TT of F - K u has ranks f + R r; while they stay within the QR limit (256)
// its norm comes from orthogonalisation (TT arithmetic).  Above it, F and K u are
// expanded to dense vectors by GEMM chains and subtracted entry by entry (the
// difference is resolved to FP64 rounding of ||F||), as long as the vectors
// (2^22 entries) and the cores of K u (2^27 doubles) stay small; otherwise -1.
double residual_norm(Ctx *c, const TT3 &F, double Fnorm, const TT3 &K, const int n[3], int b, int p, const TT3 &u) {
  TT3 Ku;
  for (int k = 0; k < 3; ++k) Ku.m[k] = n[k];
  for (int k = 0; k < 4; ++k) Ku.r[k] = K.r[k] * u.r[k];
  const bool tt_ok = Ku.r[1] + F.r[1] <= 256 && Ku.r[2] + F.r[2] <= 256;
  const long long N = (long long)n[0] * n[1] * n[2];
  size_t ku_max = 0;
  for (int k = 0; k < 3; ++k) ku_max = std::max(ku_max, Ku.core_elems(k));
  if (!tt_ok && (N > (1LL << 22) || ku_max > ((size_t)1 << 27))) return -1.0;
  Ku.alloc(c);
  for (int k = 0; k < 3; ++k) {
    BandCore A{K.core[k].d(), nullptr, K.r[k], n[k], b, p, K.r[k + 1]};
    tt_matvec_core(c, A, u.core[k].d(), u.r[k], u.r[k + 1], Ku.core[k].d());
  }
  if (tt_ok) {
    TT3 W;
    tt_sum(c, F, 1.0, Ku, -1.0, W);
    return tt_norm(c, W) / Fnorm;
  }
  DBuf fd(c, N * sizeof(double)), kd(c, N * sizeof(double));
  tt_dense(c, F, fd.d());
  tt_dense(c, Ku, kd.d());
  k_sub<<<grid1d(N, 256), 256, 0, c->stream>>>(fd.d(), kd.d(), N);
  TTI_LAUNCH();
  return host_nrm2(c, kd.d(), N) / Fnorm;
}

}  // namespace

struct Amen {
  Ctx *c;
  const tt_iga_system *S;
  const TT3 &F;
  double Fnorm;
  tt_iga_solve_opts o;
  TT3 u, z;
  BandCore A[3];
  DBuf A32[3];
  int R[4], f[4];
  DBuf PhiL[3], PhiR[3], PsiL[3], PsiR[3], PhiLz[3], PhiRz[3], PsiLz[3], PsiRz[3];
  Work<double> w64;
  Work<float> w32;
  tt_iga_stats st{};
  double last_local = 0.0;
  bool last_pcg_converged = false;
  int trunc_hint[2] = {0, 0};  // rank chosen by the last truncation of cores 0 and 1
  // scratch scalars on the device: [0] rz, [1] pq, [2] rz_new, [8..] partials
  DBuf scal;
  // fork / join events of the preconditioner build on a helper stream (created on first use)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // The enrichment chain (z) on a helper stream: its work area, fork / join events, and
  // whether a join is pending.
  Work<double> wz;
  cudaEvent_t ev_zin = nullptr, ev_zout = nullptr;
  bool z_pending = false;

  const TT3 *u0 = nullptr;  // initial iterate (warm start), or null for a random rank-2 TT

  Amen(Ctx *c_, const tt_iga_system *s, const tt_iga_solve_opts &opts, const TT3 *start)
      : c(c_), S(s), F(s->F[opts.rhs_index]), Fnorm(s->F_norm[opts.rhs_index]), o(opts), u0(start), w64{c_}, w32{c_}, wz{c_} {
    for (int k = 0; k < 4; ++k) { R[k] = S->K.r[k]; f[k] = F.r[k]; }
    for (int k = 0; k < 3; ++k) {
      A[k].A = S->K.core[k].d();
      A[k].A32 = nullptr;
      A[k].Rl = R[k]; A[k].Rr = R[k + 1];
      A[k].n = S->n[k]; A[k].b = S->b; A[k].p = S->p;
    }
    scal = DBuf(c, 256 * sizeof(double));
    if (o.precision != TT_IGA_FP64) {
      for (int k = 0; k < 3; ++k) {
        const long long ne = (long long)S->K.core_elems(k);
        A32[k] = DBuf(c, ne * sizeof(float));
        convert_f64_to_f32(c, A[k].A, A32[k].as<float>(), ne);
        A[k].A32 = A32[k].as<float>();
      }
    }
  }

  ~Amen() {
    if (z_pending) cudaStreamWaitEvent(c->stream, ev_zout, 0);  // helper reads end before the frees
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_zin) cudaEventDestroy(ev_zin);
    if (ev_zout) cudaEventDestroy(ev_zout);
  }

  // Context of the enrichment chain: a helper stream under the same conditions as the
  // preconditioner build (one live context, no caller allocator, no stage timers), else c.
  // The z cores and their interfaces depend on u only through the truncated solution and
  // u's interfaces, so the z chain of a step (projected residual and its QR; the backward
  // orthogonalisation of z) overlaps the u chain and joins before its result is read.
  Ctx *z_ctx() {
    if (o.kickrank <= 0 || c->alloc_fn || o.verbose >= 2 || g_live_contexts.load(std::memory_order_relaxed) > 1)
      return c;
    return c->sub(1);  // helper 0 builds preconditioners
  }
  void z_fork(Ctx *h) {
    if (!ev_zin) {
      TTI_CUDA(cudaEventCreateWithFlags(&ev_zin, cudaEventDisableTiming));
      TTI_CUDA(cudaEventCreateWithFlags(&ev_zout, cudaEventDisableTiming));
    }
    TTI_CUDA(cudaEventRecord(ev_zin, c->stream));
    TTI_CUDA(cudaStreamWaitEvent(h->stream, ev_zin, 0));
  }
  void z_done(Ctx *h) {
    TTI_CUDA(cudaEventRecord(ev_zout, h->stream));
    z_pending = true;
  }
  void z_join() {
    if (!z_pending) return;
    TTI_CUDA(cudaStreamWaitEvent(c->stream, ev_zout, 0));
    z_pending = false;
  }
  // Joins on scope exit, also when an exception unwinds the step: the buffers the helper
  // reads are freed on c afterwards.
  struct ZJoinGuard {
    Amen *a;
    ~ZJoinGuard() {
      if (a->z_pending) cudaStreamWaitEvent(a->c->stream, a->ev_zout, 0);
      a->z_pending = false;
    }
  };
  // Backward orthogonalisation step of z at core k.  Its replaced core k-1 is handed to the
  // helper first, so that the old buffer is freed in the helper's stream order.
  void z_orth(int k) {
    Ctx *h = z_ctx();
    if (h == c) {
      orth_right_step(c, z, k);
      return;
    }
    z_fork(h);
    z.core[k - 1].rehome(h);
    orth_right_step(h, z, k);
    z.core[k - 1].rehome(c);
    z_done(h);
  }
  Amen(const Amen &) = delete;
  Amen &operator=(const Amen &) = delete;

  int rl(int k) const { return u.r[k]; }
  int rr(int k) const { return u.r[k + 1]; }
  int n(int k) const { return S->n[k]; }

  void right_interfaces(int k) {  // from core k (1 or 2) into index k-1
    PhiR[k - 1] = DBuf(c, (size_t)u.r[k] * R[k] * u.r[k] * sizeof(double));
    right_update(c, w64, u.core[k].d(), u.r[k], u.r[k + 1], A[k], PhiR[k].d(), u.core[k].d(), u.r[k], u.r[k + 1],
                 PhiR[k - 1].d());
    PsiR[k - 1] = DBuf(c, (size_t)u.r[k] * f[k] * sizeof(double));
    rhs_right_update(c, w64, u.core[k].d(), u.r[k], u.r[k + 1], F.core[k].d(), f[k], n(k), f[k + 1], PsiR[k].d(),
                     PsiR[k - 1].d());
    // z's interfaces on the enrichment stream (after z's core k there, after u's core k here);
    // read on c only by the enrichment of a truncation, which joins first
    Ctx *h = z_ctx();
    Work<double> &w = (h == c) ? w64 : wz;
    if (h != c) {
      wz.c = h;
      z_fork(h);
    }
    DBuf phz(h, (size_t)z.r[k] * R[k] * u.r[k] * sizeof(double)), psz(h, (size_t)z.r[k] * f[k] * sizeof(double));
    right_update(h, w, z.core[k].d(), z.r[k], z.r[k + 1], A[k], PhiRz[k].d(), u.core[k].d(), u.r[k], u.r[k + 1],
                 phz.d());
    rhs_right_update(h, w, z.core[k].d(), z.r[k], z.r[k + 1], F.core[k].d(), f[k], n(k), f[k + 1], PsiRz[k].d(),
                     psz.d());
    if (h != c) {
      phz.rehome(c);
      psz.rehome(c);
      z_done(h);
    }
    PhiRz[k - 1] = std::move(phz);
    PsiRz[k - 1] = std::move(psz);
  }

  void left_interfaces(int k) {  // from core k (0 or 1) into index k+1
    PhiL[k + 1] = DBuf(c, (size_t)u.r[k + 1] * R[k + 1] * u.r[k + 1] * sizeof(double));
    left_update(c, w64, u.core[k].d(), u.r[k], u.r[k + 1], PhiL[k].d(), A[k], u.core[k].d(), u.r[k], u.r[k + 1],
                PhiL[k + 1].d());
    PsiL[k + 1] = DBuf(c, (size_t)u.r[k + 1] * f[k + 1] * sizeof(double));
    rhs_left_update(c, w64, u.core[k].d(), u.r[k], u.r[k + 1], PsiL[k].d(), F.core[k].d(), f[k], n(k), f[k + 1],
                    PsiL[k + 1].d());
    // z's interfaces on the enrichment stream, overlapping the next local solve; read there by
    // the next step's z chain, and on c by the last core's z update after a join
    Ctx *h = z_ctx();
    Work<double> &w = (h == c) ? w64 : wz;
    if (h != c) {
      wz.c = h;
      z_fork(h);
    }
    DBuf phz(h, (size_t)z.r[k + 1] * R[k + 1] * u.r[k + 1] * sizeof(double)),
        psz(h, (size_t)z.r[k + 1] * f[k + 1] * sizeof(double));
    left_update(h, w, z.core[k].d(), z.r[k], z.r[k + 1], PhiLz[k].d(), A[k], u.core[k].d(), u.r[k], u.r[k + 1],
                phz.d());
    rhs_left_update(h, w, z.core[k].d(), z.r[k], z.r[k + 1], PsiLz[k].d(), F.core[k].d(), f[k], n(k), f[k + 1],
                    psz.d());
    if (h != c) {
      phz.rehome(c);
      psz.rehome(c);
      z_done(h);
    }
    PhiLz[k + 1] = std::move(phz);
    PsiLz[k + 1] = std::move(psz);
  }

  void init() {
    const int m[3] = {n(0), n(1), n(2)};
    if (u0) {
      tt_copy(c, *u0, u);
    } else {
      const int r0 = std::max(1, std::min(2, std::min(m[0], m[2])));
      random_tt(c, u, m, r0, r0, 0x5EED5EEDULL + 31 * o.rhs_index);
    }
    tt_orth_rl(c, u);
    const int rho = std::max(0, o.kickrank);
    if (rho > 0) {
      const int zr = std::min(rho, std::min(m[0], m[2]));
      random_tt(c, z, m, zr, zr, 0xC0FFEEULL + 17 * o.rhs_index);
      tt_orth_rl(c, z);
    } else {
      random_tt(c, z, m, 1, 1, 0xC0FFEEULL);
    }
    PhiL[0] = ones(c); PsiL[0] = ones(c); PhiLz[0] = ones(c); PsiLz[0] = ones(c);
    PhiR[2] = ones(c); PsiR[2] = ones(c); PhiRz[2] = ones(c); PsiRz[2] = ones(c);
    right_interfaces(2);
    right_interfaces(1);
  }

  // B x for core k in FP64
  void matvec64(int k, const double *x, double *y) {
    apply_local<double>(c, w64, PhiL[k].d(), rl(k), rl(k), A[k], A[k].A, PhiR[k].d(), rr(k), rr(k), x, y);
    st.local_matvecs++;
    st.local_matvecs_fp64++;
  }

  // Local residual r = rhs - B x, returns ||r||.
  double residual64(int k, const double *rhs, const double *x, double *r) {
    const long long N = (long long)rl(k) * n(k) * rr(k);
    matvec64(k, x, r);
    k_sub<<<grid1d(N, 256), 256, 0, c->stream>>>(rhs, r, N);
    TTI_LAUNCH();
    return host_nrm2(c, r, N);
  }

  // PCG on B d = r (type T), d starts at zero; one cooperative launch for all
  // iterations.  Absolute tolerance tol on ||r - B d||.  Returns iterations.
  template <typename T>
  int pcg(int k, const T *PhiLk, const T *PhiRk, const T *Ak, const float *L, const BBPrec *bb, const T *b, T *x,
          double tol, int maxit) {
    const long long N = (long long)rl(k) * n(k) * rr(k);
    PcgArgs<T> a{};
    a.PhiL = PhiLk; a.PhiR = PhiRk; a.A = Ak; a.Lf = L; a.b = b; a.x = x;
    if (bb) {
      a.edge = 1;
      a.bbLinv = bb->Linv.as<float>(); a.bbUl = bb->Ul.as<float>(); a.bbUr = bb->Ur.as<float>();
      a.bbM = bb->M;
      a.bbS = bb->S;
    }
    a.rl = rl(k); a.rr = rr(k); a.Rl = R[k]; a.Rr = R[k + 1]; a.n = n(k); a.p = S->p;
    a.tol2 = tol * tol;
    a.maxit = maxit;
    a.tc = (sizeof(T) == 4 && o.precision == TT_IGA_MIXED_TF32) ? 1 : 0;
    const int grid = pcg_fused_grid<T>(c, a);
    const size_t slab_scratch = a.dense_off >= 0 ? 0 : (size_t)grid * a.dense_stride;  // none in shared memory
    DBuf vec(c, 5 * N * sizeof(T)), scr(c, slab_scratch * sizeof(T)), aux(c, (3 * (size_t)grid + 8) * sizeof(double));
    a.r = vec.as<T>(); a.z = a.r + N; a.pv = a.z + N; a.pv2 = a.pv + N; a.q = a.pv2 + N;
    a.scratch = scr.as<T>();
    a.part = aux.d();
    a.out = aux.d() + 3 * grid;
    a.bar = reinterpret_cast<Barrier *>(aux.d() + 3 * grid + 2);
    a.err = reinterpret_cast<int *>(aux.d() + 3 * grid + 3);
    c->zero(a.err, sizeof(int));
    DBuf trace;
    if (o.verbose >= 2) {
      a.trace_cap = 2 + 2 * 128 + 8;
      trace = DBuf(c, a.trace_cap * sizeof(unsigned long long));
      a.trace = trace.as<unsigned long long>();
    }
    pcg_fused<T>(c, a, grid);
    double hout[4];
    c->d2h(hout, a.out, 4 * sizeof(double));
    if (o.verbose >= 2) {
      std::vector<unsigned long long> tr(a.trace_cap);
      c->d2h(tr.data(), a.trace, tr.size() * sizeof(unsigned long long));
      const int iters = std::min((int)hout[0], 128);
      double ph[2] = {0, 0};
      for (int i = 0; i < iters; ++i) {
        ph[0] += (double)(tr[2 + 2 * i] - tr[1 + 2 * i]);
        ph[1] += (double)(tr[3 + 2 * i] - tr[2 + 2 * i]);
      }
      fprintf(stderr, "[tt_iga pcg] core %d %s %s grid %d slab %d n %d rl %d rr %d R %d/%d it %d init %.1f us, per "
                      "iteration dense %.1f precond %.1f us\n",
              k, sizeof(T) == 8 ? "fp64" : (a.tc ? "fp32+tf32-tc" : "fp32"), a.edge ? "block-band" : "band-jacobi", grid,
              a.slab, a.n, a.rl, a.rr,
              a.Rl, a.Rr, (int)hout[0],
              (tr[1] - tr[0]) * 1e-3, iters ? ph[0] / iters * 1e-3 : 0.0, iters ? ph[1] / iters * 1e-3 : 0.0);
      if (a.edge) {
        const unsigned long long *sb = tr.data() + 2 + 2 * 128;
        fprintf(stderr, "[tt_iga pcg]   block-band apply: update %.1f, forward %.1f, top %.1f, backward %.1f, "
                        "scatter %.1f us\n",
                (sb[1] - sb[0]) * 1e-3, (sb[2] - sb[1]) * 1e-3, (sb[3] - sb[2]) * 1e-3, (sb[4] - sb[3]) * 1e-3,
                (sb[6] - sb[5]) * 1e-3);
      }
    }
    int err = 0;
    memcpy(&err, &hout[3], sizeof(int));
    if (err)
      fail(TT_IGA_ERR_TIMEOUT, "pcg: a %s wait ran out", err == 3 ? "tensor-core completion" : "grid barrier");
    const int it = (int)hout[0];
    last_pcg_converged = (it < maxit) && hout[1] <= a.tol2;
    {
      // algorithmic FLOPs per PCG iteration: right-interface, band and left-interface stages
      // of the local matvec plus the two band triangular solves of the preconditioner
      const double rl_ = a.rl, rr_ = a.rr, n_ = a.n, Rl_ = a.Rl, Rr_ = a.Rr, b_ = 2.0 * a.p + 1.0;
      const double m_ = rl_ * rr_;
      const double f_prec = a.edge ? 4.0 * n_ * (a.p + 1) * m_ * m_ : 4.0 * m_ * n_ * (a.p + 1);
      const double f_iter = 2.0 * rl_ * n_ * rr_ * Rr_ * rr_ + 2.0 * Rl_ * rl_ * n_ * rr_ * b_ * Rr_ +
                            2.0 * rl_ * n_ * rr_ * Rl_ * rl_ + f_prec + 10.0 * N;
      prof_set_last_work(c, PROF_PCG_FUSED, f_iter * it);
    }
    st.local_matvecs += it;
    if (sizeof(T) == 8) st.local_matvecs_fp64 += it;
    if (a.tc) st.local_matvecs_tensor += it;
    return it;
  }

  Work<double> &work(double *) { return w64; }
  Work<float> &work(float *) { return w32; }

  // Solve the local system of core k for x (in/out).  Returns the residual before the solve.
  // With check_below > 0, a residual at or below it returns at once with *checked = true
  // and x untouched (the caller then evaluates the exact TT residual).
  double local_solve(int k, const double *rhs, double *x, double tol_abs, double check_below = -1.0,
                     bool *checked = nullptr) {
    const long long N = (long long)rl(k) * n(k) * rr(k);
    DBuf rbuf(c, N * sizeof(double));
    const size_t Lsz = (size_t)n(k) * (S->p + 1) * rl(k) * rr(k);
    // Small interface blocks (m = rl rr <= 8): exact block-band preconditioner.
    // Otherwise band block-Jacobi over the interface pairs.
    const bool edge = bb_eligible(rl(k) * rr(k), n(k), S->p);
    BBPrec bb;
    DBuf L;
    // The lazy convergence check (check_below > 0) usually returns here: its residual is
    // evaluated before any preconditioner is built, so a converged solve builds none.
    double res0 = -1.0;
    if (checked) {
      res0 = residual64(k, rhs, x, rbuf.d());
      if (res0 <= check_below) {
        *checked = true;
        return res0;
      }
    }
    // The preconditioner does not depend on the initial residual: it is built on a
    // helper stream while this stream evaluates that residual (whose norm the host
    // waits for); this stream joins the helper before anything uses or frees it.
    // Not when the residual is known already (the check above).
    // Only while this is the one live context: several contexts (batch lanes, a
    // server's lanes) already overlap their work, and the extra stream and events
    // of every local solve then cost more than they hide.  Sequential too with a
    // caller-supplied allocator, whose streams helpers must not touch, and under
    // the verbose stage timers.
    Ctx *const parent = c;
    Ctx *hb = (res0 >= 0.0 || c->alloc_fn || o.verbose >= 2 || g_live_contexts.load(std::memory_order_relaxed) > 1)
                  ? c
                  : c->sub(0);
    if (hb != parent) {
      if (!ev_in) {
        TTI_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
        TTI_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
      }
      TTI_CUDA(cudaEventRecord(ev_in, parent->stream));
      TTI_CUDA(cudaStreamWaitEvent(hb->stream, ev_in, 0));
    }
    if (edge) {
      cudaEvent_t ev[2] = {nullptr, nullptr};
      if (o.verbose >= 2) {
        TTI_CUDA(cudaEventCreate(&ev[0]));
        TTI_CUDA(cudaEventCreate(&ev[1]));
        TTI_CUDA(cudaEventRecord(ev[0], c->stream));
      }
      bb_prec_build(hb, PhiL[k].d(), rl(k), A[k], PhiR[k].d(), rr(k), bb);
      if (o.verbose >= 2) {
        float ms = 0.f;
        TTI_CUDA(cudaEventRecord(ev[1], c->stream));
        TTI_CUDA(cudaEventSynchronize(ev[1]));
        TTI_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        fprintf(stderr, "[tt_iga pcg] core %d block-band preconditioner (m %d n %d): %d super-rows of %d, %d "
                        "reduction levels, build and factor %.1f us\n", k, rl(k) * rr(k), n(k), bb.S, bb.q, bb.levels,
                ms * 1e3);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
      }
    } else {
      L = DBuf(hb, Lsz * sizeof(float));
      precond_build<float>(hb, PhiL[k].d(), rl(k), A[k], PhiR[k].d(), rr(k), L.as<float>());
    }
    if (hb != parent) {
      TTI_CUDA(cudaEventRecord(ev_out, hb->stream));
      L.rehome(parent);
      bb.Linv.rehome(parent);
      bb.Ul.rehome(parent);
      bb.Ur.rehome(parent);
    }
    if (res0 < 0.0) {
      try {
        res0 = residual64(k, rhs, x, rbuf.d());
      } catch (...) {
        if (hb != parent) cudaStreamWaitEvent(parent->stream, ev_out, 0);
        throw;
      }
    }
    if (hb != parent) TTI_CUDA(cudaStreamWaitEvent(parent->stream, ev_out, 0));
    if (res0 <= tol_abs) return res0;
    // inexact local solve (local_rtol > 0): a local system is solved only to local_rtol times its
    // initial residual when that is above the absolute bound.  Far from convergence (early sweeps,
    // poor interfaces) this saves most of the PCG iterations; the exact global residual decides
    // convergence, so the late sweeps, whose initial residuals are small, solve to full accuracy.
    if (o.local_rtol > 0.0) tol_abs = std::max(tol_abs, o.local_rtol * res0);
    const int maxit = o.local_maxit;
    const BBPrec *bbp = edge ? &bb : nullptr;
    if (o.precision == TT_IGA_FP64) {
      // preconditioner factors in FP32 (see pcg_fused_impl.cuh, bbprec.cu)
      DBuf d(c, N * sizeof(double));
      // correction form: B d = r, x += d, checked in FP64
      // correction form B d = r; in FP64 the PCG recurrence residual is the residual of
      // x + d to working accuracy, so an explicit check is only needed when PCG stopped early
      for (int rep = 0; rep < 3; ++rep) {
        pcg<double>(k, PhiL[k].d(), PhiR[k].d(), A[k].A, L.as<float>(), bbp, rbuf.d(), d.d(), 0.5 * tol_abs, maxit);
        axpy<double>(c, N, 1.0, d.d(), x);
        if (last_pcg_converged) break;
        if (residual64(k, rhs, x, rbuf.d()) <= tol_abs) break;
      }
    } else {
      // FP32 PCG on the correction inside FP64 iterative refinement.
      DBuf d32(c, N * sizeof(float)), r32(c, N * sizeof(float)), d64(c, N * sizeof(double));
      const long long nl = (long long)rl(k) * R[k] * rl(k), nr = (long long)rr(k) * R[k + 1] * rr(k);
      DBuf pl(c, nl * sizeof(float)), pr(c, nr * sizeof(float));
      convert_f64_to_f32(c, PhiL[k].d(), pl.as<float>(), nl);
      convert_f64_to_f32(c, PhiR[k].d(), pr.as<float>(), nr);
      double res = res0;
      for (int rep = 0; rep < 12 && res > tol_abs; ++rep) {
        // scale the residual to unit norm so FP32 keeps its relative precision
        convert_f64_to_f32(c, rbuf.d(), r32.as<float>(), N);
        scale<float>(c, r32.as<float>(), N, (float)(1.0 / res));
        pcg<float>(k, pl.as<float>(), pr.as<float>(), A[k].A32, L.as<float>(), bbp, r32.as<float>(), d32.as<float>(),
                   std::max(1e-5, 0.5 * tol_abs / res), maxit);
        convert_f32_to_f64(c, d32.as<float>(), d64.d(), N);
        axpy<double>(c, N, res, d64.d(), x);
        res = residual64(k, rhs, x, rbuf.d());
      }
    }
    return res0;
  }

  // Truncate the solution x of core k (k < 2) and enrich; updates u cores k, k+1.
  void truncate_enrich(int k, const double *rhs, const double *x, double tol_trunc) {
    z_join();  // z's interfaces from the enrichment stream
    const int a = rl(k), nk = n(k), b = rr(k);
    const int rows = a * nk;
    DBuf Q(c, (size_t)rows * b * sizeof(double)), Rm(c, (size_t)b * b * sizeof(double));
    qr(c, rows, b, x, b, Q.d(), Rm.d());
    DBuf Ur(c, (size_t)b * b * sizeof(double)), Sv(c, (size_t)b * sizeof(double)), V(c, (size_t)b * b * sizeof(double));
    svd_small(c, b, Rm.d(), Ur.d(), Sv.d(), V.d());
    std::vector<double> s(b);
    c->d2h(s.data(), Sv.d(), b * sizeof(double));
    // SVt[j][l] = s_j V[l][j]
    DBuf SVt(c, (size_t)b * b * sizeof(double));
    svt(c, Sv.d(), V.d(), b, b, SVt.d());
    DBuf QU(c, (size_t)rows * b * sizeof(double));
    gemm<double>(c, false, false, rows, b, b, 1.0, Q.d(), b, 0, Ur.d(), b, 0, 0.0, QU.d(), b, 0, 1);
    // numerical rank
    int rmax = b;
    while (rmax > 1 && s[rmax - 1] <= 1e-15 * s[0]) --rmax;
    const long long N = (long long)rows * b;
    DBuf xt(c, N * sizeof(double)), rt(c, N * sizeof(double));
    auto res_at = [&](int r) {
      gemm<double>(c, false, false, rows, b, r, 1.0, QU.d(), b, 0, SVt.d(), b, 0, 0.0, xt.d(), b, 0, 1);
      return residual64(k, rhs, xt.d(), rt.d());
    };
    // smallest rank whose local residual meets the tolerance (binary search, the residual
    // being non-increasing in the rank); the previous sweep's rank of this core is tried
    // first, which settles the search in two evaluations when the rank is unchanged
    int lo = 1, hi = rmax;
    const int hint = trunc_hint[k];
    bool done = false;
    if (hint >= 1 && hint <= rmax) {
      if (res_at(hint) <= tol_trunc) {
        hi = hint;
        if (hint == 1 || res_at(hint - 1) > tol_trunc) {
          lo = hint;
          done = true;
        } else {
          hi = hint - 1;
        }
      } else {
        lo = hint + 1;
        if (lo > rmax) {
          lo = rmax;  // cannot meet the tolerance: keep everything
          done = true;
        }
      }
    }
    if (!done) {
      if (hint < 1 || hint > rmax) {
        if (res_at(hi) > tol_trunc) {
          lo = hi;  // cannot meet the tolerance: keep everything
          done = true;
        }
      }
      while (!done && lo < hi) {
        const int mid = (lo + hi) / 2;
        if (res_at(mid) <= tol_trunc) hi = mid; else lo = mid + 1;
      }
    }
    int r = lo;
    trunc_hint[k] = r;
    if (o.max_rank > 0) r = std::min(r, o.max_rank);
    // a rank above the product of the remaining mode sizes only adds null directions
    const long long right_cap = (k == 0) ? (long long)n(1) * n(2) : (long long)n(2);
    r = (int)std::min<long long>(r, right_cap);
    // truncated solution xt = QU[:, :r] SVt[:r]
    gemm<double>(c, false, false, rows, b, r, 1.0, QU.d(), b, 0, SVt.d(), b, 0, 0.0, xt.d(), b, 0, 1);
    // z core k: residual of xt projected on z's interfaces, on the helper stream when one is
    // free (it reads xt, z's interfaces and the operator, none of which the enrichment below
    // changes); joined at the end of this step, before xt is freed and z's interfaces read it
    if (o.kickrank > 0) {
      Ctx *h = z_ctx();
      Work<double> &w = (h == c) ? w64 : wz;
      if (h != c) {
        wz.c = h;
        z_fork(h);
      }
      const int zl = z.r[k], zr = z.r[k + 1];
      DBuf zk(h, (size_t)zl * nk * zr * sizeof(double)), bz(h, (size_t)zl * nk * zr * sizeof(double));
      rhs_local(h, w, PsiLz[k].d(), zl, F.core[k].d(), f[k], nk, f[k + 1], PsiRz[k].d(), zr, zk.d());
      apply_local<double>(h, w, PhiLz[k].d(), zl, a, A[k], A[k].A, PhiRz[k].d(), zr, b, xt.d(), bz.d());
      k_sub<<<grid1d((long long)zl * nk * zr, 256), 256, 0, h->stream>>>(zk.d(), bz.d(), (long long)zl * nk * zr);
      TTI_LAUNCH();
      DBuf Zq(h, (size_t)zl * nk * zr * sizeof(double)), Zr(h, (size_t)zr * zr * sizeof(double));
      qr(h, zl * nk, zr, bz.d(), zr, Zq.d(), Zr.d());
      if (h != c) {
        Zq.rehome(c);
        z_done(h);
      }
      z.core[k] = std::move(Zq);
    }
    ZJoinGuard zguard{this};  // declared after xt: joins before xt is freed
    // enrichment from the residual projected on z's right interface
    int rho = (o.kickrank > 0) ? z.r[k + 1] : 0;
    rho = std::min(rho, std::max(0, rows - r));
    rho = (int)std::min<long long>(rho, std::max<long long>(0, right_cap - r));
    if (o.max_rank > 0) rho = std::min(rho, std::max(0, o.max_rank - r));
    const int rn = r + rho;
    // new core Qe = [QU[:, :r] | Qz]: the enrichment columns E (residual projected on z's
    // right interface) are orthogonalised against the orthonormal QU[:, :r] by two classical
    // Gram-Schmidt passes, and only these rho columns go through a QR.  In the factor
    // Re of [QU[:, :r] | E] = Qe Re the first r columns are [I; 0], so the next core takes
    // C = Re[:, :r] SVt[:r] = [SVt[:r]; 0].
    DBuf Qe(c, (size_t)rows * rn * sizeof(double));
    copy2d(c, Qe.d(), rn, QU.d(), b, rows, r);
    if (rho > 0) {
      const int zr = z.r[k + 1];
      DBuf ez(c, (size_t)rows * zr * sizeof(double)), bz(c, (size_t)rows * zr * sizeof(double));
      rhs_local(c, w64, PsiL[k].d(), a, F.core[k].d(), f[k], nk, f[k + 1], PsiRz[k].d(), zr, ez.d());
      apply_local<double>(c, w64, PhiL[k].d(), a, a, A[k], A[k].A, PhiRz[k].d(), zr, b, xt.d(), bz.d());
      k_sub<<<grid1d((long long)rows * zr, 256), 256, 0, c->stream>>>(ez.d(), bz.d(), (long long)rows * zr);
      TTI_LAUNCH();
      DBuf E(c, (size_t)rows * rho * sizeof(double)), W(c, (size_t)r * rho * sizeof(double));
      copy2d(c, E.d(), rho, bz.d(), zr, rows, rho);
      for (int pass = 0; pass < 2; ++pass) {
        gemm<double>(c, true, false, r, rho, rows, 1.0, QU.d(), b, 0, E.d(), rho, 0, 0.0, W.d(), rho, 0, 1);
        gemm<double>(c, false, false, rows, rho, r, -1.0, QU.d(), b, 0, W.d(), rho, 0, 1.0, E.d(), rho, 0, 1);
      }
      DBuf Qz(c, (size_t)rows * rho * sizeof(double)), Rz(c, (size_t)rho * rho * sizeof(double));
      qr(c, rows, rho, E.d(), rho, Qz.d(), Rz.d());
      copy2d(c, Qe.d() + r, rn, Qz.d(), rho, rows, rho);
    }
    DBuf C(c, (size_t)rn * b * sizeof(double));
    if (rho > 0) c->zero(C.get(), (size_t)rn * b * sizeof(double));
    copy2d(c, C.d(), b, SVt.d(), b, r, b);
    const long long cols = (long long)n(k + 1) * u.r[k + 2];
    DBuf next(c, (size_t)rn * cols * sizeof(double));
    gemm<double>(c, false, false, rn, (int)cols, b, 1.0, C.d(), b, 0, u.core[k + 1].d(), cols, 0, 0.0, next.d(), cols,
                 0, 1);
    u.core[k] = std::move(Qe);
    u.core[k + 1] = std::move(next);
    u.r[k + 1] = rn;
    z_join();
  }

  void last_core_z(const double *x) {
    if (o.kickrank <= 0) return;
    z_join();  // z's left interfaces of core 2
    const int k = 2, zl = z.r[2], nk = n(2);
    DBuf zk(c, (size_t)zl * nk * sizeof(double)), bz(c, (size_t)zl * nk * sizeof(double));
    rhs_local(c, w64, PsiLz[k].d(), zl, F.core[k].d(), f[k], nk, 1, PsiRz[k].d(), 1, zk.d());
    apply_local<double>(c, w64, PhiLz[k].d(), zl, rl(k), A[k], A[k].A, PhiRz[k].d(), 1, 1, x, bz.d());
    k_sub<<<grid1d((long long)zl * nk, 256), 256, 0, c->stream>>>(zk.d(), bz.d(), (long long)zl * nk);
    TTI_LAUNCH();
    z.core[2] = std::move(bz);
  }

  double exact_residual() { return residual_norm(c, F, Fnorm, S->K, S->n, S->b, S->p, u); }

  int run(tt_iga_solution *out) {
    init();
    const double tol_abs = o.tol * Fnorm;
    const double tol_solve = 0.1 * tol_abs / sqrt(3.0);
    const double tol_trunc = 0.3 * tol_abs / sqrt(3.0);
    int status = TT_IGA_ERR_NOT_CONVERGED;
    // The exact residual of a finished sweep is evaluated lazily.  After the backward
    // pass the interfaces of core 0 are orthonormal, so the local residual of core 0 in
    // the next sweep is the norm of a projection of F - K u: when it exceeds tol ||F||
    // the sweep cannot have converged and the exact residual is skipped; otherwise it
    // is evaluated on the unchanged u before core 0 is touched.  The last allowed
    // sweep is always checked at once.
    bool check_pending = false;
    double prev_maxloc = 0.0;
    auto converged = [&](double res, double maxloc) {
      return (res >= 0.0 && res <= o.tol) || (res < 0.0 && maxloc <= o.tol);
    };
    for (int sweep = 0; sweep < o.max_sweeps; ++sweep) {
      double maxloc = 0.0;
      bool stop_now = false;
      // stage timer for verbose >= 2 (synchronises, diagnosis only)
      auto now_ms = [&]() {
        if (o.verbose >= 2) c->sync();
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
      };
      double t_solve = 0, t_trunc = 0, t_iface = 0;
      for (int k = 0; k < 3; ++k) {
        const long long N = (long long)rl(k) * n(k) * rr(k);
        DBuf rhs(c, N * sizeof(double)), x(c, N * sizeof(double));
        const double t0 = now_ms();
        rhs_local(c, w64, PsiL[k].d(), rl(k), F.core[k].d(), f[k], n(k), f[k + 1], PsiR[k].d(), rr(k), rhs.d());
        TTI_CUDA(cudaMemcpyAsync(x.d(), u.core[k].d(), N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        double r0;
        if (k == 0 && check_pending) {
          check_pending = false;
          bool checked = false;
          r0 = local_solve(k, rhs.d(), x.d(), tol_solve, tol_abs, &checked);
          if (checked) {
            const double res = exact_residual();
            st.rel_residual = res;
            if (o.verbose)
              fprintf(stderr, "[tt_iga amen] after sweep %d: local %.3e of ||F||, exact residual %.3e\n", sweep,
                      r0 / Fnorm, res);
            if (converged(res, prev_maxloc)) {
              status = TT_IGA_OK;
              stop_now = true;
              break;
            }
            r0 = local_solve(k, rhs.d(), x.d(), tol_solve);
          } else if (o.verbose) {
            fprintf(stderr, "[tt_iga amen] after sweep %d: local %.3e of ||F|| > tol, exact residual skipped\n",
                    sweep, r0 / Fnorm);
          }
        } else {
          r0 = local_solve(k, rhs.d(), x.d(), tol_solve);
        }
        maxloc = std::max(maxloc, r0 / Fnorm);
        if (o.verbose)
          fprintf(stderr, "[tt_iga amen] sweep %d core %d: initial local residual %.3e of ||F||, ranks %d %d, "
                          "local matvecs so far %lld\n", sweep + 1, k, r0 / Fnorm, rl(k), rr(k), st.local_matvecs);
        const double t1 = now_ms();
        t_solve += t1 - t0;
        if (k < 2) {
          truncate_enrich(k, rhs.d(), x.d(), tol_trunc);
          const double t2 = now_ms();
          t_trunc += t2 - t1;
          left_interfaces(k);
          t_iface += now_ms() - t2;
        } else {
          u.core[2] = std::move(x);
          last_core_z(u.core[2].d());
        }
      }
      if (stop_now) break;
      // backward orthogonalisation of u and z, refresh right interfaces
      const double tb0 = now_ms();
      for (int k = 2; k >= 1; --k) {
        if (o.kickrank > 0) z_orth(k);  // on the helper stream, overlapping u's step
        orth_right_step(c, u, k);
        right_interfaces(k);
      }
      const double tb1 = now_ms();
      st.sweeps = sweep + 1;
      last_local = maxloc;
      st.local_residual = maxloc;
      prev_maxloc = maxloc;
      const bool last = sweep + 1 == o.max_sweeps;
      const double res = last ? exact_residual() : -2.0;
      if (o.verbose >= 2)
        fprintf(stderr, "[tt_iga amen] sweep %d stages: local solves %.2f ms, truncation+enrichment %.2f ms, "
                        "left interfaces %.2f ms, backward pass %.2f ms, exact residual %.2f ms\n",
                sweep + 1, t_solve, t_trunc, t_iface, tb1 - tb0, now_ms() - tb1);
      if (o.verbose)
        fprintf(stderr, "[tt_iga amen] sweep %d ranks %d %d local %.3e matvecs %lld\n", sweep + 1, u.r[1], u.r[2],
                maxloc, st.local_matvecs);
      if (last) {
        st.rel_residual = res;
        if (converged(res, maxloc)) status = TT_IGA_OK;
      } else {
        check_pending = true;
      }
    }
    z_join();  // the solve ends when its helper work does
    st.ranks[0] = u.r[1];
    st.ranks[1] = u.r[2];
    st.converged = status == TT_IGA_OK;
    out->ctx = c;
    for (int k = 0; k < 3; ++k) out->n[k] = n(k);
    out->p = S->p;
    out->u = std::move(u);
    return status;
  }
};


int amen_solve(Ctx *c, const tt_iga_system *s, const tt_iga_solve_opts &o, tt_iga_solution *out, tt_iga_stats *st,
               const tt_iga_solution *start) {
  cudaEvent_t e0, e1;
  TTI_CUDA(cudaEventCreate(&e0));
  TTI_CUDA(cudaEventCreate(&e1));
  TTI_CUDA(cudaEventRecord(e0, c->stream));
  Amen a(c, s, o, start ? &start->u : nullptr);
  int status = a.run(out);
  TTI_CUDA(cudaEventRecord(e1, c->stream));
  TTI_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  a.st.ms_total = ms;
  if (st) *st = a.st;
  return status;
}

double exact_residual(Ctx *c, const tt_iga_system *s, const tt_iga_solution *sol, int k) {
  return residual_norm(c, s->F[k], s->F_norm[k], s->K, s->n, s->b, s->p, sol->u);
}

}  // namespace ttiga
