// AMEn local-system contractions: three-stage local matvec (dense GEMM with
// the right interface, band contraction with the operator core, dense GEMM
// with the left interface), interface updates, load projections, the band
// block-Jacobi preconditioner and the TT matvec core.
#include "amen_ops.cuh"
#include "linalg.cuh"

namespace ttiga {

// T2[g][a][i][c] = sum_{o,d} A[g][i][o][d] T1[a][i+o-p][c][d]
template <typename T>
__global__ void k_band_right(const T *__restrict__ A, int Rl, int n, int b, int p, int Rr, const T *__restrict__ T1,
                             int na, int nc, T *__restrict__ T2) {
  const long long tot = (long long)Rl * na * n * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int cc = (int)(e % nc);
    long long t = e / nc;
    const int i = (int)(t % n);
    t /= n;
    const int a = (int)(t % na);
    const int g = (int)(t / na);
    T acc = T(0);
    const T *Ar = A + ((long long)g * n + i) * b * Rr;
    for (int o = 0; o < b; ++o) {
      const int j = i + o - p;
      if (j < 0 || j >= n) continue;
      const T *Ao = Ar + (long long)o * Rr;
      const T *Tj = T1 + (((long long)a * n + j) * nc + cc) * Rr;
      for (int d = 0; d < Rr; ++d) acc += Ao[d] * Tj[d];
    }
    T2[e] = acc;
  }
}

// T2[a][i][d][c] = sum_{g,o} A[g][i][o][d] T1[a][g][i+o-p][c]
__global__ void k_band_left(const double *__restrict__ A, int Rl, int n, int b, int p, int Rr,
                            const double *__restrict__ T1, int na, int nc, double *__restrict__ T2) {
  const long long tot = (long long)na * n * Rr * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int cc = (int)(e % nc);
    long long t = e / nc;
    const int d = (int)(t % Rr);
    t /= Rr;
    const int i = (int)(t % n);
    const int a = (int)(t / n);
    double acc = 0.0;
    for (int g = 0; g < Rl; ++g) {
      const double *Ar = A + ((long long)g * n + i) * b * Rr + d;
      const double *Tg = T1 + ((long long)a * Rl + g) * n * nc + cc;
      for (int o = 0; o < b; ++o) {
        const int j = i + o - p;
        if (j < 0 || j >= n) continue;
        acc += Ar[(long long)o * Rr] * Tg[(long long)j * nc];
      }
    }
    T2[e] = acc;
  }
}

template <typename T>
void apply_local(Ctx *c, Work<T> &w, const T *PhiL, int ol, int il, const BandCore &A, const T *Ak, const T *PhiR,
                 int orr, int ir, const T *x, T *y) {
  const int n = A.n, Rl = A.Rl, Rr = A.Rr;
  T *T1 = w.get1((size_t)il * n * orr * Rr);
  gemm<T>(c, false, true, il * n, orr * Rr, ir, T(1), x, ir, 0, PhiR, ir, 0, T(0), T1, (long long)orr * Rr, 0, 1);
  T *T2 = w.get2((size_t)Rl * il * n * orr);
  const long long tot = (long long)Rl * il * n * orr;
  {
    // algorithmic FLOPs of the band stage: 2 per (output, band slot inside the mesh, operator rank)
    ProfScope ps(c, PROF_LOCAL_BAND, 2.0 * tot * A.b * Rr);
    k_band_right<T><<<grid1d(tot, 256, 152 * 32), 256, 0, c->stream>>>(Ak, Rl, n, A.b, A.p, Rr, T1, il, orr, T2);
    TTI_LAUNCH();
  }
  gemm<T>(c, false, false, ol, n * orr, Rl * il, T(1), PhiL, (long long)Rl * il, 0, T2, (long long)n * orr, 0, T(0), y,
          (long long)n * orr, 0, 1);
}
template void apply_local<double>(Ctx *, Work<double> &, const double *, int, int, const BandCore &, const double *,
                                  const double *, int, int, const double *, double *);
template void apply_local<float>(Ctx *, Work<float> &, const float *, int, int, const BandCore &, const float *,
                                 const float *, int, int, const float *, float *);

void left_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const double *PhiL, const BandCore &A,
                 const double *U, int ul, int ur, double *out) {
  const int n = A.n, Rl = A.Rl, Rr = A.Rr;
  double *T1 = w.get1((size_t)tl * Rl * n * ur);
  gemm<double>(c, false, false, tl * Rl, n * ur, ul, 1.0, PhiL, ul, 0, U, (long long)n * ur, 0, 0.0, T1,
               (long long)n * ur, 0, 1);
  double *T2 = w.get2((size_t)tl * n * Rr * ur);
  const long long tot = (long long)tl * n * Rr * ur;
  k_band_left<<<grid1d(tot, 256, 152 * 32), 256, 0, c->stream>>>(A.A, Rl, n, A.b, A.p, Rr, T1, tl, ur, T2);
  TTI_LAUNCH();
  gemm<double>(c, true, false, tr, Rr * ur, tl * n, 1.0, Z, tr, 0, T2, (long long)Rr * ur, 0, 0.0, out,
               (long long)Rr * ur, 0, 1);
}

void right_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const BandCore &A, const double *PhiR,
                  const double *U, int ul, int ur, double *out) {
  const int n = A.n, Rl = A.Rl, Rr = A.Rr;
  double *T1 = w.get1((size_t)ul * n * tr * Rr);
  gemm<double>(c, false, true, ul * n, tr * Rr, ur, 1.0, U, ur, 0, PhiR, ur, 0, 0.0, T1, (long long)tr * Rr, 0, 1);
  double *T2 = w.get2((size_t)Rl * ul * n * tr);
  const long long tot = (long long)Rl * ul * n * tr;
  k_band_right<double><<<grid1d(tot, 256, 152 * 32), 256, 0, c->stream>>>(A.A, Rl, n, A.b, A.p, Rr, T1, ul, tr, T2);
  TTI_LAUNCH();
  gemm<double>(c, false, true, tl, Rl * ul, n * tr, 1.0, Z, (long long)n * tr, 0, T2, (long long)n * tr, 0, 0.0, out,
               (long long)Rl * ul, 0, 1);
}

void rhs_local(Ctx *c, Work<double> &w, const double *PsiL, int ol, const double *F, int fl, int n, int fr,
               const double *PsiR, int orr, double *y) {
  double *T = w.get1((size_t)ol * n * fr);
  gemm<double>(c, false, false, ol, n * fr, fl, 1.0, PsiL, fl, 0, F, (long long)n * fr, 0, 0.0, T, (long long)n * fr, 0,
               1);
  gemm<double>(c, false, true, ol * n, orr, fr, 1.0, T, fr, 0, PsiR, fr, 0, 0.0, y, orr, 0, 1);
}

void rhs_left_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const double *PsiL, const double *F,
                     int fl, int n, int fr, double *out) {
  double *T = w.get1((size_t)tl * n * fr);
  gemm<double>(c, false, false, tl, n * fr, fl, 1.0, PsiL, fl, 0, F, (long long)n * fr, 0, 0.0, T, (long long)n * fr, 0,
               1);
  gemm<double>(c, true, false, tr, fr, tl * n, 1.0, Z, tr, 0, T, fr, 0, 0.0, out, fr, 0, 1);
}

void rhs_right_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const double *F, int fl, int n, int fr,
                      const double *PsiR, double *out) {
  double *T = w.get1((size_t)fl * n * tr);
  gemm<double>(c, false, true, fl * n, tr, fr, 1.0, F, fr, 0, PsiR, fr, 0, 0.0, T, tr, 0, 1);
  gemm<double>(c, false, true, tl, fl, n * tr, 1.0, Z, (long long)n * tr, 0, T, (long long)n * tr, 0, 0.0, out, fl, 0,
               1);
}

// ------------------------------------------------------- preconditioner

// D[a][g] = Phi[a][g][a]
__global__ void k_diag_interface(const double *Phi, int r, int R, double *D) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * R; e += gridDim.x * blockDim.x) {
    const int a = e / R, g = e % R;
    D[e] = Phi[((long long)a * R + g) * r + a];
  }
}

// Band Cholesky per (alpha, beta) pair of the symmetrised band matrix
// P[a][i][o][b] (half-bandwidth PB).  Output L[i][k][pair] = L(i, i-PB+k) for
// k < PB and the reciprocal of the diagonal in slot PB.  With j = i-PB+k,
//   L(i,j) = (A(i,j) - sum_{m=i-PB}^{j-1} L(i,m) L(j,m)) / L(j,j),
//   L(i,i) = sqrt(A(i,i) - sum_{m=i-PB}^{i-1} L(i,m)^2).
// The arithmetic runs in the factor's own type T: the row-to-row recurrence is
// a chain of dependent operations, and in FP32 each link costs a few cycles
// instead of the tens to hundreds of an FP64 FMA, square root or divide.  A
// pivot that cancellation drives to zero or below is replaced by the row's
// diagonal entry (the factor stays SPD; PCG convergence is checked in FP64);
// a diagonal entry that is itself not positive flags a breakdown.
// The previous PB rows of L stay in registers (win[q] = row i-PB+q).
template <typename T> __device__ __forceinline__ T recip_sqrt(T v);
template <> __device__ __forceinline__ float recip_sqrt<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double recip_sqrt<double>(double v) { return 1.0 / sqrt(v); }

template <typename T, int PB>
__global__ void k_band_cholesky(const double *__restrict__ Pm, int rl, int n, int rr, T *__restrict__ L, int *status) {
  // rows are loaded in groups of RG, one group ahead, so the memory latency is
  // exposed once per group instead of once per row
  constexpr int RG = 4;
  const int npair = rl * rr, b = 2 * PB + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += gridDim.x * blockDim.x) {
    const int a = t / rr, bb = t % rr;
    const double *Pp = Pm + (long long)a * n * b * rr + bb;
    T win[PB][PB + 1];
#pragma unroll
    for (int q = 0; q < PB; ++q)
#pragma unroll
      for (int k = 0; k <= PB; ++k) win[q][k] = T(0);
    bool bad = false;
    // symmetrised band entries of a row: A(i, i-PB+k) for k <= PB
    auto load_row = [&](int i, T *out) {
      if (i >= n) return;
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        const int j = i - PB + k;
        out[k] = (j >= 0) ? (T)(0.5 * (Pp[((long long)i * b + k) * rr] + Pp[((long long)j * b + (2 * PB - k)) * rr]))
                          : T(0);
      }
      out[PB] = (T)Pp[((long long)i * b + PB) * rr];
    };
    T nxt[RG][PB + 1];
#pragma unroll
    for (int g = 0; g < RG; ++g) load_row(g, nxt[g]);
    for (int i0 = 0; i0 < n; i0 += RG) {
      T cur[RG][PB + 1];
#pragma unroll
      for (int g = 0; g < RG; ++g)
#pragma unroll
        for (int k = 0; k <= PB; ++k) cur[g][k] = nxt[g][k];
#pragma unroll
      for (int g = 0; g < RG; ++g) load_row(i0 + RG + g, nxt[g]);
#pragma unroll
      for (int g = 0; g < RG; ++g) {
        const int i = i0 + g;
        if (i >= n) break;
        T row[PB + 1];
#pragma unroll
        for (int k = 0; k < PB; ++k) {
          const int j = i - PB + k;
          if (j < 0) {
            row[k] = T(0);
            continue;
          }
          T sv = cur[g][k];
#pragma unroll
          for (int mm = 0; mm < k; ++mm) sv -= row[mm] * win[k][mm + PB - k];
          row[k] = sv * win[k][PB];
        }
        T sd = cur[g][PB];
#pragma unroll
        for (int mm = 0; mm < PB; ++mm) sd -= row[mm] * row[mm];
        if (!(sd > T(1e-6) * cur[g][PB])) {
          if (!(cur[g][PB] > T(0))) bad = true;
          sd = (cur[g][PB] > T(0)) ? cur[g][PB] : T(1);
        }
        row[PB] = recip_sqrt<T>(sd);
#pragma unroll
        for (int k = 0; k <= PB; ++k) L[((long long)i * (PB + 1) + k) * npair + t] = row[k];
#pragma unroll
        for (int q = 0; q + 1 < PB; ++q)
#pragma unroll
          for (int k = 0; k <= PB; ++k) win[q][k] = win[q + 1][k];
#pragma unroll
        for (int k = 0; k <= PB; ++k) win[PB - 1][k] = row[k];
      }
    }
    if (bad) atomicMax(status, (int)DS_BREAKDOWN);
  }
}

template <typename T>
void precond_build(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, T *L) {
  const int n = A.n, b = A.b, Rl = A.Rl, Rr = A.Rr;
  DBuf dL(c, (size_t)rl * Rl * sizeof(double)), dR(c, (size_t)rr * Rr * sizeof(double));
  k_diag_interface<<<grid1d((long long)rl * Rl, 128), 128, 0, c->stream>>>(PhiL, rl, Rl, dL.d());
  TTI_LAUNCH();
  k_diag_interface<<<grid1d((long long)rr * Rr, 128), 128, 0, c->stream>>>(PhiR, rr, Rr, dR.d());
  TTI_LAUNCH();
  // W[(g,i,o)][b] = sum_d A[g][i][o][d] dR[b][d]
  DBuf W(c, (size_t)Rl * n * b * rr * sizeof(double));
  gemm<double>(c, false, true, Rl * n * b, rr, Rr, 1.0, A.A, Rr, 0, dR.d(), Rr, 0, 0.0, W.d(), rr, 0, 1);
  // P[a][(i,o,b)] = sum_g dL[a][g] W[g][(i,o,b)]
  DBuf P(c, (size_t)rl * n * b * rr * sizeof(double));
  gemm<double>(c, false, false, rl, n * b * rr, Rl, 1.0, dL.d(), Rl, 0, W.d(), (long long)n * b * rr, 0, 0.0, P.d(),
               (long long)n * b * rr, 0, 1);
  const unsigned grid = grid1d((long long)rl * rr, 32), blk = 32;
  switch (A.p) {
    case 1: k_band_cholesky<T, 1><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    case 2: k_band_cholesky<T, 2><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    case 3: k_band_cholesky<T, 3><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    case 4: k_band_cholesky<T, 4><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    case 5: k_band_cholesky<T, 5><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    case 6: k_band_cholesky<T, 6><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    case 7: k_band_cholesky<T, 7><<<grid, blk, 0, c->stream>>>(P.d(), rl, n, rr, L, c->dstatus); break;
    default: fail(TT_IGA_ERR_ARG, "preconditioner: degree %d outside 1..7", A.p);
  }
  TTI_LAUNCH();
}
template void precond_build<double>(Ctx *, const double *, int, const BandCore &, const double *, int, double *);
template void precond_build<float>(Ctx *, const double *, int, const BandCore &, const double *, int, float *);

// Solve L L^T z = r per (alpha, beta) pair with the factors of k_band_cholesky
// (reciprocal diagonal in slot PB).  Forward: y_i = (r_i - sum_k L(i,i-PB+k)
// y_{i-PB+k}) / L(i,i); backward: z_i = (y_i - sum_{d=1..PB} L(i+d,i) z_{i+d}) /
// L(i,i).  The last PB solution values are kept in registers; the factor
// loads do not depend on them and pipeline freely.
template <typename T, int PB>
__global__ void k_band_solve(const T *__restrict__ L, int rl, int n, int rr, const T *__restrict__ r,
                             T *__restrict__ z) {
  const int npair = rl * rr;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += gridDim.x * blockDim.x) {
    const int a = t / rr, bb = t % rr;
    const long long base = (long long)a * n * rr + bb;
    T w[PB];
#pragma unroll
    for (int k = 0; k < PB; ++k) w[k] = T(0);
    for (int i = 0; i < n; ++i) {
      const T *Li = L + (long long)i * (PB + 1) * npair + t;
      T sv = r[base + (long long)i * rr];
#pragma unroll
      for (int k = 0; k < PB; ++k) sv -= Li[(long long)k * npair] * w[k];
      const T y = sv * Li[(long long)PB * npair];
      z[base + (long long)i * rr] = y;
#pragma unroll
      for (int k = 0; k + 1 < PB; ++k) w[k] = w[k + 1];
      w[PB - 1] = y;
    }
#pragma unroll
    for (int k = 0; k < PB; ++k) w[k] = T(0);  // w[d-1] = z_{i+d}
    for (int i = n - 1; i >= 0; --i) {
      T sv = z[base + (long long)i * rr];
#pragma unroll
      for (int d = 1; d <= PB; ++d)
        if (i + d < n) sv -= L[((long long)(i + d) * (PB + 1) + (PB - d)) * npair + t] * w[d - 1];
      const T zi = sv * L[((long long)i * (PB + 1) + PB) * npair + t];
      z[base + (long long)i * rr] = zi;
#pragma unroll
      for (int d = PB - 1; d > 0; --d) w[d] = w[d - 1];
      w[0] = zi;
    }
  }
}

template <typename T> void precond_apply(Ctx *c, const T *L, int rl, int n, int p, int rr, const T *r, T *z) {
  const unsigned grid = grid1d((long long)rl * rr, 32), blk = 32;
  switch (p) {
    case 1: k_band_solve<T, 1><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    case 2: k_band_solve<T, 2><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    case 3: k_band_solve<T, 3><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    case 4: k_band_solve<T, 4><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    case 5: k_band_solve<T, 5><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    case 6: k_band_solve<T, 6><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    case 7: k_band_solve<T, 7><<<grid, blk, 0, c->stream>>>(L, rl, n, rr, r, z); break;
    default: fail(TT_IGA_ERR_ARG, "preconditioner: degree %d outside 1..7", p);
  }
  TTI_LAUNCH();
}
template void precond_apply<double>(Ctx *, const double *, int, int, int, int, const double *, double *);
template void precond_apply<float>(Ctx *, const float *, int, int, int, int, const float *, float *);

// out[(g,a)][i][(d,c)] = sum_o A[g][i][o][d] U[a][i+o-p][c]
__global__ void k_tt_matvec_core(const double *__restrict__ A, int Rl, int n, int b, int p, int Rr,
                                 const double *__restrict__ U, int ul, int ur, double *__restrict__ out) {
  const long long tot = (long long)Rl * ul * n * Rr * ur;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int cc = (int)(e % ur);
    long long t = e / ur;
    const int d = (int)(t % Rr);
    t /= Rr;
    const int i = (int)(t % n);
    t /= n;
    const int a = (int)(t % ul);
    const int g = (int)(t / ul);
    double acc = 0.0;
    for (int o = 0; o < b; ++o) {
      const int j = i + o - p;
      if (j < 0 || j >= n) continue;
      acc += A[(((long long)g * n + i) * b + o) * Rr + d] * U[((long long)a * n + j) * ur + cc];
    }
    out[e] = acc;
  }
}

void tt_matvec_core(Ctx *c, const BandCore &A, const double *U, int ul, int ur, double *out) {
  const long long tot = (long long)A.Rl * ul * A.n * A.Rr * ur;
  k_tt_matvec_core<<<grid1d(tot, 256), 256, 0, c->stream>>>(A.A, A.Rl, A.n, A.b, A.p, A.Rr, U, ul, ur, out);
  TTI_LAUNCH();
}

}  // namespace ttiga
