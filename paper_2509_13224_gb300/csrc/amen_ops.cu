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

// Symmetrised band entries in the factor's type, S[i][k][pair] = (A(i, i-PB+k) +
// A(i-PB+k, i)) / 2 for k < PB (0 outside the matrix) and S[i][PB][pair] = A(i, i),
// from P[a][i][o][b] (pair = a rr + b): one thread per entry, so the FP64 reads and
// conversions leave the sequential factorisation below.
template <typename T, int PB>
__global__ void k_band_sym(const double *__restrict__ Pm, int rl, int n, int rr, T *__restrict__ S) {
  const int npair = rl * rr, b = 2 * PB + 1;
  const long long tot = (long long)n * (PB + 1) * npair;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e % npair);
    const long long q = e / npair;
    const int k = (int)(q % (PB + 1)), i = (int)(q / (PB + 1));
    const int a = t / rr, bb = t % rr;
    const double *Pp = Pm + (long long)a * n * b * rr + bb;
    T v;
    if (k == PB) {
      v = (T)Pp[((long long)i * b + PB) * rr];
    } else {
      const int j = i - PB + k;
      v = (j >= 0) ? (T)(0.5 * (Pp[((long long)i * b + k) * rr] + Pp[((long long)j * b + (2 * PB - k)) * rr])) : T(0);
    }
    S[e] = v;
  }
}

template <typename T, int PB>
__global__ void k_band_cholesky(const T *__restrict__ S, int rl, int n, int rr, T *__restrict__ L, int *status) {
  // rows are loaded in groups of RG, one group ahead (coalesced over the pairs of a
  // warp), so the memory latency is exposed once per group instead of once per row
  constexpr int RG = 8;
  const int npair = rl * rr;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += gridDim.x * blockDim.x) {
    T win[PB][PB + 1];
#pragma unroll
    for (int q = 0; q < PB; ++q)
#pragma unroll
      for (int k = 0; k <= PB; ++k) win[q][k] = T(0);
    bool bad = false;
    auto load_row = [&](int i, T *out) {
      if (i >= n) return;
#pragma unroll
      for (int k = 0; k <= PB; ++k) out[k] = S[((long long)i * (PB + 1) + k) * npair + t];
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

template <typename T, int PB> static void band_factor(Ctx *c, const double *P, int rl, int n, int rr, T *L) {
  DBuf Sb(c, (size_t)n * (PB + 1) * rl * rr * sizeof(T));
  const long long tot = (long long)n * (PB + 1) * rl * rr;
  k_band_sym<T, PB><<<grid1d(tot, 256), 256, 0, c->stream>>>(P, rl, n, rr, Sb.as<T>());
  TTI_LAUNCH();
  // one pair per thread; small CTAs spread the independent chains over many SMs
  const unsigned grid = grid1d((long long)rl * rr, 32), blk = 32;
  k_band_cholesky<T, PB><<<grid, blk, 0, c->stream>>>(Sb.as<T>(), rl, n, rr, L, c->dstatus);
  TTI_LAUNCH();
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
  switch (A.p) {
    case 1: band_factor<T, 1>(c, P.d(), rl, n, rr, L); break;
    case 2: band_factor<T, 2>(c, P.d(), rl, n, rr, L); break;
    case 3: band_factor<T, 3>(c, P.d(), rl, n, rr, L); break;
    case 4: band_factor<T, 4>(c, P.d(), rl, n, rr, L); break;
    case 5: band_factor<T, 5>(c, P.d(), rl, n, rr, L); break;
    case 6: band_factor<T, 6>(c, P.d(), rl, n, rr, L); break;
    case 7: band_factor<T, 7>(c, P.d(), rl, n, rr, L); break;
    default: fail(TT_IGA_ERR_ARG, "preconditioner: degree %d outside 1..7", A.p);
  }
}
template void precond_build<float>(Ctx *, const double *, int, const BandCore &, const double *, int, float *);


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
