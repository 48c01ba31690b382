// Exact block-band preconditioner of small-interface AMEn local systems:
// assembly of the symmetric block band (FP64 contractions, FP32 result), then
// the odd-even (cyclic) reduction of its block-tridiagonal super-row form, one
// launch per level, so the factorisation is log2 of the super-row count deep.
#include "bbprec.cuh"

namespace ttiga {

namespace {

// Blow[i][l][e][f] = Bsym(i, i-p+l)[e][f] for l = 0..p: the lower block band of
// the symmetric part of the local matrix, with
//   B(i, j)[(a,c)][(a',c')] = sum_{g,d} PhiL[a][g][a'] A[g][i][j-i+p][d] PhiR[c][d][c'].
template <int M>
__global__ void k_bb_build(const double *__restrict__ PhiL, int rl, int Rl, const double *__restrict__ A, int n, int p,
                           int Rr, const double *__restrict__ PhiR, int rr, float *__restrict__ Blow) {
  const int b = 2 * p + 1, m = rl * rr;
  const long long tot = (long long)n * (p + 1) * M * M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(t % M), e = (int)((t / M) % M);
    const long long il = t / (M * M);
    const int l = (int)(il % (p + 1)), i = (int)(il / (p + 1));
    const int j = i - p + l;
    float v;
    if (e >= m || f >= m) {
      v = (l == p && e == f) ? 1.f : 0.f;
    } else if (j < 0) {
      v = 0.f;
    } else {
      const int a = e / rr, c = e % rr, a2 = f / rr, c2 = f % rr;
      double s1 = 0.0, s2 = 0.0;
      for (int g = 0; g < Rl; ++g) {
        const double pl1 = PhiL[((long long)a * Rl + g) * rl + a2], pl2 = PhiL[((long long)a2 * Rl + g) * rl + a];
        const double *A1 = A + (((long long)g * n + i) * b + l) * Rr;
        const double *A2 = A + (((long long)g * n + j) * b + (2 * p - l)) * Rr;
        for (int d = 0; d < Rr; ++d) {
          s1 += pl1 * A1[d] * PhiR[((long long)c * Rr + d) * rr + c2];
          s2 += pl2 * A2[d] * PhiR[((long long)c2 * Rr + d) * rr + c];
        }
      }
      v = (float)(0.5 * (s1 + s2));
    }
    Blow[t] = v;
  }
}

// D[J] (q x q) and C[J] = B(super-row J, super-row J - 1) from the lower block band:
// entry (a M + e, b M + f) of a super-row pair is B(i, j)[e][f] with i = p J + a and
// j = p J + b (D) or p (J - 1) + b (C); B(i, j) = B(j, i)^T above the diagonal, and
// block rows past n carry the identity with no coupling.
__global__ void k_bcr_init(const float *__restrict__ Blow, int n, int p, int M, int S, int q, float *__restrict__ D,
                           float *__restrict__ C) {
  const long long per = (long long)q * q, tot = (long long)S * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * tot;
       t += (long long)gridDim.x * blockDim.x) {
    const bool coup = t >= tot;
    const long long u = coup ? t - tot : t;
    const int J = (int)(u / per), rc = (int)(u % per), r = rc / q, cc = rc % q;
    const int a = r / M, e = r % M, bb = cc / M, f = cc % M;
    const long long i = (long long)p * J + a, j = coup ? (long long)p * (J - 1) + bb : (long long)p * J + bb;
    float v = 0.f;
    if (coup && J == 0) {
      v = 0.f;
    } else if (i >= n || j >= n) {
      v = (i == j && e == f) ? 1.f : 0.f;
    } else if (j <= i && i - j <= p) {
      v = Blow[(i * (p + 1) + (j - i + p)) * M * M + e * M + f];
    } else if (j > i && j - i <= p) {
      v = Blow[(j * (p + 1) + (i - j + p)) * M * M + f * M + e];
    }
    (coup ? C : D)[u] = v;
  }
}

// O = alpha op(A) op(B) for Q x Q shared-memory matrices (leading dimension Q + 1); O has
// leading dimension ldo and may be global.
template <int Q, bool TA, bool TB>
__device__ __forceinline__ void bcr_mm(const float *A, const float *B, float *O, int ldo, float alpha) {
  constexpr int LD = Q + 1;
  for (int e = threadIdx.x; e < Q * Q; e += blockDim.x) {
    const int r = e / Q, c = e % Q;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int k = 0; k < Q; k += 2) {
      s0 += (TA ? A[k * LD + r] : A[r * LD + k]) * (TB ? B[c * LD + k] : B[k * LD + c]);
      s1 += (TA ? A[(k + 1) * LD + r] : A[r * LD + k + 1]) * (TB ? B[c * LD + k + 1] : B[(k + 1) * LD + c]);
    }
    O[(long long)r * ldo + c] = alpha * (s0 + s1);
  }
}

// Elimination of the super-rows that are odd multiples of h (j = h + 2 h blockIdx.x), one
// CTA each, or of the top row 0 (root, h = the first power of two >= S).  Row j first takes
// the Schur terms of every lower level h2 < h, in level order: D_j -= SR_{j-h2} + SL_{j+h2},
// and its couplings of this level, CN_{j-h/2} with j - h and CN_{j+h/2} with j + h (the
// original C at level 0).  Then: Cholesky of D_j by one warp (a pivot that cancellation
// drives below 1e-6 of the diagonal entry is replaced by that entry: the factor stays SPD
// and PCG checks convergence), Linv_j = L_j^{-1} (a thread per column), Ul_j = Linv_j C_j,
// Ur_j = Linv_j C_{j+h}^T, and the Schur terms SL_j = Ul_j^T Ul_j, SR_j = Ur_j^T Ur_j,
// CN_j = -Ur_j^T Ul_j that the rows of later levels take.  Each row is eliminated once, so
// the terms of all levels stay in SL, SR, CN.  Q = p M is a template parameter so that the
// loops over a super-row unroll.
template <int Q>
__global__ void __launch_bounds__(256) k_bcr_elim(const float *__restrict__ D, const float *__restrict__ C, int S,
                                                  int h, int root, float *__restrict__ Linv, float *__restrict__ Ul,
                                                  float *__restrict__ Ur, float *SL, float *SR, float *CN) {
  constexpr int LD = Q + 1;
  constexpr long long per = (long long)Q * Q;
  extern __shared__ float bsm[];
  float *Lm = bsm;            // D_j, factored in place (lower triangle)
  float *Li = Lm + Q * LD;    // L_j^{-1}
  float *Cl = Li + Q * LD;    // C_j: rows of j, columns of j - h
  float *Cr = Cl + Q * LD;    // C_{j+h}^T: rows of j, columns of j + h
  float *Wl = Cr + Q * LD;    // Ul_j
  float *Wr = Wl + Q * LD;    // Ur_j
  float *diag0 = Wr + Q * LD;
  float *rdiag = diag0 + Q;   // 1 / L_rr
  const int j = root ? 0 : h + 2 * h * (int)blockIdx.x;
  const bool hasl = !root, hasr = !root && j + h < S;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < Q * Q; e += nt) {
    const int r = e / Q, c = e % Q;
    float d = D[j * per + e];
    for (int h2 = 1; h2 < h; h2 <<= 1) {
      if (j >= h2) d -= SR[(j - h2) * per + e];
      if (j + h2 < S) d -= SL[(j + h2) * per + e];
    }
    Lm[r * LD + c] = d;
    if (r == c) diag0[r] = d;
    Cl[r * LD + c] = hasl ? (h == 1 ? C[j * per + e] : CN[(j - h / 2) * per + e]) : 0.f;
    Cr[c * LD + r] = hasr ? (h == 1 ? C[(j + h) * per + e] : CN[(j + h / 2) * per + e]) : 0.f;
  }
  __syncthreads();
  if (Q <= 32 && tid < 32) {
    // right-looking Cholesky in registers: lane r holds row r, the pivot and the entries of
    // column c come from their owners by shuffles
    constexpr int NR = (Q + 31) / 32;
    const int lane = tid;
    float R[NR][Q];
#pragma unroll
    for (int u = 0; u < NR; ++u) {
      const int r = lane + 32 * u;
#pragma unroll
      for (int k = 0; k < Q; ++k) R[u][k] = (r < Q) ? Lm[r * LD + k] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      float piv = __shfl_sync(0xffffffffu, R[c / 32][c], c % 32);
      const float d0 = diag0[c];
      if (!(piv > 1e-6f * d0)) piv = (d0 > 0.f) ? d0 : 1.f;
      const float l = sqrtf(piv), inv = 1.f / l;
#pragma unroll
      for (int u = 0; u < NR; ++u) {
        const int r = lane + 32 * u;
        if (r == c) R[u][c] = l;
        else if (r > c) R[u][c] *= inv;
      }
      if (lane == 0) rdiag[c] = inv;
#pragma unroll
      for (int cc = c + 1; cc < Q; ++cc) {
        const float v = __shfl_sync(0xffffffffu, R[cc / 32][c], cc % 32);  // L[cc][c]
#pragma unroll
        for (int u = 0; u < NR; ++u)
          if (lane + 32 * u >= cc) R[u][cc] -= R[u][c] * v;
      }
    }
#pragma unroll
    for (int u = 0; u < NR; ++u) {
      const int r = lane + 32 * u;
      if (r < Q)
#pragma unroll
        for (int k = 0; k < Q; ++k) Lm[r * LD + k] = R[u][k];
    }
  } else if (Q > 32 && tid < 32) {
    // the same in shared memory (rows of up to 56 entries do not fit the registers): lane r
    // owns rows r and r + 32; column c is read into registers before the row updates
    const int lane = tid;
    for (int c = 0; c < Q; ++c) {
      float piv = Lm[c * LD + c];
      const float d0 = diag0[c];
      if (!(piv > 1e-6f * d0)) piv = (d0 > 0.f) ? d0 : 1.f;
      const float l = sqrtf(piv), inv = 1.f / l;
      __syncwarp();
      for (int r = lane; r < Q; r += 32) {
        if (r == c) {
          Lm[c * LD + c] = l;
          rdiag[c] = inv;
        } else if (r > c) {
          Lm[r * LD + c] *= inv;
        }
      }
      __syncwarp();
      for (int r = lane; r < Q; r += 32) {
        if (r <= c) continue;
        const float lrc = Lm[r * LD + c];
        float col[Q];
#pragma unroll
        for (int cc = 0; cc < Q; ++cc) col[cc] = Lm[cc * LD + c];
#pragma unroll
        for (int cc = 1; cc < Q; ++cc)
          if (cc > c && cc <= r) Lm[r * LD + cc] -= lrc * col[cc];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // L^{-1}: forward substitution against each unit vector, a thread per column
  if (tid < Q) {
    const int col = tid;
    float x[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int k = 0; k < r; ++k) {
        const float t = (k >= col) ? Lm[r * LD + k] * x[k] : 0.f;
        if (k & 1) s1 += t;
        else s0 += t;
      }
      x[r] = (r < col) ? 0.f : (((r == col) ? 1.f : 0.f) - (s0 + s1)) * rdiag[r];
    }
#pragma unroll
    for (int r = 0; r < Q; ++r) Li[r * LD + col] = x[r];
  }
  __syncthreads();
  for (int e = tid; e < Q * Q; e += nt) Linv[j * per + e] = Li[(e / Q) * LD + e % Q];
  if (root) return;
  bcr_mm<Q, false, false>(Li, Cl, Wl, LD, 1.f);
  bcr_mm<Q, false, false>(Li, Cr, Wr, LD, 1.f);
  __syncthreads();
  for (int e = tid; e < Q * Q; e += nt) {
    Ul[j * per + e] = Wl[(e / Q) * LD + e % Q];
    Ur[j * per + e] = Wr[(e / Q) * LD + e % Q];
  }
  bcr_mm<Q, true, false>(Wl, Wl, SL + j * per, Q, 1.f);
  bcr_mm<Q, true, false>(Wr, Wr, SR + j * per, Q, 1.f);
  bcr_mm<Q, true, false>(Wr, Wl, CN + j * per, Q, -1.f);
}

constexpr size_t kBcrSmemMax = 100 * 1024;

size_t bcr_smem(int q) { return ((size_t)6 * q * (q + 1) + 2 * q) * sizeof(float); }

// Super-row sizes q = p M of the instantiated eliminations (p <= 7, M = 4 or 8).
template <int Q> void bcr_launch(Ctx *c, int grid, size_t smem, const float *D, const float *C, int S, int h, int root,
                                 BBPrec &P, float *SL, float *SR, float *CN) {
  set_smem_limit_once((const void *)k_bcr_elim<Q>, (int)kBcrSmemMax);
  k_bcr_elim<Q><<<grid, 256, smem, c->stream>>>(D, C, S, h, root, P.Linv.as<float>(), P.Ul.as<float>(),
                                                P.Ur.as<float>(), SL, SR, CN);
  TTI_LAUNCH();
}

void bcr_elim(Ctx *c, int q, int grid, size_t smem, const float *D, const float *C, int S, int h, int root,
              BBPrec &P, float *SL, float *SR, float *CN) {
  switch (q) {
    case 4: bcr_launch<4>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 8: bcr_launch<8>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 12: bcr_launch<12>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 16: bcr_launch<16>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 20: bcr_launch<20>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 24: bcr_launch<24>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 28: bcr_launch<28>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 32: bcr_launch<32>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 40: bcr_launch<40>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 48: bcr_launch<48>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    case 56: bcr_launch<56>(c, grid, smem, D, C, S, h, root, P, SL, SR, CN); break;
    default: fail(TT_IGA_ERR_ARG, "block-band preconditioner: super-row size %d not instantiated", q);
  }
}

template <int M>
void build_m(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, BBPrec &P) {
  const int n = A.n, p = A.p;
  constexpr int BS = M * M;
  DBuf Blow(c, (size_t)n * (p + 1) * BS * sizeof(float));
  {
    const long long tot = (long long)n * (p + 1) * BS;
    k_bb_build<M><<<grid1d(tot, 256), 256, 0, c->stream>>>(PhiL, rl, A.Rl, A.A, n, p, A.Rr, PhiR, rr,
                                                           Blow.as<float>());
    TTI_LAUNCH();
  }
  const int q = P.q, S = P.S;
  const size_t mat = (size_t)S * q * q * sizeof(float);
  DBuf D(c, mat), C(c, mat), SL(c, mat), SR(c, mat), CN(c, mat);
  P.Linv = DBuf(c, mat);
  P.Ul = DBuf(c, mat);
  P.Ur = DBuf(c, mat);
  k_bcr_init<<<grid1d(2LL * S * q * q, 256), 256, 0, c->stream>>>(Blow.as<float>(), n, p, M, S, q, D.as<float>(),
                                                                  C.as<float>());
  TTI_LAUNCH();
  const size_t smem = bcr_smem(q);
  ProfScope ps(c, PROF_PRECOND, 0.0);
  P.levels = 0;
  int h = 1;
  for (; h < S; h <<= 1, ++P.levels)
    bcr_elim(c, q, (S - h + 2 * h - 1) / (2 * h), smem, D.as<float>(), C.as<float>(), S, h, 0, P, SL.as<float>(),
             SR.as<float>(), CN.as<float>());
  bcr_elim(c, q, 1, smem, D.as<float>(), C.as<float>(), S, h, 1, P, SL.as<float>(), SR.as<float>(), CN.as<float>());
}

}  // namespace

bool bb_eligible(int m, int n, int p) {
  return m >= 1 && m <= kBBMaxM && n >= 1 && n <= 1024 && p >= 1 && p <= 7 &&
         bcr_smem(p * bb_pad(m)) <= kBcrSmemMax;
}

void bb_prec_build(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, BBPrec &P) {
  const int m = rl * rr;
  TTI_CHECK_ARG(bb_eligible(m, A.n, A.p), "block-band preconditioner: m=%d n=%d p=%d out of range", m, A.n, A.p);
  P.n = A.n;
  P.p = A.p;
  P.m = m;
  P.M = bb_pad(m);
  P.q = A.p * P.M;
  P.S = (A.n + A.p - 1) / A.p;
  if (P.M == 4) build_m<4>(c, PhiL, rl, A, PhiR, rr, P);
  else build_m<8>(c, PhiL, rl, A, PhiR, rr, P);
}

}  // namespace ttiga
