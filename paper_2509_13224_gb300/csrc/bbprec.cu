// Exact block-band preconditioner of small-interface AMEn local systems:
// assembly of the symmetric block band (FP64 contractions, FP32 result), then
// the odd-even (cyclic) reduction of its block-tridiagonal super-row form, one
// launch pair per level (eliminations, then the Schur updates of the rows
// left), so the factorisation is log2 of the super-row count deep.
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

// O = alpha op(A) op(B) for q x q shared-memory matrices (leading dimension ld); O has
// leading dimension ldo and may be global.
__device__ __forceinline__ void bcr_mm(const float *A, bool ta, const float *B, bool tb, float *O, int ldo, int q,
                                       int ld, float alpha) {
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int r = e / q, c = e % q;
    float s0 = 0.f, s1 = 0.f;
    int k = 0;
    for (; k + 1 < q; k += 2) {
      s0 += (ta ? A[k * ld + r] : A[r * ld + k]) * (tb ? B[c * ld + k] : B[k * ld + c]);
      s1 += (ta ? A[(k + 1) * ld + r] : A[r * ld + k + 1]) * (tb ? B[c * ld + k + 1] : B[(k + 1) * ld + c]);
    }
    if (k < q) s0 += (ta ? A[k * ld + r] : A[r * ld + k]) * (tb ? B[c * ld + k] : B[k * ld + c]);
    O[(long long)r * ldo + c] = alpha * (s0 + s1);
  }
}

// Elimination of the super-rows that are odd multiples of h (j = h + 2 h blockIdx.x), one
// CTA each, or of the top row 0 (root): Cholesky of D_j (a pivot that cancellation drives
// below 1e-6 of the diagonal entry is replaced by that entry: the factor stays SPD and PCG
// checks convergence), Linv_j = L_j^{-1}, Ul_j = Linv_j C_j, Ur_j = Linv_j C_{j+h}^T, and the
// Schur terms SL_j = Ul_j^T Ul_j, SR_j = Ur_j^T Ur_j, CN_j = -Ur_j^T Ul_j for the update.
__global__ void __launch_bounds__(256) k_bcr_elim(const float *__restrict__ D, const float *__restrict__ C, int S,
                                                  int q, int h, int root, float *__restrict__ Linv,
                                                  float *__restrict__ Ul, float *__restrict__ Ur, float *__restrict__ SL,
                                                  float *__restrict__ SR, float *__restrict__ CN) {
  extern __shared__ float bsm[];
  const int ld = q + 1;
  float *Lm = bsm;            // D_j, factored in place (lower triangle)
  float *Li = Lm + q * ld;    // L_j^{-1}
  float *Cl = Li + q * ld;    // C_j: rows of j, columns of j - h
  float *Cr = Cl + q * ld;    // C_{j+h}^T: rows of j, columns of j + h
  float *Wl = Cr + q * ld;    // Ul_j
  float *Wr = Wl + q * ld;    // Ur_j
  float *diag0 = Wr + q * ld;
  __shared__ float inv_s;
  const int j = root ? 0 : h + 2 * h * (int)blockIdx.x;
  const bool hasl = !root, hasr = !root && j + h < S;
  const long long per = (long long)q * q;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < q * q; e += nt) {
    const int r = e / q, c = e % q;
    Lm[r * ld + c] = D[j * per + e];
    Cl[r * ld + c] = hasl ? C[j * per + e] : 0.f;
    Cr[c * ld + r] = hasr ? C[(j + h) * per + e] : 0.f;
  }
  __syncthreads();
  for (int r = tid; r < q; r += nt) diag0[r] = Lm[r * ld + r];
  __syncthreads();
  for (int c = 0; c < q; ++c) {
    if (tid == 0) {
      float piv = Lm[c * ld + c];
      const float d0 = diag0[c];
      if (!(piv > 1e-6f * d0)) piv = (d0 > 0.f) ? d0 : 1.f;
      const float l = sqrtf(piv);
      Lm[c * ld + c] = l;
      inv_s = 1.f / l;
    }
    __syncthreads();
    const float inv = inv_s;
    for (int r = c + 1 + tid; r < q; r += nt) Lm[r * ld + c] *= inv;
    __syncthreads();
    const int w = q - c - 1;
    for (int e = tid; e < w * w; e += nt) {
      const int r = c + 1 + e / w, cc = c + 1 + e % w;
      if (cc <= r) Lm[r * ld + cc] -= Lm[r * ld + c] * Lm[cc * ld + c];
    }
    __syncthreads();
  }
  // L^{-1}: forward substitution against each unit vector, a thread per column
  for (int col = tid; col < q; col += nt)
    for (int r = 0; r < q; ++r) {
      float v = 0.f;
      if (r >= col) {
        float sv = (r == col) ? 1.f : 0.f;
        for (int k = col; k < r; ++k) sv -= Lm[r * ld + k] * Li[k * ld + col];
        v = sv / Lm[r * ld + r];
      }
      Li[r * ld + col] = v;
    }
  __syncthreads();
  for (int e = tid; e < q * q; e += nt) Linv[j * per + e] = Li[(e / q) * ld + e % q];
  if (root) return;
  bcr_mm(Li, false, Cl, false, Wl, ld, q, ld, 1.f);
  bcr_mm(Li, false, Cr, false, Wr, ld, q, ld, 1.f);
  __syncthreads();
  for (int e = tid; e < q * q; e += nt) {
    Ul[j * per + e] = Wl[(e / q) * ld + e % q];
    Ur[j * per + e] = Wr[(e / q) * ld + e % q];
  }
  bcr_mm(Wl, true, Wl, false, SL + j * per, q, q, ld, 1.f);
  bcr_mm(Wr, true, Wr, false, SR + j * per, q, q, ld, 1.f);
  bcr_mm(Wr, true, Wl, false, CN + j * per, q, q, ld, -1.f);
}

// Rows active at the next level (J = 2 h t): D_J -= SR_{J-h} + SL_{J+h}, and C_J becomes
// CN_{J-h}, the coupling of J with J - 2 h through the eliminated row between them.
__global__ void k_bcr_update(float *__restrict__ D, float *__restrict__ C, const float *__restrict__ SL,
                             const float *__restrict__ SR, const float *__restrict__ CN, int S, int q, int h) {
  const long long per = (long long)q * q;
  const long long na = (S + 2LL * h - 1) / (2LL * h);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < na * per;
       t += (long long)gridDim.x * blockDim.x) {
    const long long J = 2LL * h * (t / per), e = t % per;
    float d = D[J * per + e];
    if (J >= h) d -= SR[(J - h) * per + e];
    if (J + h < S) d -= SL[(J + h) * per + e];
    D[J * per + e] = d;
    if (J >= 2LL * h) C[J * per + e] = CN[(J - h) * per + e];
  }
}

constexpr size_t kBcrSmemMax = 100 * 1024;

size_t bcr_smem(int q) { return ((size_t)6 * q * (q + 1) + q) * sizeof(float); }

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
  set_smem_limit_once((const void *)k_bcr_elim, (int)kBcrSmemMax);
  const size_t smem = bcr_smem(q);
  ProfScope ps(c, PROF_PRECOND, 0.0);
  P.levels = 0;
  for (int h = 1; h < S; h <<= 1, ++P.levels) {
    const int ne = (S - h + 2 * h - 1) / (2 * h);
    k_bcr_elim<<<ne, 256, smem, c->stream>>>(D.as<float>(), C.as<float>(), S, q, h, 0, P.Linv.as<float>(),
                                             P.Ul.as<float>(), P.Ur.as<float>(), SL.as<float>(), SR.as<float>(),
                                             CN.as<float>());
    TTI_LAUNCH();
    const long long na = (S + 2LL * h - 1) / (2LL * h);
    k_bcr_update<<<grid1d(na * q * q, 256), 256, 0, c->stream>>>(D.as<float>(), C.as<float>(), SL.as<float>(),
                                                                 SR.as<float>(), CN.as<float>(), S, q, h);
    TTI_LAUNCH();
  }
  k_bcr_elim<<<1, 256, smem, c->stream>>>(D.as<float>(), C.as<float>(), S, q, 0, 1, P.Linv.as<float>(),
                                          P.Ul.as<float>(), P.Ur.as<float>(), SL.as<float>(), SR.as<float>(),
                                          CN.as<float>());
  TTI_LAUNCH();
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
