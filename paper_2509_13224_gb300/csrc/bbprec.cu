// Exact block-band preconditioner of small-interface AMEn local systems:
// assembly of the symmetric block band (FP64 contractions, FP32 result), the
// sequential right-looking block Cholesky in one CTA, and the parallel
// post-pass that turns the factor into the blocks the substitutions use.
// Block size M (4 or 8) is m = rl * rr rounded up; padding rows and columns
// carry the identity.
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

// Right-looking block Cholesky of the block band by one warp.
// The live blocks (i+k, i+l), 0 <= l <= k <= p, sit in a ring of (p+1)^2 block
// slots indexed by absolute block row and column modulo p+1, so nothing moves
// between steps.  Step i: (a) every lane factors the M x M diagonal block
// redundantly in its own registers (no shuffles on the dependent path; the
// reciprocal pivots are the rsqrt results); (b) the panel X_k = W(i+k, i)
// L_ii^{-T} by row-wise forward substitution against the register copy of
// L_ii; (c) the trailing update W(i+k, i+l) -= X_k X_l^T in 4 x 4 register
// tiles, and block row i+1+p (loaded into registers at the start of the step)
// enters the slots of row i.  FP32 throughout: each step is a chain of
// dependent operations, and this is a preconditioner.  A pivot that
// cancellation drives below 1e-6 of the diagonal entry is replaced by that
// entry (the factor stays SPD; PCG checks convergence).
// Outputs: Ld[i] = L_ii (zero above), Lx[i][k-1] = L(i+k, i).
template <int M>
__global__ void __launch_bounds__(32) k_bb_factor(const float *__restrict__ Blow, int n, int p, int m,
                                                   float *__restrict__ Ld, float *__restrict__ Lx,
                                                   unsigned long long *phase_clk) {
  constexpr int BS = M * M, T4 = M / 4, TB = T4 * T4, PE = (BS + 31) / 32;
  // phase_clk (optional): SM clock cycles lane 0 spends in each phase of all steps
  unsigned long long ck0 = 0, ck1 = 0, ck2 = 0, t0 = 0;
  const bool prof = phase_clk != nullptr && threadIdx.x == 0;
  auto stamp = [&](unsigned long long &acc) {
    if (prof) {
      const unsigned long long t1 = clock64();
      acc += t1 - t0;
      t0 = t1;
    }
  };
  extern __shared__ float4 fsm4[];
  float *fsm = reinterpret_cast<float *>(fsm4);
  const int nb = p + 1, P = p * M, npairs = p * (p + 1) / 2;
  float *Wr = fsm;                // nb x nb ring of M x M blocks
  float *Xs = Wr + nb * nb * BS;  // panel [p M][M]
  int *pairs = reinterpret_cast<int *>(Xs + P * M);  // (kb, lb) of pair index, [28][2]
  const int lane = threadIdx.x;
  auto wrap = [nb](int v) { return v >= nb ? v - nb : v; };  // v < 2 nb
  auto slot = [&](int sr, int sc) { return Wr + (sr * nb + sc) * BS; };
  auto ident = [](int e) { return (e / M == e % M) ? 1.f : 0.f; };
  if (lane == 0)
    for (int kb = 1, q = 0; kb <= p; ++kb)
      for (int lb = 1; lb <= kb; ++lb, ++q) {
        pairs[2 * q] = kb;
        pairs[2 * q + 1] = lb;
      }
  for (int k = 0; k < nb; ++k)
    for (int l = 0; l <= k; ++l) {
      float *dst = slot(k, l);
      for (int e = lane; e < BS; e += 32)
        dst[e] = (k < n) ? Blow[((long long)k * nb + (p - k + l)) * BS + e] : (l == k ? ident(e) : 0.f);
    }
  __syncwarp();
  int s0 = 0;  // slot of block row / column i
  for (int i = 0; i < n; ++i, s0 = wrap(s0 + 1)) {
    if (prof) t0 = clock64();
    const int inew = i + 1 + p;
    float pre[8][PE];
#pragma unroll
    for (int l = 0; l < 8; ++l)
#pragma unroll
      for (int u = 0; u < PE; ++u) {
        const int e = lane + u * 32;
        pre[l][u] = 0.f;
        if (l < nb && e < BS)
          pre[l][u] = (inew < n) ? Blow[((long long)inew * nb + l) * BS + e] : (l == p ? ident(e) : 0.f);
      }
    // (a) diagonal block, factored by every lane
    float Lr[M][M], ir[M];
    {
      const float4 *D4 = reinterpret_cast<const float4 *>(slot(s0, s0));
#pragma unroll
      for (int r = 0; r < M; ++r)
#pragma unroll
        for (int c4 = 0; c4 < T4; ++c4) {
          const float4 v = D4[r * T4 + c4];
          Lr[r][4 * c4 + 0] = v.x;
          Lr[r][4 * c4 + 1] = v.y;
          Lr[r][4 * c4 + 2] = v.z;
          Lr[r][4 * c4 + 3] = v.w;
        }
#pragma unroll
      for (int j = 0; j < M; ++j) {
        ir[j] = 1.f;
        if (j < m) {
          float piv = Lr[j][j];
          const float d0 = slot(s0, s0)[j * (M + 1)];
          if (!(piv > 1e-6f * d0)) piv = (d0 > 0.f) ? d0 : 1.f;
          const float inv = rsqrtf(piv);
          ir[j] = inv;
          Lr[j][j] = piv * inv;
#pragma unroll
          for (int r = j + 1; r < M; ++r) Lr[r][j] *= inv;
#pragma unroll
          for (int r = j + 1; r < M; ++r)
#pragma unroll
            for (int c = j + 1; c <= r; ++c) Lr[r][c] -= Lr[r][j] * Lr[c][j];
        }
      }
      if (lane == 0) {
        float4 *dst = reinterpret_cast<float4 *>(Ld + (long long)i * BS);
#pragma unroll
        for (int r = 0; r < M; ++r)
#pragma unroll
          for (int c4 = 0; c4 < T4; ++c4)
            dst[r * T4 + c4] = make_float4(4 * c4 + 0 <= r ? Lr[r][4 * c4 + 0] : 0.f,
                                           4 * c4 + 1 <= r ? Lr[r][4 * c4 + 1] : 0.f,
                                           4 * c4 + 2 <= r ? Lr[r][4 * c4 + 2] : 0.f,
                                           4 * c4 + 3 <= r ? Lr[r][4 * c4 + 3] : 0.f);
      }
    }
    stamp(ck0);
    // (b) panel rows: x (row e of X_k) solves L_ii x = w
    for (int t = lane; t < P; t += 32) {
      const int k = 1 + t / M, e = t % M;
      const float4 *w4 = reinterpret_cast<const float4 *>(slot(wrap(s0 + k), s0) + e * M);
      float x[M];
#pragma unroll
      for (int c4 = 0; c4 < T4; ++c4) {
        const float4 v = w4[c4];
        x[4 * c4 + 0] = v.x;
        x[4 * c4 + 1] = v.y;
        x[4 * c4 + 2] = v.z;
        x[4 * c4 + 3] = v.w;
      }
#pragma unroll
      for (int cc = 0; cc < M; ++cc) {
        x[cc] *= ir[cc];
#pragma unroll
        for (int c = cc + 1; c < M; ++c) x[c] -= Lr[c][cc] * x[cc];
      }
      float4 *xs = reinterpret_cast<float4 *>(Xs + t * M);
      float4 *xg = reinterpret_cast<float4 *>(Lx + (((long long)i * p + (k - 1)) * M + e) * M);
#pragma unroll
      for (int c4 = 0; c4 < T4; ++c4) {
        const float4 v = make_float4(x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2], x[4 * c4 + 3]);
        xs[c4] = v;
        xg[c4] = v;
      }
    }
    __syncwarp();
    stamp(ck1);
    // (c) trailing update in 4 x 4 tiles over block pairs (kb, lb), 1 <= lb <= kb <= p
    for (int t = lane; t < npairs * TB; t += 32) {
      const int pr = t / TB, tt = t % TB;
      const int kb = pairs[2 * pr], lb = pairs[2 * pr + 1];
      const int tr = tt / T4, tc = tt % T4;
      float *dst = slot(wrap(s0 + kb), wrap(s0 + lb)) + (4 * tr) * M + 4 * tc;
      const float *xa = Xs + ((kb - 1) * M + 4 * tr) * M;
      const float *xb = Xs + ((lb - 1) * M + 4 * tc) * M;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4 d = *reinterpret_cast<const float4 *>(dst + a * M);
        acc[a][0] = d.x;
        acc[a][1] = d.y;
        acc[a][2] = d.z;
        acc[a][3] = d.w;
      }
#pragma unroll
      for (int s4 = 0; s4 < T4; ++s4) {
        float4 va[4], vb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          va[a] = *reinterpret_cast<const float4 *>(xa + a * M + 4 * s4);
          vb[a] = *reinterpret_cast<const float4 *>(xb + a * M + 4 * s4);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int bq = 0; bq < 4; ++bq)
            acc[a][bq] -= va[a].x * vb[bq].x + va[a].y * vb[bq].y + va[a].z * vb[bq].z + va[a].w * vb[bq].w;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4 *>(dst + a * M) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
    }
    // block row i+1+p takes the slots of row i: slot row s0, slot columns s0+1+l
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l < nb) {
        float *dst = slot(s0, wrap(s0 + 1 + l));
#pragma unroll
        for (int u = 0; u < PE; ++u) {
          const int e = lane + u * 32;
          if (e < BS) dst[e] = pre[l][u];
        }
      }
    __syncwarp();
    stamp(ck2);
  }
  if (prof) {
    phase_clk[0] = ck0;
    phase_clk[1] = ck1;
    phase_clk[2] = ck2;
  }
}

// Per block row: Linv = L_ii^{-1}, G_k = L_ii^{-1} L(i, i-k), H_k = L_ii^{-T} L(i+k, i)^T
// for k = 1..p, rows padded to the stride S with zeros.  256 / M^2 block rows per
// CTA, one thread per (row, entry) of a block.
template <int M>
__global__ void __launch_bounds__(256) k_bb_post(const float *__restrict__ Ld, const float *__restrict__ Lx, int n,
                                                  int p, float *__restrict__ Linv, float *__restrict__ G,
                                                  float *__restrict__ H) {
  constexpr int BS = M * M, RP = 256 / BS, S = bb_stride(M), M1 = M + 1;
  __shared__ float Lsh[RP][BS], Li[RP][M * M1], X[RP][M * M1];
  const int g = threadIdx.x / BS, lt = threadIdx.x % BS, e = lt / M, f = lt % M;
  const int i = blockIdx.x * RP + g;
  const bool live = i < n;
  Lsh[g][lt] = live ? Ld[(long long)i * BS + lt] : (e == f ? 1.f : 0.f);
  __syncthreads();
  if (lt < M) {
    // column col of L^{-1}: forward substitution against the unit vector
    const int col = lt;
    float v[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
      float sv = (r == col) ? 1.f : 0.f;
#pragma unroll
      for (int q = 0; q < r; ++q) sv -= (q >= col) ? Lsh[g][r * M + q] * v[q] : 0.f;
      v[r] = (r >= col) ? sv / Lsh[g][r * (M + 1)] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < M; ++r) Li[g][r * M1 + col] = v[r];
  }
  __syncthreads();
  if (live) Linv[(long long)i * BS + lt] = Li[g][e * M1 + f];
  for (int k = 1; k <= p; ++k) {
    const long long orow = (((long long)i * p + (k - 1)) * M + e) * S;
    X[g][e * M1 + f] = (live && i - k >= 0) ? Lx[((long long)(i - k) * p + (k - 1)) * BS + e * M + f] : 0.f;
    __syncthreads();
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < M; ++s) acc += Li[g][e * M1 + s] * X[g][s * M1 + f];
    if (live) {
      G[orow + f] = acc;
      if (f < S - M) G[orow + M + f] = 0.f;
    }
    __syncthreads();
    X[g][e * M1 + f] = (live && i + k < n) ? Lx[((long long)i * p + (k - 1)) * BS + e * M + f] : 0.f;
    __syncthreads();
    acc = 0.f;
#pragma unroll
    for (int s = 0; s < M; ++s) acc += Li[g][s * M1 + e] * X[g][f * M1 + s];
    if (live) {
      H[orow + f] = acc;
      if (f < S - M) H[orow + M + f] = 0.f;
    }
    __syncthreads();
  }
}

constexpr size_t kFactorSmemMax = 200 * 1024;

size_t factor_smem(int M, int p) {
  const size_t nb = (size_t)p + 1, BS = (size_t)M * M;
  return (nb * nb * BS + (size_t)p * M * M) * sizeof(float) + 2 * 28 * sizeof(int);
}

template <int M>
void build_m(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, BBPrec &P,
             unsigned long long *phase_clk) {
  const int n = A.n, p = A.p, m = rl * rr;
  constexpr int BS = M * M, S = bb_stride(M), RP = 256 / BS;
  DBuf Blow(c, (size_t)n * (p + 1) * BS * sizeof(float));
  {
    const long long tot = (long long)n * (p + 1) * BS;
    k_bb_build<M><<<grid1d(tot, 256), 256, 0, c->stream>>>(PhiL, rl, A.Rl, A.A, n, p, A.Rr, PhiR, rr,
                                                           Blow.as<float>());
    TTI_LAUNCH();
  }
  DBuf Ld(c, (size_t)n * BS * sizeof(float)), Lx(c, (size_t)n * p * BS * sizeof(float));
  {
    const size_t smem = factor_smem(M, p);
    TTI_CUDA(cudaFuncSetAttribute(k_bb_factor<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax));
    ProfScope ps(c, PROF_PRECOND, 0.0);
    k_bb_factor<M><<<1, 32, smem, c->stream>>>(Blow.as<float>(), n, p, m, Ld.as<float>(), Lx.as<float>(), phase_clk);
    TTI_LAUNCH();
  }
  P.Linv = DBuf(c, (size_t)n * BS * sizeof(float));
  P.G = DBuf(c, (size_t)n * p * M * S * sizeof(float));
  P.H = DBuf(c, (size_t)n * p * M * S * sizeof(float));
  k_bb_post<M><<<(n + RP - 1) / RP, 256, 0, c->stream>>>(Ld.as<float>(), Lx.as<float>(), n, p, P.Linv.as<float>(),
                                                         P.G.as<float>(), P.H.as<float>());
  TTI_LAUNCH();
}

}  // namespace

bool bb_eligible(int m, int n, int p) {
  return m >= 1 && m <= kBBMaxM && n >= 1 && n <= 1024 && p >= 1 && p <= 7 &&
         factor_smem(bb_pad(m), p) <= kFactorSmemMax;
}

void bb_prec_build(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, BBPrec &P,
                   unsigned long long *phase_clk) {
  const int m = rl * rr;
  TTI_CHECK_ARG(bb_eligible(m, A.n, A.p), "block-band preconditioner: m=%d n=%d p=%d out of range", m, A.n, A.p);
  P.n = A.n;
  P.p = A.p;
  P.m = m;
  P.M = bb_pad(m);
  if (P.M == 4) build_m<4>(c, PhiL, rl, A, PhiR, rr, P, phase_clk);
  else build_m<8>(c, PhiL, rl, A, PhiR, rr, P, phase_clk);
}

}  // namespace ttiga
