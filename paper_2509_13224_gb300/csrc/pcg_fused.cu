// Fused preconditioned conjugate gradients for one AMEn local system.
//
// One cooperative launch runs every PCG iteration of a local solve
//   B d = r,  B = PhiL (x) A_k (x) PhiR,  preconditioner = band block-Jacobi,
// so the local solve costs one launch instead of about a dozen launches and a
// host read-back per iteration.  Each iteration is six grid-wide phases:
//   A  T1 = p PhiR^T            (dense, right interface)
//   B  T2 = band(A_k, T1)       (banded operator core)
//   C  q  = PhiL T2,  <p, q>    (dense, left interface; partial dot)
//   D  x += alpha p, r -= alpha q, <r, r>
//   E  stop test; z = P^{-1} r (one thread per (alpha, beta) band system), <r, z>
//   F  p = z + beta p
// Reductions are deterministic: every CTA writes one partial per phase and
// all CTAs sum the partials in the same order.  The grid barrier spins with an
// iteration limit; on expiry it raises an error flag and the kernel returns.
#include <algorithm>

#include "amen_ops.cuh"
#include "pcg_fused.cuh"

namespace ttiga {

struct Barrier {
  unsigned int count;
  unsigned int gen;
};

namespace {

constexpr long long kSpinLimit = 1LL << 24;  // x 64 ns sleep: about one second

__device__ __forceinline__ bool grid_sync(Barrier *bar, unsigned int nblocks, int *err) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int *vgen = &bar->gen;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > kSpinLimit) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int *)err) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Sum of one double per thread over the CTA; thread 0 writes it to part[blockIdx.x].
__device__ __forceinline__ void cta_partial(double v, double *part) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
  __syncthreads();
}

// Same-order sum of the partials, broadcast to the CTA.
__device__ __forceinline__ double grid_total(const double *part) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) t += ((volatile const double *)part)[b];
    tot = t;
  }
  __syncthreads();
  const double v = tot;
  __syncthreads();
  return v;
}

template <typename T, int PB>
__device__ __forceinline__ double band_solve_pair(const T *__restrict__ L, int rl, int n, int rr, const T *r, T *z,
                                                  int t) {
  // forward / backward substitution of one (alpha, beta) band system; returns <r, z> over it
  const int npair = rl * rr;
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
  for (int k = 0; k < PB; ++k) w[k] = T(0);
  double rz = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    T sv = z[base + (long long)i * rr];
#pragma unroll
    for (int d = 1; d <= PB; ++d)
      if (i + d < n) sv -= L[((long long)(i + d) * (PB + 1) + (PB - d)) * npair + t] * w[d - 1];
    const T zi = sv * L[((long long)i * (PB + 1) + PB) * npair + t];
    z[base + (long long)i * rr] = zi;
    rz += (double)r[base + (long long)i * rr] * (double)zi;
#pragma unroll
    for (int d = PB - 1; d > 0; --d) w[d] = w[d - 1];
    w[0] = zi;
  }
  return rz;
}

template <typename T, int PB>
__global__ void __launch_bounds__(256) k_pcg_fused(PcgArgs<T> a) {
  const int rl = a.rl, rr = a.rr, Rl = a.Rl, Rr = a.Rr, n = a.n, b = 2 * PB + 1;
  const long long N = (long long)rl * n * rr;
  const long long nA = (long long)rl * n * rr * Rr, nB = (long long)Rl * rl * n * rr;
  const int npair = rl * rr;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
  const unsigned int G = gridDim.x;
  double *p_pq = a.part, *p_rr = a.part + G, *p_rz = a.part + 2 * G;

  // x = 0, r = b
  for (long long e = tid; e < N; e += nth) {
    a.x[e] = T(0);
    a.r[e] = a.b[e];
  }
  if (!grid_sync(a.bar, G, a.err)) return;
  double rz_loc = 0.0;
  for (long long t = tid; t < npair; t += nth) rz_loc += band_solve_pair<T, PB>(a.L, rl, n, rr, a.r, a.z, (int)t);
  double rr_loc = 0.0;
  for (long long e = tid; e < N; e += nth) rr_loc += (double)a.r[e] * (double)a.r[e];
  cta_partial(rz_loc, p_rz);
  cta_partial(rr_loc, p_rr);
  if (!grid_sync(a.bar, G, a.err)) return;
  double rz = grid_total(p_rz);
  double res2 = grid_total(p_rr);
  for (long long e = tid; e < N; e += nth) a.pv[e] = a.z[e];
  int it = 0;
  if (res2 > a.tol2) {
    if (!grid_sync(a.bar, G, a.err)) return;
    for (; it < a.maxit; ++it) {
      // A: T1[(aa, j)][(c, d)] = sum_e p[aa][j][e] PhiR[c][d][e]
      for (long long e = tid; e < nA; e += nth) {
        const int d = (int)(e % Rr);
        long long t = e / Rr;
        const int c = (int)(t % rr);
        const long long row = t / rr;  // aa * n + j
        const T *pr = a.pv + row * rr;
        const T *ph = a.PhiR + ((long long)c * Rr + d) * rr;
        T s = T(0);
        for (int f = 0; f < rr; ++f) s += pr[f] * ph[f];
        a.T1[e] = s;
      }
      if (!grid_sync(a.bar, G, a.err)) return;
      // B: T2[g][aa][i][c] = sum_{o, d} A[g][i][o][d] T1[aa][i+o-p][c][d]
      for (long long e = tid; e < nB; e += nth) {
        const int c = (int)(e % rr);
        long long t = e / rr;
        const int i = (int)(t % n);
        t /= n;
        const int aa = (int)(t % rl);
        const int g = (int)(t / rl);
        const T *Ar = a.A + ((long long)g * n + i) * b * Rr;
        T s = T(0);
#pragma unroll
        for (int o = 0; o < b; ++o) {
          const int j = i + o - PB;
          if (j < 0 || j >= n) continue;
          const T *Ao = Ar + o * Rr;
          const T *Tj = a.T1 + (((long long)aa * n + j) * rr + c) * Rr;
          for (int d = 0; d < Rr; ++d) s += Ao[d] * Tj[d];
        }
        a.T2[e] = s;
      }
      if (!grid_sync(a.bar, G, a.err)) return;
      // C: q[al][i][c] = sum_{g, aa} PhiL[al][g][aa] T2[g][aa][i][c];  <p, q>
      double pq_loc = 0.0;
      for (long long e = tid; e < N; e += nth) {
        const long long ic = e % ((long long)n * rr);
        const int al = (int)(e / ((long long)n * rr));
        const T *ph = a.PhiL + (long long)al * Rl * rl;
        T s = T(0);
        for (int g = 0; g < Rl; ++g)
          for (int aa = 0; aa < rl; ++aa) s += ph[g * rl + aa] * a.T2[((long long)g * rl + aa) * n * rr + ic];
        a.q[e] = s;
        pq_loc += (double)a.pv[e] * (double)s;
      }
      cta_partial(pq_loc, p_pq);
      if (!grid_sync(a.bar, G, a.err)) return;
      // D: x += alpha p, r -= alpha q;  <r, r>
      const double pq = grid_total(p_pq);
      const double alpha = (pq != 0.0) ? rz / pq : 0.0;
      rr_loc = 0.0;
      for (long long e = tid; e < N; e += nth) {
        a.x[e] += (T)alpha * a.pv[e];
        const T rv = a.r[e] - (T)alpha * a.q[e];
        a.r[e] = rv;
        rr_loc += (double)rv * (double)rv;
      }
      cta_partial(rr_loc, p_rr);
      if (!grid_sync(a.bar, G, a.err)) return;
      // E: stop test, z = P^{-1} r, <r, z>
      res2 = grid_total(p_rr);
      if (res2 <= a.tol2 || !(pq > 0.0)) {
        ++it;
        break;
      }
      rz_loc = 0.0;
      for (long long t = tid; t < npair; t += nth) rz_loc += band_solve_pair<T, PB>(a.L, rl, n, rr, a.r, a.z, (int)t);
      cta_partial(rz_loc, p_rz);
      if (!grid_sync(a.bar, G, a.err)) return;
      // F: p = z + beta p
      const double rz_new = grid_total(p_rz);
      const double beta = (rz != 0.0) ? rz_new / rz : 0.0;
      rz = rz_new;
      for (long long e = tid; e < N; e += nth) a.pv[e] = a.z[e] + (T)beta * a.pv[e];
      if (!grid_sync(a.bar, G, a.err)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = (double)it;
    a.out[1] = res2;
  }
}

template <typename T, int PB> const void *kernel_ptr() { return (const void *)k_pcg_fused<T, PB>; }

template <typename T> const void *pick(int p) {
  switch (p) {
    case 1: return kernel_ptr<T, 1>();
    case 2: return kernel_ptr<T, 2>();
    case 3: return kernel_ptr<T, 3>();
    case 4: return kernel_ptr<T, 4>();
    case 5: return kernel_ptr<T, 5>();
    case 6: return kernel_ptr<T, 6>();
    case 7: return kernel_ptr<T, 7>();
    default: fail(TT_IGA_ERR_ARG, "pcg: degree %d outside 1..7", p);
  }
}

}  // namespace

template <typename T> int pcg_fused_grid(Ctx *c, const PcgArgs<T> &a) {
  // One thread per output of the widest phase (the band stage or the right-interface
  // stage), all CTAs co-resident; the FP64 pipe needs every SM, so small systems
  // still spread over the whole GPU while the work allows at least one output per thread.
  const void *k = pick<T>(a.p);
  int per_sm = 0;
  TTI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0));
  const long long nA = (long long)a.rl * a.n * a.rr * a.Rr, nB = (long long)a.Rl * a.rl * a.n * a.rr;
  const long long work = std::max(nA, nB);
  long long g = (work + 255) / 256;
  const long long cap = (long long)c->num_sms * std::max(1, std::min(per_sm, 2));
  g = std::max<long long>(1, std::min(g, cap));
  return (int)g;
}

template <typename T> void pcg_fused(Ctx *c, PcgArgs<T> a, int grid) {
  const void *k = pick<T>(a.p);
  TTI_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(Barrier), c->stream));
  void *args[] = {&a};
  {
    ProfScope ps(c, PROF_PCG_FUSED, 0.0);
    TTI_CUDA(cudaLaunchCooperativeKernel(k, dim3(grid), dim3(256), args, 0, c->stream));
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template int pcg_fused_grid<double>(Ctx *, const PcgArgs<double> &);
template int pcg_fused_grid<float>(Ctx *, const PcgArgs<float> &);
template void pcg_fused<double>(Ctx *, PcgArgs<double>, int);
template void pcg_fused<float>(Ctx *, PcgArgs<float>, int);

}  // namespace ttiga
