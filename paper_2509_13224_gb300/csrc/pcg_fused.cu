// Fused preconditioned conjugate gradients for one AMEn local system.
//
// One cooperative launch runs every PCG iteration of a local solve
//   B d = r,  B = PhiL (x) A_k (x) PhiR,  preconditioner = band block-Jacobi,
// so the local solve costs one launch instead of about a dozen launches and a
// host read-back per iteration.  Each iteration is four grid-wide phases:
//   A  p = z + beta p_prev (double-buffered), T1 = p PhiR^T  (right interface)
//   B  T2 = band(A_k, T1)                                    (operator core)
//   C  q  = PhiL T2,  <p, q>                                 (left interface)
//   E  per (alpha, beta) band system: x += alpha p, r -= alpha q,
//      z = P^{-1} r;  <r, r>, <r, z>; stop test after the barrier
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

constexpr size_t kPcgSmemBytes = 200 * 1024;
constexpr long long kSpinLimit = 1LL << 22;  // polls of about 0.25-0.5 us: one to two seconds

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acqrel(unsigned int *p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(unsigned int *p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned int *p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier over co-resident CTAs (cooperative launch): arrival counter
// plus generation number; the last arriver resets the counter and releases the
// generation, the others poll it with acquire loads.  A wait that exceeds the
// poll limit sets *err and returns false instead of hanging.
__device__ __forceinline__ bool grid_sync(Barrier *bar, unsigned int nblocks, int *err) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int g = ld_acquire(&bar->gen);
    if (atom_add_acqrel(&bar->count, 1u) == nblocks - 1) {
      st_relaxed(&bar->count, 0u);
      red_add_release(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (ld_acquire(&bar->gen) == g) {
        if (++spins > kSpinLimit) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
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

// Sum of the per-CTA partials, identical on every CTA (fixed lane assignment and
// shuffle order), broadcast to the CTA.  Warp 0 loads the partials in parallel.
__device__ __forceinline__ double grid_total(const double *part) {
  __shared__ double tot;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += 32) t += ((volatile const double *)part)[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) tot = t;
  }
  __syncthreads();
  const double v = tot;
  __syncthreads();
  return v;
}

// Phase timestamps of CTA 0 (global timer, ns) when a trace buffer is given.
__device__ __forceinline__ void trace_mark(unsigned long long *trace, int cap, int &slot) {
  if (trace && blockIdx.x == 0 && threadIdx.x == 0 && slot < cap) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    trace[slot] = t;
  }
  ++slot;
}

// The (alpha, beta) band systems of the preconditioner, `slots` at a time per
// CTA.  All threads of the CTA gather each system's factor rows (FP32) and its
// entries of r, q, p, x, apply x += alpha p, r -= alpha q (or x = 0, r = b when
// init) in parallel, and stage r in shared memory; lane 0 of warp w then runs
// system w's forward / backward substitution in FP32 out of shared memory
// (the only sequential part; on GB300 a dependent FP64 operation costs about
// 64 cycles against 4.5 for FP32, and a preconditioner needs no accuracy);
// finally the CTA scatters z in the working precision and accumulates <r, r>
// and <r, z> in FP64 with every thread on its own chain.
// Shared layout per slot: L[n][PB+1] (float), r[n] (float).
template <typename T, int PB>
__device__ __forceinline__ void band_systems(const PcgArgs<T> &a, const T *__restrict__ pcur, double alpha, bool init,
                                             double &rr_out, double &rz_out) {
  extern __shared__ unsigned char esm_raw[];
  float *esm = reinterpret_cast<float *>(esm_raw);
  const int rl = a.rl, rr = a.rr, n = a.n, slots = a.slots;
  const int npair = rl * rr;
  const int per = n * (PB + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long t0 = (long long)blockIdx.x * slots; t0 < npair; t0 += (long long)gridDim.x * slots) {
    const int cnt = (int)((npair - t0 < slots) ? (npair - t0) : slots);
    for (int e = threadIdx.x; e < cnt * n * (PB + 1); e += blockDim.x) {
      const int s_ = e / (n * (PB + 1)), rem = e - s_ * (n * (PB + 1));
      const int i = rem / (PB + 1), k = rem - i * (PB + 1);
      esm[s_ * per + rem] = a.Lf[((long long)i * (PB + 1) + k) * npair + t0 + s_];
    }
    double rr_th = 0.0;
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
      const int s_ = e / n, i = e - s_ * n;
      const long long t = t0 + s_;
      const long long idx = ((t / rr) * n + i) * rr + (t % rr);
      T r;
      if (init) {
        r = a.b[idx];
        a.x[idx] = T(0);
      } else {
        a.x[idx] += (T)alpha * pcur[idx];
        r = a.r[idx] - (T)alpha * a.q[idx];
      }
      a.r[idx] = r;
      rr_th += (double)r * (double)r;
      esm[s_ * per + n * (PB + 1) + i] = (float)r;
    }
    rr_out += rr_th;
    __syncthreads();
    if (warp < cnt && lane == 0) {
      const float *Ls = esm + warp * per;
      float *rs = esm + warp * per + n * (PB + 1);  // overwritten by z
      float w[PB];
#pragma unroll
      for (int k = 0; k < PB; ++k) w[k] = 0.f;
      for (int i = 0; i < n; ++i) {
        const float *Li = Ls + i * (PB + 1);
        float sv = rs[i];
#pragma unroll
        for (int k = 0; k < PB; ++k) sv -= Li[k] * w[k];
        const float y = sv * Li[PB];
        rs[i] = y;
#pragma unroll
        for (int k = 0; k + 1 < PB; ++k) w[k] = w[k + 1];
        w[PB - 1] = y;
      }
#pragma unroll
      for (int k = 0; k < PB; ++k) w[k] = 0.f;  // w[d-1] = z_{i+d}
      for (int i = n - 1; i >= 0; --i) {
        float sv = rs[i];
#pragma unroll
        for (int d = 1; d <= PB; ++d)
          if (i + d < n) sv -= Ls[(i + d) * (PB + 1) + (PB - d)] * w[d - 1];
        const float zi = sv * Ls[i * (PB + 1) + PB];
        rs[i] = zi;
#pragma unroll
        for (int d = PB - 1; d > 0; --d) w[d] = w[d - 1];
        w[0] = zi;
      }
    }
    __syncthreads();
    double rz_th = 0.0;
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
      const int s_ = e / n, i = e - s_ * n;
      const long long t = t0 + s_;
      const long long idx = ((t / rr) * n + i) * rr + (t % rr);
      const T zi = (T)esm[s_ * per + n * (PB + 1) + i];
      a.z[idx] = zi;
      rz_th += (double)a.r[idx] * (double)zi;
    }
    rz_out += rz_th;
    __syncthreads();
  }
}

template <typename T, int PB>
__global__ void __launch_bounds__(256, 1) k_pcg_fused(PcgArgs<T> a) {
  const int rl = a.rl, rr = a.rr, Rl = a.Rl, Rr = a.Rr, n = a.n, b = 2 * PB + 1;
  const unsigned int G = gridDim.x;
  double *p_pq = a.part, *p_rr = a.part + G, *p_rz = a.part + 2 * G;

  int slot = 0;
  trace_mark(a.trace, a.trace_cap, slot);
  // r = b, x = 0, z = P^{-1} r;  <r, r>, <r, z>
  double rr_loc = 0.0, rz_loc = 0.0;
  band_systems<T, PB>(a, nullptr, 0.0, true, rr_loc, rz_loc);
  cta_partial(rr_loc, p_rr);
  cta_partial(rz_loc, p_rz);
  if (!grid_sync(a.bar, G, a.err)) return;
  trace_mark(a.trace, a.trace_cap, slot);
  double res2 = grid_total(p_rr);
  double rz = grid_total(p_rz), rz_prev = 1.0;
  int it = 0;
  for (; it < a.maxit && res2 > a.tol2; ++it) {
    const double beta = (it == 0 || rz_prev == 0.0) ? 0.0 : rz / rz_prev;
    T *pcur = (it & 1) ? a.pv2 : a.pv;
    const T *pprev = (it & 1) ? a.pv : a.pv2;
    // A+B+C on slabs of S mode rows, one slab per CTA at a time, so only CTA barriers
    // are needed: T1 on the slab plus its +-p halo rows (recomputed from z and p_prev),
    // T2 and q on the slab rows, <p, q> partial.  p rows of the slab are written once.
    double pq_loc = 0.0;
    {
      const int S = a.slab, nslab = (n + S - 1) / S;
      T *T1s = a.T1 + (long long)blockIdx.x * a.t1_stride;
      T *T2s = a.T2 + (long long)blockIdx.x * a.t2_stride;
      for (int sl = blockIdx.x; sl < nslab; sl += G) {
        const int i0 = sl * S, i1 = min(n, i0 + S);
        const int j0 = max(0, i0 - PB), j1 = min(n, i1 + PB);
        const int nj = j1 - j0, ni = i1 - i0;
        // A: T1s[aa][jj][c][d] = sum_f p[aa][j][f] PhiR[c][d][f], p = z + beta p_prev
        const int nA1 = rl * nj * rr * Rr;
        for (int e = threadIdx.x; e < nA1; e += blockDim.x) {
          const int d = e % Rr;
          int t = e / Rr;
          const int c = t % rr;
          t /= rr;
          const int jj = t % nj, aa = t / nj;
          const int j = j0 + jj;
          const long long row = (long long)aa * n + j;
          const T *zr = a.z + row * rr;
          const T *pr = pprev + row * rr;
          const T *ph = a.PhiR + ((long long)c * Rr + d) * rr;
          const bool writer = (c == 0 && d == 0 && j >= i0 && j < i1);
          T s0 = T(0), s1 = T(0);
          for (int f = 0; f < rr; ++f) {
            const T pf = (it == 0) ? zr[f] : zr[f] + (T)beta * pr[f];
            if (writer) pcur[row * rr + f] = pf;
            if (f & 1) s1 += pf * ph[f]; else s0 += pf * ph[f];
          }
          T1s[e] = s0 + s1;
        }
        __syncthreads();
        // B: T2s[g][aa][ii][c] = sum_{o, d} A[g][i][o][d] T1s[aa][i+o-p-j0][c][d]
        const int nB1 = Rl * rl * ni * rr;
        for (int e = threadIdx.x; e < nB1; e += blockDim.x) {
          const int c = e % rr;
          int t = e / rr;
          const int ii = t % ni;
          t /= ni;
          const int aa = t % rl, g = t / rl;
          const int i = i0 + ii;
          const T *Ar = a.A + ((long long)g * n + i) * b * Rr;
          T s0 = T(0), s1 = T(0);
#pragma unroll
          for (int o = 0; o < b; ++o) {
            const int j = i + o - PB;
            if (j < 0 || j >= n) continue;
            const T *Ao = Ar + o * Rr;
            const T *Tj = T1s + (((long long)aa * nj + (j - j0)) * rr + c) * Rr;
            if (o & 1)
              for (int d = 0; d < Rr; ++d) s1 += Ao[d] * Tj[d];
            else
              for (int d = 0; d < Rr; ++d) s0 += Ao[d] * Tj[d];
          }
          T2s[e] = s0 + s1;
        }
        __syncthreads();
        // C: q[al][i][c] = sum_{g, aa} PhiL[al][g][aa] T2s[g][aa][ii][c];  <p, q>
        const int nC1 = rl * ni * rr;
        const int ga = Rl * rl;
        for (int e = threadIdx.x; e < nC1; e += blockDim.x) {
          const int c = e % rr;
          const int t = e / rr;
          const int ii = t % ni, al = t / ni;
          const T *ph = a.PhiL + (long long)al * ga;
          T s4[4] = {T(0), T(0), T(0), T(0)};
          for (int q = 0; q < ga; ++q) s4[q & 3] += ph[q] * T2s[((long long)q * ni + ii) * rr + c];
          const T sv = (s4[0] + s4[1]) + (s4[2] + s4[3]);
          const long long idx = ((long long)al * n + i0 + ii) * rr + c;
          a.q[idx] = sv;
          pq_loc += (double)pcur[idx] * (double)sv;
        }
        __syncthreads();
      }
    }
    cta_partial(pq_loc, p_pq);
    if (!grid_sync(a.bar, G, a.err)) return;
    trace_mark(a.trace, a.trace_cap, slot);
    // E: x += alpha p, r -= alpha q, z = P^{-1} r per band system;  <r, r>, <r, z>
    const double pq = grid_total(p_pq);
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    rr_loc = 0.0;
    rz_loc = 0.0;
    band_systems<T, PB>(a, pcur, alpha, false, rr_loc, rz_loc);
    cta_partial(rr_loc, p_rr);
    cta_partial(rz_loc, p_rz);
    if (!grid_sync(a.bar, G, a.err)) return;
    trace_mark(a.trace, a.trace_cap, slot);
    res2 = grid_total(p_rr);
    rz_prev = rz;
    rz = grid_total(p_rz);
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

// Band systems staged per CTA at a time (one warp each) and the shared memory they need.
template <typename T> static int band_slots(const PcgArgs<T> &a) {
  const size_t per = (size_t)a.n * (a.p + 2) * sizeof(float);
  int slots = (int)std::min<size_t>(8, kPcgSmemBytes / std::max<size_t>(per, 1));
  return std::max(1, slots);
}

template <typename T> int pcg_fused_grid(Ctx *c, PcgArgs<T> &a) {
  // Slabs of S mode rows for the dense phase (at least 256 band-stage outputs
  // each), enough CTAs for the slabs and for the band systems, all co-resident.
  const void *k = pick<T>(a.p);
  a.slots = band_slots(a);
  a.smem = (int)((size_t)a.slots * a.n * (a.p + 2) * sizeof(float));
  TTI_CHECK_ARG((size_t)a.n * (a.p + 2) * sizeof(float) <= kPcgSmemBytes, "pcg: n=%d too large for one band system",
                a.n);
  TTI_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPcgSmemBytes));
  int per_sm = 0;
  TTI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, a.smem));
  TTI_CHECK_ARG(per_sm >= 1, "pcg: kernel does not fit on an SM");
  const long long cap = (long long)c->num_sms * std::max(1, std::min(per_sm, 2));
  const long long row_out = (long long)a.Rl * a.rl * a.rr;
  long long S = std::max<long long>((256 + row_out - 1) / row_out, (a.n + cap - 1) / cap);
  S = std::max<long long>(1, std::min<long long>(S, a.n));
  a.slab = (int)S;
  const long long nslab = (a.n + S - 1) / S;
  const long long npair = (long long)a.rl * a.rr;
  long long g = std::max(nslab, (npair + a.slots - 1) / a.slots);
  g = std::max<long long>(1, std::min(g, cap));
  a.t1_stride = (long long)a.rl * (S + 2 * a.p) * a.rr * a.Rr;
  a.t2_stride = (long long)a.Rl * a.rl * S * a.rr;
  return (int)g;
}

template <typename T> void pcg_fused(Ctx *c, PcgArgs<T> a, int grid) {
  const void *k = pick<T>(a.p);
  TTI_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(Barrier), c->stream));
  void *args[] = {&a};
  {
    ProfScope ps(c, PROF_PCG_FUSED, 0.0);
    TTI_CUDA(cudaLaunchCooperativeKernel(k, dim3(grid), dim3(256), args, (size_t)a.smem, c->stream));
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template int pcg_fused_grid<double>(Ctx *, PcgArgs<double> &);
template int pcg_fused_grid<float>(Ctx *, PcgArgs<float> &);
template void pcg_fused<double>(Ctx *, PcgArgs<double>, int);
template void pcg_fused<float>(Ctx *, PcgArgs<float>, int);

}  // namespace ttiga
