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
#pragma once
#include <algorithm>

#include <type_traits>

#include "amen_ops.cuh"
#include "bbprec.cuh"
#include "pcg_fused.cuh"
#include "tc_tf32.cuh"

namespace ttiga {

struct Barrier {
  unsigned int count;
  unsigned int gen;
};

namespace {

constexpr size_t kPcgSmemBytes = 220 * 1024;
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

// Banded triangular solves of one band system by one warp, in FP32 out of
// shared memory.  The forward solve y_i = (r_i - sum_k L_i[k] y_{i-PB+k}) d_i
// (L_i[k] = L(i, i-PB+k), d_i the reciprocal diagonal) is an affine
// recurrence in the state s_i = (y_{i-PB+1}, .., y_i): s_i = M_i s_{i-1} + u_i.
// The rows are cut into 32 contiguous chunks, one per lane; each lane composes
// the maps of its chunk, a Hillis-Steele scan over the lanes composes the chunk
// maps (5 shuffle rounds), and each lane reruns its chunk from its true start
// state.  The backward solve z_i = (y_i - sum_d L(i+d, i) z_{i+d}) d_i is the
// same recurrence with the rows taken from the bottom.  The dependent chain is
// about n/32 + 5 compositions instead of n rows.  A preconditioner needs no
// accuracy; the recurrences of a banded SPD factor do not grow, so FP32 suffices.
template <int PB>
__device__ __forceinline__ void warp_band_sweep(const float *__restrict__ Ls, float *__restrict__ v, int n, int lane,
                                                bool backward) {
  const int c = (n + 31) >> 5;
  const int q = backward ? 31 - lane : lane;  // chunk index of this lane
  const int lo = min(n, q * c), hi = min(n, lo + c);
  // coefficient of state component k for row i; the reciprocal diagonal is Ls[i (PB+1) + PB]
  auto coef = [&](int i, int k) -> float {
    if (!backward) return Ls[i * (PB + 1) + k];
    const int row = i + PB - k;  // L(i + d, i) with d = PB - k
    return row < n ? Ls[row * (PB + 1) + k] : 0.f;
  };
  float M[PB][PB], u[PB];
#pragma unroll
  for (int j = 0; j < PB; ++j) {
#pragma unroll
    for (int k = 0; k < PB; ++k) M[j][k] = (j == k) ? 1.f : 0.f;
    u[j] = 0.f;
  }
  for (int t = 0; t < hi - lo; ++t) {
    const int i = backward ? hi - 1 - t : lo + t;
    const float d = Ls[i * (PB + 1) + PB];
    float Mn[PB], un = v[i];
#pragma unroll
    for (int k = 0; k < PB; ++k) Mn[k] = 0.f;
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const float lj = coef(i, j);
#pragma unroll
      for (int k = 0; k < PB; ++k) Mn[k] -= lj * M[j][k];
      un -= lj * u[j];
    }
#pragma unroll
    for (int j = 0; j + 1 < PB; ++j) {
#pragma unroll
      for (int k = 0; k < PB; ++k) M[j][k] = M[j + 1][k];
      u[j] = u[j + 1];
    }
#pragma unroll
    for (int k = 0; k < PB; ++k) M[PB - 1][k] = Mn[k] * d;
    u[PB - 1] = un * d;
  }
  // inclusive scan: (M, u) <- (M, u) o (M', u') of the lane `off` below (earlier rows)
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    float Mp[PB][PB], up[PB];
#pragma unroll
    for (int j = 0; j < PB; ++j) {
#pragma unroll
      for (int k = 0; k < PB; ++k) Mp[j][k] = __shfl_up_sync(0xffffffffu, M[j][k], off);
      up[j] = __shfl_up_sync(0xffffffffu, u[j], off);
    }
    if (lane >= off) {
      float Mc[PB][PB], uc[PB];
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        float a = u[j];
#pragma unroll
        for (int k = 0; k < PB; ++k) {
          float m = 0.f;
#pragma unroll
          for (int l = 0; l < PB; ++l) m += M[j][l] * Mp[l][k];
          Mc[j][k] = m;
          a += M[j][k] * up[k];
        }
        uc[j] = a;
      }
#pragma unroll
      for (int j = 0; j < PB; ++j) {
#pragma unroll
        for (int k = 0; k < PB; ++k) M[j][k] = Mc[j][k];
        u[j] = uc[j];
      }
    }
  }
  // start state of this chunk: the composed map of the chunks before it applied to 0
  float st[PB];
#pragma unroll
  for (int j = 0; j < PB; ++j) {
    const float w = __shfl_up_sync(0xffffffffu, u[j], 1);
    st[j] = lane == 0 ? 0.f : w;
  }
  for (int t = 0; t < hi - lo; ++t) {
    const int i = backward ? hi - 1 - t : lo + t;
    float sv = v[i];
#pragma unroll
    for (int k = 0; k < PB; ++k) sv -= coef(i, k) * st[k];
    const float y = sv * Ls[i * (PB + 1) + PB];
    v[i] = y;
#pragma unroll
    for (int k = 0; k + 1 < PB; ++k) st[k] = st[k + 1];
    st[PB - 1] = y;
  }
}

// The (alpha, beta) band systems of the preconditioner, `slots` at a time per
// CTA.  All threads of the CTA apply x += alpha p, r -= alpha q (or x = 0,
// r = b when init) to each system's entries in parallel and stage r in shared
// memory; warp w then solves system w (warp_band_sweep, forward and backward);
// finally the CTA scatters z in the working precision and accumulates <r, r>
// and <r, z> in FP64 with every thread on its own chain.  The FP32 factor rows
// of the CTA's systems are gathered into shared memory once, at init, when
// every system has its own slot in the grid (a.resident), else per round.
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
    if (init || !a.resident) {
      for (int e = threadIdx.x; e < cnt * n * (PB + 1); e += blockDim.x) {
        const int s_ = e / (n * (PB + 1)), rem = e - s_ * (n * (PB + 1));
        const int i = rem / (PB + 1), k = rem - i * (PB + 1);
        esm[s_ * per + rem] = a.Lf[((long long)i * (PB + 1) + k) * npair + t0 + s_];
      }
    }
    // entries are taken BU per thread at a time, all loads first, so a thread waits for one
    // memory latency per batch rather than per entry (the entries of a system are rr apart)
    constexpr int BU = 4;
    double rr_th = 0.0;
    for (int e0 = threadIdx.x; e0 < cnt * n; e0 += BU * blockDim.x) {
      long long ix[BU];
      int sl[BU];
      T xv[BU], pv[BU], rv[BU], qv[BU];
#pragma unroll
      for (int u = 0; u < BU; ++u) {
        const int e = e0 + u * blockDim.x;
        ix[u] = -1;
        xv[u] = pv[u] = rv[u] = qv[u] = T(0);
        if (e < cnt * n) {
          const int s_ = e / n, i = e - s_ * n;
          const long long t = t0 + s_;
          ix[u] = ((t / rr) * n + i) * rr + (t % rr);
          sl[u] = s_ * per + n * (PB + 1) + i;
          if (init) {
            rv[u] = a.b[ix[u]];
          } else {
            xv[u] = a.x[ix[u]];
            pv[u] = pcur[ix[u]];
            rv[u] = a.r[ix[u]];
            qv[u] = a.q[ix[u]];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < BU; ++u) {
        if (ix[u] < 0) continue;
        T r;
        if (init) {
          r = rv[u];
          a.x[ix[u]] = T(0);
        } else {
          a.x[ix[u]] = xv[u] + (T)alpha * pv[u];
          r = rv[u] - (T)alpha * qv[u];
        }
        a.r[ix[u]] = r;
        rr_th += (double)r * (double)r;
        esm[sl[u]] = (float)r;
      }
    }
    rr_out += rr_th;
    __syncthreads();
    if (warp < cnt) {
      const float *Ls = esm + warp * per;
      float *rs = esm + warp * per + n * (PB + 1);  // r, overwritten by y, then by z
      warp_band_sweep<PB>(Ls, rs, n, lane, false);
      __syncwarp();
      warp_band_sweep<PB>(Ls, rs, n, lane, true);
    }
    __syncthreads();
    double rz_th = 0.0;
    for (int e0 = threadIdx.x; e0 < cnt * n; e0 += BU * blockDim.x) {
      long long ix[BU];
      T rv[BU], zv[BU];
#pragma unroll
      for (int u = 0; u < BU; ++u) {
        const int e = e0 + u * blockDim.x;
        ix[u] = -1;
        rv[u] = zv[u] = T(0);
        if (e < cnt * n) {
          const int s_ = e / n, i = e - s_ * n;
          const long long t = t0 + s_;
          ix[u] = ((t / rr) * n + i) * rr + (t % rr);
          rv[u] = a.r[ix[u]];
          zv[u] = (T)esm[s_ * per + n * (PB + 1) + i];
        }
      }
#pragma unroll
      for (int u = 0; u < BU; ++u) {
        if (ix[u] < 0) continue;
        a.z[ix[u]] = zv[u];
        rz_th += (double)rv[u] * (double)zv[u];
      }
    }
    rz_out += rz_th;
    __syncthreads();
  }
}

// ---- block-band preconditioner (small interface blocks, CTA 0 only)

// Sub-phase timestamp of the block-band apply (init call only, verbose trace).
__device__ __forceinline__ void bb_mark(unsigned long long *trace, int cap, bool on, int k) {
  if (on && trace && threadIdx.x == 0 && cap >= 2 + 2 * 128 + 8) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    trace[2 + 2 * 128 + k] = t;
  }
}

// Products of one warp with the Q x Q matrices of the odd-even reduction (row-major,
// global memory, written by the preconditioner build) and vectors in shared memory:
// lane t owns output entries t and t + 32.
template <int Q> struct BcrOut {
  float v[(Q + 31) / 32];
};

// o_t += sum_c A[t][c] x[c]
template <int Q> __device__ __forceinline__ void bcr_mv(const float *__restrict__ A, const float *x, BcrOut<Q> &o) {
  const int lane = threadIdx.x & 31;
  const float4 *x4 = reinterpret_cast<const float4 *>(x);
#pragma unroll
  for (int u = 0; u < (Q + 31) / 32; ++u) {
    const int t = lane + 32 * u;
    if (t >= Q) continue;
    const float4 *a4 = reinterpret_cast<const float4 *>(A + t * Q);
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int c4 = 0; c4 < Q / 4; ++c4) {
      const float4 av = __ldg(a4 + c4), w = x4[c4];
      s0 += av.x * w.x + av.z * w.z;
      s1 += av.y * w.y + av.w * w.w;
    }
    o.v[u] += s0 + s1;
  }
}

// o_t += sum_c A[c][t] x[c]
template <int Q> __device__ __forceinline__ void bcr_mvt(const float *__restrict__ A, const float *x, BcrOut<Q> &o) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < (Q + 31) / 32; ++u) {
    const int t = lane + 32 * u;
    if (t >= Q) continue;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
    for (int c = 0; c < Q; c += 2) {
      s0 += __ldg(A + c * Q + t) * x[c];
      s1 += __ldg(A + (c + 1) * Q + t) * x[c + 1];
    }
    o.v[u] += s0 + s1;
  }
}

template <int Q> __device__ __forceinline__ void bcr_store(float *dst, const BcrOut<Q> &o) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < (Q + 31) / 32; ++u)
    if (lane + 32 * u < Q) dst[lane + 32 * u] = o.v[u];
}

// E phase with the block-band preconditioner, run by CTA 0 alone (the other
// CTAs contribute zero partials): x += alpha p, r -= alpha q (or x = 0, r = b),
// then z = B^{-1} r by the forward and backward passes of the odd-even reduction
// (levels of independent super-rows, one warp per super-row, a CTA barrier per
// phase); <r, r>, <r, z>.  When <r, r> already meets the tolerance the solve is
// skipped: the iteration stops after the barrier and never reads z (the exact
// block-band preconditioner of an edge core often converges in one iteration,
// whose second application would otherwise be half the launch).
// Shared layout: rs[S][Q] (b, then z), ys[S][Q] (y), a Q-entry scratch per warp;
// super-row J entry a M + e is block row p J + a, entry e, so rs is the [n][M]
// vector padded with zeros to S p block rows.
// The element loops load a batch of kU entries per thread before computing, so
// a thread waits for one memory latency per batch rather than per entry.
constexpr int kU = 4;

template <typename T, int PB, int M>
__device__ void bb_apply(const PcgArgs<T> &a, const T *__restrict__ pcur, double alpha, bool init, double &rr_out,
                         double &rz_out) {
  constexpr int Q = PB * M;
  constexpr long long QQ = (long long)Q * Q;
  bb_mark(a.trace, a.trace_cap, init, 0);
  extern __shared__ float4 esm4[];
  const int n = a.n, rr = a.rr, m = a.rl * a.rr, S = a.bbS, tot = n * M, totp = S * Q, B = blockDim.x;
  float *rs = reinterpret_cast<float *>(esm4);
  float *ys = rs + totp;
  float *ws = ys + totp;
  auto index_of = [&](int e) { return ((long long)((e % M) / rr) * n + e / M) * rr + ((e % M) % rr); };
  double rr_th = 0.0;
  for (int e0 = threadIdx.x; e0 < tot; e0 += kU * B) {
    T bx[kU], bq[kU], bp[kU], br[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * B;
      bx[u] = bq[u] = bp[u] = br[u] = T(0);
      if (e < tot && (e % M) < m) {
        const long long idx = index_of(e);
        if (init) {
          br[u] = a.b[idx];
        } else {
          bx[u] = a.x[idx];
          bp[u] = pcur[idx];
          br[u] = a.r[idx];
          bq[u] = a.q[idx];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * B;
      if (e >= tot) continue;
      float rv = 0.f;
      if ((e % M) < m) {
        const long long idx = index_of(e);
        T r;
        if (init) {
          r = br[u];
          a.x[idx] = T(0);
        } else {
          a.x[idx] = bx[u] + (T)alpha * bp[u];
          r = br[u] - (T)alpha * bq[u];
        }
        a.r[idx] = r;
        rr_th += (double)r * (double)r;
        rv = (float)r;
      }
      rs[e] = rv;
    }
  }
  for (int e = tot + threadIdx.x; e < totp; e += B) rs[e] = 0.f;
  rr_out += rr_th;
  // <r, r> over the CTA, formed exactly as the caller's partial (CTA 0 owns every entry and the
  // other partials are zero, so this is the value of the stop test)
  {
    __shared__ double red[32];
    __shared__ int done;
    double v = rr_out;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      done = !(t > a.tol2);
    }
    __syncthreads();
    if (done) {
      bb_mark(a.trace, a.trace_cap, init, 6);
      return;
    }
  }
  bb_mark(a.trace, a.trace_cap, init, 1);
  const int warp = threadIdx.x >> 5, nw = B >> 5;
  const float *Li = a.bbLinv, *Ul = a.bbUl, *Ur = a.bbUr;
  // forward: y_j = Linv_j b_j for the rows eliminated at level h, then the rows left take
  // b_J -= Ur_{J-h}^T y_{J-h} + Ul_{J+h}^T y_{J+h}
  int hmax = 0;
  for (int h = 1; h < S; h <<= 1) {
    hmax = h;
    const int ne = (S - h + 2 * h - 1) / (2 * h), na = (S + 2 * h - 1) / (2 * h);
    for (int t = warp; t < ne; t += nw) {
      const int j = h + 2 * h * t;
      BcrOut<Q> o = {};
      bcr_mv<Q>(Li + j * QQ, rs + j * Q, o);
      bcr_store<Q>(ys + j * Q, o);
    }
    __syncthreads();
    for (int t = warp; t < na; t += nw) {
      const int J = 2 * h * t;
      BcrOut<Q> o = {};
      if (J >= h) bcr_mvt<Q>(Ur + (J - h) * QQ, ys + (J - h) * Q, o);
      if (J + h < S) bcr_mvt<Q>(Ul + (J + h) * QQ, ys + (J + h) * Q, o);
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int u = 0; u < (Q + 31) / 32; ++u)
        if (lane + 32 * u < Q) rs[J * Q + lane + 32 * u] -= o.v[u];
    }
    __syncthreads();
  }
  bb_mark(a.trace, a.trace_cap, init, 2);
  // top row: y_0 = Linv_0 b_0, z_0 = Linv_0^T y_0
  if (warp == 0) {
    BcrOut<Q> o = {};
    bcr_mv<Q>(Li, rs, o);
    bcr_store<Q>(ys, o);
    __syncwarp();
    BcrOut<Q> z = {};
    bcr_mvt<Q>(Li, ys, z);
    bcr_store<Q>(rs, z);
  }
  __syncthreads();
  bb_mark(a.trace, a.trace_cap, init, 3);
  // backward: z_j = Linv_j^T (y_j - Ul_j z_{j-h} - Ur_j z_{j+h}), levels top down
  for (int h = hmax; h >= 1; h >>= 1) {
    const int ne = (S - h + 2 * h - 1) / (2 * h);
    float *w = ws + warp * Q;
    for (int t = warp; t < ne; t += nw) {
      const int j = h + 2 * h * t;
      BcrOut<Q> o = {};
      bcr_mv<Q>(Ul + j * QQ, rs + (j - h) * Q, o);
      if (j + h < S) bcr_mv<Q>(Ur + j * QQ, rs + (j + h) * Q, o);
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int u = 0; u < (Q + 31) / 32; ++u)
        if (lane + 32 * u < Q) w[lane + 32 * u] = ys[j * Q + lane + 32 * u] - o.v[u];
      __syncwarp();
      BcrOut<Q> z = {};
      bcr_mvt<Q>(Li + j * QQ, w, z);
      bcr_store<Q>(rs + j * Q, z);
      __syncwarp();
    }
    __syncthreads();
  }
  bb_mark(a.trace, a.trace_cap, init, 4);
  bb_mark(a.trace, a.trace_cap, init, 5);
  double rz_th = 0.0;
  for (int e0 = threadIdx.x; e0 < tot; e0 += kU * B) {
    T br[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * B;
      br[u] = T(0);
      if (e < tot && (e % M) < m) br[u] = a.r[index_of(e)];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * B;
      if (e < tot && (e % M) < m) {
        const T zi = (T)rs[e];
        a.z[index_of(e)] = zi;
        rz_th += (double)br[u] * (double)zi;
      }
    }
  }
  rz_out += rz_th;
  __syncthreads();
  bb_mark(a.trace, a.trace_cap, init, 6);
}

// Block-band E phase for the block size of this system (CTA 0 only).
template <typename T, int PB>
__device__ __forceinline__ void bb_phase(const PcgArgs<T> &a, const T *pcur, double alpha, bool init, double &rr_out,
                                         double &rz_out) {
  if (blockIdx.x != 0) return;
  if (a.bbM == 4) bb_apply<T, PB, 4>(a, pcur, alpha, init, rr_out, rz_out);
  else bb_apply<T, PB, 8>(a, pcur, alpha, init, rr_out, rz_out);
}

template <typename T, int PB>
__global__ void __launch_bounds__(256, 1) k_pcg_fused(PcgArgs<T> a) {
  const int rl = a.rl, rr = a.rr, Rl = a.Rl, Rr = a.Rr, n = a.n, b = 2 * PB + 1;
  const unsigned int G = gridDim.x;
  double *p_pq = a.part, *p_rr = a.part + G, *p_rz = a.part + 2 * G;

  int slot = 0;
  trace_mark(a.trace, a.trace_cap, slot);
  // The interfaces do not change during the solve: with room for them they are copied
  // into shared memory once (PhiR rows padded to an odd stride against bank conflicts).
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int phr_ld = a.iface_off >= 0 ? a.phr_ld : rr;  // row stride of PhiR where it is read from
  const T *PhiRs = a.PhiR, *PhiLs = a.PhiL;
  if (a.iface_off >= 0) {
    T *pr_s = reinterpret_cast<T *>(dsm_raw + a.iface_off);
    T *pl_s = pr_s + (long long)rr * Rr * phr_ld;
    for (int e = threadIdx.x; e < rr * Rr * rr; e += blockDim.x) pr_s[(e / rr) * phr_ld + e % rr] = a.PhiR[e];
    for (int e = threadIdx.x; e < rl * Rl * rl; e += blockDim.x) pl_s[e] = a.PhiL[e];
    PhiRs = pr_s;
    PhiLs = pl_s;
    __syncthreads();
  }
  // Tensor-core stages (MIXED_TF32, FP32 PCG only): TMEM for the accumulators, one
  // completion barrier, and the two interface operands split into TF32 high and low
  // parts in the canonical K-major layout, built once per solve.
  constexpr bool kTc = std::is_same<T, float>::value;
  __shared__ uint32_t tc_tmem;
  __shared__ __align__(8) uint64_t tc_bar;
  uint32_t tc_phase = 0;
  const int szPR = tc::operand_bytes(a.tcNA, a.tcKA), szPL = tc::operand_bytes(a.tcNC, a.tcKC),
            szPS = tc::operand_bytes(a.tcMA, a.tcKA);
  unsigned char *opPRh = dsm_raw + (a.tc ? a.tc_off : 0);
  unsigned char *opPRl = opPRh + szPR, *opPLh = opPRl + szPR, *opPLl = opPLh + szPL;
  unsigned char *opPSh = opPLl + szPL, *opPSl = opPSh + szPS;
  unsigned char *opT2h = opPSl + szPS, *opT2l = opT2h + tc::operand_bytes(a.tcMC, a.tcKC);
  if constexpr (kTc) {
    if (a.tc) {
      if (threadIdx.x < 32) tc::tmem_alloc(&tc_tmem, (uint32_t)a.tc_cols);
      if (threadIdx.x == 0) tc::mbar_init1(&tc_bar);
      for (int e = threadIdx.x; e < a.tcNA * a.tcKA; e += blockDim.x) {
        const int r = e / a.tcKA, k = e % a.tcKA;  // row c Rr + d, column f
        const float x = (r < rr * Rr && k < rr) ? (float)a.PhiR[(long long)r * rr + k] : 0.f;
        const float h = tc::to_tf32(x);
        *reinterpret_cast<float *>(opPRh + tc::operand_offset(r, k, a.tcKA)) = h;
        *reinterpret_cast<float *>(opPRl + tc::operand_offset(r, k, a.tcKA)) = tc::to_tf32(x - h);
      }
      for (int e = threadIdx.x; e < a.tcNC * a.tcKC; e += blockDim.x) {
        const int r = e / a.tcKC, k = e % a.tcKC;  // row al, column g rl + aa
        const float x = (r < rl && k < Rl * rl) ? (float)a.PhiL[(long long)r * Rl * rl + k] : 0.f;
        const float h = tc::to_tf32(x);
        *reinterpret_cast<float *>(opPLh + tc::operand_offset(r, k, a.tcKC)) = h;
        *reinterpret_cast<float *>(opPLl + tc::operand_offset(r, k, a.tcKC)) = tc::to_tf32(x - h);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
  }
  bool aborted = false;
  // r = b, x = 0, z = P^{-1} r;  <r, r>, <r, z>
  double rr_loc = 0.0, rz_loc = 0.0;
  if (a.edge) bb_phase<T, PB>(a, nullptr, 0.0, true, rr_loc, rz_loc);
  else band_systems<T, PB>(a, nullptr, 0.0, true, rr_loc, rz_loc);
  cta_partial(rr_loc, p_rr);
  cta_partial(rz_loc, p_rz);
  if (!grid_sync(a.bar, G, a.err)) aborted = true;
  trace_mark(a.trace, a.trace_cap, slot);
  double res2 = aborted ? 0.0 : grid_total(p_rr);
  double rz = aborted ? 0.0 : grid_total(p_rz), rz_prev = 1.0;
  int it = 0;
  for (; !aborted && it < a.maxit && res2 > a.tol2; ++it) {
    const double beta = (it == 0 || rz_prev == 0.0) ? 0.0 : rz / rz_prev;
    T *pcur = (it & 1) ? a.pv2 : a.pv;
    const T *pprev = (it & 1) ? a.pv : a.pv2;
    // A+B+C on slabs of S mode rows, one slab per CTA at a time, so only CTA barriers
    // are needed: p on the slab plus its +-p halo rows (recomputed from z and p_prev),
    // T1 on those rows, T2 and q on the slab rows, <p, q> partial.  p rows of the slab
    // are written once.  The slab scratch lives in shared memory when it fits.
    double pq_loc = 0.0;
    {
      const int S = a.slab, nslab = (n + S - 1) / S;
      T *Ps = a.dense_off >= 0 ? reinterpret_cast<T *>(dsm_raw + a.dense_off)
                               : a.scratch + (long long)blockIdx.x * a.dense_stride;
      T *T1s = Ps + a.p_stride;
      T *T2s = T1s + a.t1_stride;
      for (int sl = blockIdx.x; sl < nslab; sl += G) {
        const int i0 = sl * S, i1 = min(n, i0 + S);
        const int j0 = max(0, i0 - PB), j1 = min(n, i1 + PB);
        const int nj = j1 - j0, ni = i1 - i0;
        // A0: Ps[aa][jj][f] = z + beta p_prev on the slab and halo rows (contiguous in f, jj)
        const int nP = rl * nj * rr;
        bool use_tc = false;
        if constexpr (kTc) use_tc = a.tc != 0;
        if (!use_tc) {
          for (int e = threadIdx.x; e < nP; e += blockDim.x) {
            const int f = e % rr;
            const int t = e / rr;
            const int jj = t % nj, aa = t / nj;
            const int j = j0 + jj;
            const long long idx = ((long long)aa * n + j) * rr + f;
            const T pf = (it == 0) ? a.z[idx] : a.z[idx] + (T)beta * pprev[idx];
            Ps[e] = pf;
            if (j >= i0 && j < i1) pcur[idx] = pf;
          }
          __syncthreads();
        }
        if constexpr (kTc) {
          if (use_tc) {
            // A0 with the tensor-core operand: every padded position of the Ps operand
            // (rows aa nj + jj, columns f) gets its TF32 high and low parts or zero; the
            // positions of the T2 operand that stage B does not write are zeroed.  Then
            // T1 = Ps PhiR^T by tcgen05 (3xTF32), read back from TMEM into T1s.
            for (int e = threadIdx.x; e < a.tcMA * a.tcKA; e += blockDim.x) {
              const int t = e / a.tcKA, f = e % a.tcKA;
              float pf = 0.f;
              if (t < rl * nj && f < rr) {
                const int jj = t % nj, aa = t / nj;
                const int j = j0 + jj;
                const long long idx = ((long long)aa * n + j) * rr + f;
                pf = (it == 0) ? (float)a.z[idx] : (float)(a.z[idx] + (T)beta * pprev[idx]);
                Ps[t * rr + f] = (T)pf;
                if (j >= i0 && j < i1) pcur[idx] = (T)pf;
              }
              const float h = tc::to_tf32(pf);
              *reinterpret_cast<float *>(opPSh + tc::operand_offset(t, f, a.tcKA)) = h;
              *reinterpret_cast<float *>(opPSl + tc::operand_offset(t, f, a.tcKA)) = tc::to_tf32(pf - h);
            }
            for (int e = threadIdx.x; e < a.tcMC * a.tcKC; e += blockDim.x) {
              const int m = e / a.tcKC, q = e % a.tcKC;
              if (m >= ni * rr || q >= Rl * rl) {
                *reinterpret_cast<float *>(opT2h + tc::operand_offset(m, q, a.tcKC)) = 0.f;
                *reinterpret_cast<float *>(opT2l + tc::operand_offset(m, q, a.tcKC)) = 0.f;
              }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const int nMT = a.tcMA / 128;
            if (threadIdx.x == 0) {
              const uint32_t id = tc::idesc_tf32(128, a.tcNA);
              const uint32_t sboA = tc::sbo_bytes(a.tcKA);
              for (int mt = 0; mt < nMT; ++mt)
                for (int st = 0; st < a.tcKA / 8; ++st) {
                  const uint32_t ao = (uint32_t)mt * 16 * sboA + 256u * st, bo = 256u * st;
                  const uint64_t ah = tc::smem_desc(tc::smem_u32addr(opPSh) + ao, tc::kLBO, sboA);
                  const uint64_t al = tc::smem_desc(tc::smem_u32addr(opPSl) + ao, tc::kLBO, sboA);
                  const uint64_t bh = tc::smem_desc(tc::smem_u32addr(opPRh) + bo, tc::kLBO, sboA);
                  const uint64_t bl = tc::smem_desc(tc::smem_u32addr(opPRl) + bo, tc::kLBO, sboA);
                  const uint32_t d = tc_tmem + (uint32_t)(mt * a.tcNA);
                  tc::mma_tf32(d, ah, bh, id, st > 0);
                  tc::mma_tf32(d, ah, bl, id, true);
                  tc::mma_tf32(d, al, bh, id, true);
                }
              tc::mma_commit(&tc_bar);
            }
            if (!tc::mbar_wait_parity(&tc_bar, tc_phase, kSpinLimit) && (threadIdx.x & 31) == 0) atomicExch(a.err, 3);
            tc_phase ^= 1u;
            tc::fence_after_sync();
            {
              const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wq = warp & 3;
              const int ncd = rr * Rr;
              for (int mt = warp >> 2; mt < nMT; mt += (int)(blockDim.x >> 7)) {
                const int r = mt * 128 + 32 * wq + lane;
                for (int c0 = 0; c0 < a.tcNA; c0 += 16) {
                  float v[16];
                  tc::tmem_ld16(tc_tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(mt * a.tcNA + c0), v);
                  if (r < rl * nj) {
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                      if (c0 + k < ncd) T1s[(long long)r * ncd + c0 + k] = v[k];
                  }
                }
              }
            }
            tc::fence_before_sync();
            __syncthreads();
          }
        }
        // The three stages are register-tiled: each thread computes TW = 4 neighbouring
        // outputs, so one load of the shared operand feeds TW independent FMA chains.
        // Indices past the last output are clamped for the loads and not stored.
        constexpr int TW = 4;
        // A1: T1s[aa][jj][c][d] = sum_f Ps[aa][jj][f] PhiR[c][d][f], TW consecutive d
        const int nd4 = (Rr + TW - 1) / TW;
        const int nA1 = use_tc ? 0 : rl * nj * rr * nd4;
        for (int e = threadIdx.x; e < nA1; e += blockDim.x) {
          const int d0 = (e % nd4) * TW;
          const int t2 = e / nd4;
          const int c = t2 % rr, t = t2 / rr;
          const T *pr = Ps + (long long)t * rr;
          const T *ph[TW];
#pragma unroll
          for (int k = 0; k < TW; ++k) ph[k] = PhiRs + (long long)(c * Rr + min(d0 + k, Rr - 1)) * phr_ld;
          T sa[TW];
#pragma unroll
          for (int k = 0; k < TW; ++k) sa[k] = T(0);
          for (int f = 0; f < rr; ++f) {
            const T pv = pr[f];
#pragma unroll
            for (int k = 0; k < TW; ++k) sa[k] += pv * ph[k][f];
          }
          T *dst = T1s + ((long long)t * rr + c) * Rr + d0;
#pragma unroll
          for (int k = 0; k < TW; ++k)
            if (d0 + k < Rr) dst[k] = sa[k];
        }
        __syncthreads();
        // B: T2s[g][aa][ii][c] = sum_{o, d} A[g][i][o][d] T1s[aa][i+o-p-j0][c][d], TW consecutive c
        const int nc4 = (rr + TW - 1) / TW;
        const int nB1 = Rl * rl * ni * nc4;
        for (int e = threadIdx.x; e < nB1; e += blockDim.x) {
          const int c0 = (e % nc4) * TW;
          int t = e / nc4;
          const int ii = t % ni;
          t /= ni;
          const int aa = t % rl, g = t / rl;
          const int i = i0 + ii;
          const T *Ar = a.A + ((long long)g * n + i) * b * Rr;
          int cofs[TW];
#pragma unroll
          for (int k = 0; k < TW; ++k) cofs[k] = min(c0 + k, rr - 1) * Rr;
          T sb[TW];
#pragma unroll
          for (int k = 0; k < TW; ++k) sb[k] = T(0);
#pragma unroll
          for (int o = 0; o < b; ++o) {
            const int j = i + o - PB;
            if (j < 0 || j >= n) continue;
            const T *Ao = Ar + o * Rr;
            const T *Tj = T1s + ((long long)aa * nj + (j - j0)) * rr * Rr;
            for (int d = 0; d < Rr; ++d) {
              const T av = Ao[d];
#pragma unroll
              for (int k = 0; k < TW; ++k) sb[k] += av * Tj[cofs[k] + d];
            }
          }
          if constexpr (kTc) {
            if (use_tc) {
              // the T2 operand of stage C: row ii rr + c, column g rl + aa, TF32 high and low parts
#pragma unroll
              for (int k = 0; k < TW; ++k) {
                if (c0 + k >= rr) continue;
                const int m = ii * rr + c0 + k, q = g * rl + aa;
                const float x = (float)sb[k], h = tc::to_tf32(x);
                *reinterpret_cast<float *>(opT2h + tc::operand_offset(m, q, a.tcKC)) = h;
                *reinterpret_cast<float *>(opT2l + tc::operand_offset(m, q, a.tcKC)) = tc::to_tf32(x - h);
              }
              continue;
            }
          }
          T *dst = T2s + (((long long)g * rl + aa) * ni + ii) * rr + c0;
#pragma unroll
          for (int k = 0; k < TW; ++k)
            if (c0 + k < rr) dst[k] = sb[k];
        }
        if constexpr (kTc) {
          if (use_tc) tc::fence_proxy_async();
        }
        __syncthreads();
        // C: q[al][i][c] = sum_{g, aa} PhiL[al][g][aa] T2s[g][aa][ii][c], TW consecutive c;  <p, q>
        if constexpr (kTc) {
          if (use_tc) {
            // C on the tensor cores: q^T[(ii, c)][al] = sum_q T2[(ii, c)][q] PhiL[al][q] (3xTF32)
            tc::fence_after_sync();
            const int nMT = a.tcMA / 128, nMC = a.tcMC / 128;
            const uint32_t col0 = (uint32_t)(nMT * a.tcNA);
            if (threadIdx.x == 0) {
              const uint32_t id = tc::idesc_tf32(128, a.tcNC);
              const uint32_t sboC = tc::sbo_bytes(a.tcKC);
              for (int mc = 0; mc < nMC; ++mc)
                for (int st = 0; st < a.tcKC / 8; ++st) {
                  const uint32_t ao = (uint32_t)mc * 16 * sboC + 256u * st, bo = 256u * st;
                  const uint64_t ah = tc::smem_desc(tc::smem_u32addr(opT2h) + ao, tc::kLBO, sboC);
                  const uint64_t al = tc::smem_desc(tc::smem_u32addr(opT2l) + ao, tc::kLBO, sboC);
                  const uint64_t bh = tc::smem_desc(tc::smem_u32addr(opPLh) + bo, tc::kLBO, sboC);
                  const uint64_t bl = tc::smem_desc(tc::smem_u32addr(opPLl) + bo, tc::kLBO, sboC);
                  const uint32_t d = tc_tmem + col0 + (uint32_t)(mc * a.tcNC);
                  tc::mma_tf32(d, ah, bh, id, st > 0);
                  tc::mma_tf32(d, ah, bl, id, true);
                  tc::mma_tf32(d, al, bh, id, true);
                }
              tc::mma_commit(&tc_bar);
            }
            if (!tc::mbar_wait_parity(&tc_bar, tc_phase, kSpinLimit) && (threadIdx.x & 31) == 0) atomicExch(a.err, 3);
            tc_phase ^= 1u;
            tc::fence_after_sync();
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wq = warp & 3;
            for (int mc = warp >> 2; mc < nMC; mc += (int)(blockDim.x >> 7)) {
              const int m = mc * 128 + 32 * wq + lane;
              for (int c0 = 0; c0 < a.tcNC; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tc_tmem + ((uint32_t)(32 * wq) << 16) + col0 + (uint32_t)(mc * a.tcNC + c0), v);
                if (m < ni * rr) {
                  const int ii = m / rr, c = m % rr;
#pragma unroll
                  for (int k = 0; k < 16; ++k) {
                    const int al = c0 + k;
                    if (al >= rl) continue;
                    const long long idx = ((long long)al * n + i0 + ii) * rr + c;
                    a.q[idx] = (T)v[k];
                    pq_loc += (double)Ps[((long long)al * nj + (i0 + ii - j0)) * rr + c] * (double)v[k];
                  }
                }
              }
            }
            tc::fence_before_sync();
            __syncthreads();
            continue;
          }
        }
        const int nC1 = rl * ni * nc4;
        const int ga = Rl * rl;
        for (int e = threadIdx.x; e < nC1; e += blockDim.x) {
          const int c0 = (e % nc4) * TW;
          const int t = e / nc4;
          const int ii = t % ni, al = t / ni;
          const T *ph = PhiLs + (long long)al * ga;
          int cidx[TW];
#pragma unroll
          for (int k = 0; k < TW; ++k) cidx[k] = min(c0 + k, rr - 1);
          T sc[TW];
#pragma unroll
          for (int k = 0; k < TW; ++k) sc[k] = T(0);
          for (int q = 0; q < ga; ++q) {
            const T pv = ph[q];
            const T *row = T2s + ((long long)q * ni + ii) * rr;
#pragma unroll
            for (int k = 0; k < TW; ++k) sc[k] += pv * row[cidx[k]];
          }
#pragma unroll
          for (int k = 0; k < TW; ++k) {
            if (c0 + k >= rr) continue;
            const int c = c0 + k;
            const long long idx = ((long long)al * n + i0 + ii) * rr + c;
            a.q[idx] = sc[k];
            pq_loc += (double)Ps[((long long)al * nj + (i0 + ii - j0)) * rr + c] * (double)sc[k];
          }
        }
        __syncthreads();
      }
    }
    cta_partial(pq_loc, p_pq);
    if (!grid_sync(a.bar, G, a.err)) {
      aborted = true;
      break;
    }
    trace_mark(a.trace, a.trace_cap, slot);
    // E: x += alpha p, r -= alpha q, z = P^{-1} r per band system;  <r, r>, <r, z>
    const double pq = grid_total(p_pq);
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    rr_loc = 0.0;
    rz_loc = 0.0;
    if (a.edge) bb_phase<T, PB>(a, pcur, alpha, false, rr_loc, rz_loc);
    else band_systems<T, PB>(a, pcur, alpha, false, rr_loc, rz_loc);
    cta_partial(rr_loc, p_rr);
    cta_partial(rz_loc, p_rz);
    if (!grid_sync(a.bar, G, a.err)) {
      aborted = true;
      break;
    }
    trace_mark(a.trace, a.trace_cap, slot);
    res2 = grid_total(p_rr);
    rz_prev = rz;
    rz = grid_total(p_rz);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!aborted) {
      a.out[0] = (double)it;
      a.out[1] = res2;
    }
  }
  if constexpr (kTc) {
    if (a.tc) {
      tc::fence_before_sync();
      __syncthreads();
      if (threadIdx.x < 32) tc::tmem_dealloc(tc_tmem, (uint32_t)a.tc_cols);
      if (threadIdx.x == 0) tc::mbar_inval1(&tc_bar);
    }
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

// One application of the block-band preconditioner outside PCG (a test entry point):
// z = B^{-1} b with the stored factors, by the E phase of the first iteration (x = 0,
// r = b; tol2 < 0, so the substitutions always run).  One CTA.
template <typename T, int PB, int M> __global__ void __launch_bounds__(256) k_bb_apply_once(PcgArgs<T> a) {
  double rr = 0.0, rz = 0.0;
  bb_apply<T, PB, M>(a, nullptr, 0.0, true, rr, rz);
}

template <typename T, int PB> const void *bb_once_ptr(int M) {
  return M == 4 ? (const void *)k_bb_apply_once<T, PB, 4> : (const void *)k_bb_apply_once<T, PB, 8>;
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
  // block-band preconditioner: rs, ys [S][q] and a q-entry scratch per warp (8 warps)
  const size_t bb_vec = a.edge ? (2 * (size_t)a.bbS + 8) * a.p * a.bbM * sizeof(float) : 0;
  if (a.edge) {
    TTI_CHECK_ARG(bb_vec <= kPcgSmemBytes, "pcg: n=%d too large for the block-band preconditioner", a.n);
    a.slots = 1;
    a.smem = (int)bb_vec;
  } else {
    a.slots = band_slots(a);
    a.smem = (int)((size_t)a.slots * a.n * (a.p + 2) * sizeof(float));
    TTI_CHECK_ARG((size_t)a.n * (a.p + 2) * sizeof(float) <= kPcgSmemBytes,
                  "pcg: n=%d too large for one band system", a.n);
  }
  TTI_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPcgSmemBytes));
  int per_sm = 0;
  TTI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, a.smem));
  TTI_CHECK_ARG(per_sm >= 1, "pcg: kernel does not fit on an SM");
  const int sms = (c->coop_sms > 0) ? std::min(c->coop_sms, c->num_sms) : c->num_sms;
  const long long cap = (long long)sms * std::max(1, std::min(per_sm, 2));
  const long long row_out = (long long)a.Rl * a.rl * a.rr;
  long long S = std::max<long long>((256 + row_out - 1) / row_out, (a.n + cap - 1) / cap);
  S = std::max<long long>(1, std::min<long long>(S, a.n));
  a.slab = (int)S;
  const long long nslab = (a.n + S - 1) / S;
  const long long npair = a.edge ? 1 : (long long)a.rl * a.rr;
  long long g = std::max(nslab, (npair + a.slots - 1) / a.slots);
  g = std::max<long long>(1, std::min(g, cap));
  if (!a.edge) {
    // spread the band systems over the grid the dense phase needs anyway: fewer per
    // CTA shortens the gathers and scatters; with one slot each, the factors stay
    // resident in shared memory for the whole solve
    a.slots = (int)std::min<long long>(a.slots, (npair + g - 1) / g);
    a.resident = (long long)a.slots * g >= npair ? 1 : 0;
    a.smem = (int)((size_t)a.slots * a.n * (a.p + 2) * sizeof(float));
  } else {
    a.resident = 0;
  }
  a.p_stride = (long long)a.rl * (S + 2 * a.p) * a.rr;
  a.t1_stride = (long long)a.rl * (S + 2 * a.p) * a.rr * a.Rr;
  a.t2_stride = (long long)a.Rl * a.rl * S * a.rr;
  a.dense_stride = a.p_stride + a.t1_stride + a.t2_stride;
  a.phr_ld = a.rr | 1;
  // Shared memory after the preconditioner's area: the slab scratch of the dense phase
  // (p, T1, T2), then the interfaces, each when it fits; otherwise the slab scratch is in global memory
  // (one region per CTA) and the interfaces are read from global memory.  The grid
  // must stay co-resident.
  const size_t dense = (size_t)a.dense_stride * sizeof(T);
  const size_t iface = ((size_t)a.rr * a.Rr * a.phr_ld + (size_t)a.rl * a.Rl * a.rl) * sizeof(T);
  const size_t pre_smem = (size_t)a.smem;
  auto place = [&](bool want_iface, size_t reserve) {  // reserve: bytes kept free after the slab scratch
    a.dense_off = -1;
    a.iface_off = -1;
    const size_t extra = dense + (want_iface ? iface : 0) + reserve;
    {
      const size_t off = (pre_smem + 15) / 16 * 16;
      if (off + extra + 16 > kPcgSmemBytes) return;
      a.dense_off = (int)off;
      a.smem = (int)(off + dense);
    }
    if (want_iface) {
      const size_t off = ((size_t)a.smem + 15) / 16 * 16;
      a.iface_off = (int)off;
      a.smem = (int)(off + iface);
    }
  };
  // Tensor-core stages: padded shapes, TMEM columns and the operand area after the
  // slab scratch (the shared interface copies are not needed then).  Cleared when the
  // operands do not fit, when TMEM would need more than 256 columns per CTA, or when the
  // slab scratch itself is not in shared memory.
  size_t tc_bytes = 0;
  if (a.tc) {
    auto up = [](long long v, long long m) { return (int)((v + m - 1) / m * m); };
    a.tcMA = up((long long)a.rl * (S + 2 * a.p), 128);
    a.tcNA = up((long long)a.rr * a.Rr, 16);
    a.tcKA = up(a.rr, 8);
    a.tcMC = up((long long)S * a.rr, 128);
    a.tcNC = up(a.rl, 16);
    a.tcKC = up((long long)a.Rl * a.rl, 8);
    const long long cols = (long long)(a.tcMA / 128) * a.tcNA + (long long)(a.tcMC / 128) * a.tcNC;
    int tcols = 32;
    while (tcols < cols) tcols *= 2;
    a.tc_cols = tcols;
    tc_bytes = 2 * (size_t)(tc::operand_bytes(a.tcNA, a.tcKA) + tc::operand_bytes(a.tcNC, a.tcKC) +
                            tc::operand_bytes(a.tcMA, a.tcKA) + tc::operand_bytes(a.tcMC, a.tcKC));
    if (a.tcNA > 256 || a.tcNC > 256 || cols > 256) a.tc = 0;
  }
  if (a.tc) {
    place(false, tc_bytes + 128);
    if (a.dense_off >= 0) {
      const size_t off = ((size_t)a.smem + 127) / 128 * 128;
      if (off + tc_bytes <= kPcgSmemBytes) {
        a.tc_off = (int)off;
        a.smem = (int)(off + tc_bytes);
      } else {
        a.tc = 0;
      }
    } else {
      a.tc = 0;
    }
  }
  if (!a.tc) {
    place(true, 0);
    if (a.dense_off < 0) place(false, 0);
  }
  if (a.dense_off >= 0) {
    int per_sm2 = 0;
    TTI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k, 256, a.smem));
    if ((long long)per_sm2 * c->num_sms < g) {
      a.dense_off = -1;
      a.tc = 0;
    }
  }
  if (a.dense_off < 0) {
    // the sizes chosen above, slab scratch in global memory, interfaces from global memory
    a.iface_off = -1;
    a.smem = (int)pre_smem;
  }
  return (int)g;
}

template <typename T>
void bb_solve_once(Ctx *c, const BBPrec &P, int rl, int rr, int n, int p, const T *b, T *z) {
  const long long N = (long long)rl * n * rr;
  DBuf xr(c, 2 * N * sizeof(T));
  PcgArgs<T> a{};
  a.b = b;
  a.x = xr.as<T>();
  a.r = a.x + N;
  a.z = z;
  a.rl = rl;
  a.rr = rr;
  a.n = n;
  a.p = p;
  a.tol2 = -1.0;
  a.edge = 1;
  a.bbLinv = P.Linv.as<float>();
  a.bbUl = P.Ul.as<float>();
  a.bbUr = P.Ur.as<float>();
  a.bbM = P.M;
  a.bbS = P.S;
  const void *k = nullptr;
  switch (p) {
    case 1: k = bb_once_ptr<T, 1>(P.M); break;
    case 2: k = bb_once_ptr<T, 2>(P.M); break;
    case 3: k = bb_once_ptr<T, 3>(P.M); break;
    case 4: k = bb_once_ptr<T, 4>(P.M); break;
    case 5: k = bb_once_ptr<T, 5>(P.M); break;
    case 6: k = bb_once_ptr<T, 6>(P.M); break;
    case 7: k = bb_once_ptr<T, 7>(P.M); break;
    default: fail(TT_IGA_ERR_ARG, "block-band solve: degree %d outside 1..7", p);
  }
  const size_t smem = (2 * (size_t)P.S + 8) * P.q * sizeof(float);
  TTI_CHECK_ARG(smem <= kPcgSmemBytes, "block-band solve: n=%d too large", n);
  TTI_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPcgSmemBytes));
  void *args[] = {&a};
  TTI_CUDA(cudaLaunchKernel(k, dim3(1), dim3(256), args, smem, c->stream));
  g_launches.fetch_add(1, std::memory_order_relaxed);
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

}  // namespace ttiga
