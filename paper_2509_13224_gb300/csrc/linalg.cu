// Dense linear algebra kernels (FP64 unless templated): GEMM, deterministic
// reductions, tall-skinny Householder QR (TSQR tree), one-sided Jacobi SVD and
// maximum-volume row selection.  All sizes on this path are small to moderate
// (ranks <= 256); GB300's FP64 pipe (about 1.2 TFLOP/s, measured) bounds
// these kernels, so they keep FP64 work at its algorithmic minimum.
#include <algorithm>
#include <cfloat>
#include <mutex>

#include "linalg.cuh"

namespace ttiga {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (deterministic order); result returned to every thread.
__device__ double block_sum(double v, double *red) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// ------------------------------------------------------------------- GEMM

// Tiled GEMM with a BM x BN block tile (256 threads, TM x TN outputs each) so
// narrow shapes do not spend FP64 FMAs on padding; the K loop stops at the
// real K.  With ksplit > 1, blockIdx.z selects a K chunk (batch must be 1) and
// C points to a [ksplit][m][ldc] workspace of partial products.
template <typename T, int BM, int BN>
__global__ void __launch_bounds__(256) k_gemm(bool ta, bool tb, int m, int n, int k, T alpha,
                                              const T *__restrict__ A, long long lda, long long sA,
                                              const T *__restrict__ B, long long ldb, long long sB,
                                              T beta, T *__restrict__ C, long long ldc, long long sC,
                                              int ksplit, int kchunk) {
  constexpr int BK = 16;
  // thread grid: (BM / TM) x (BN / TN) = 256
  constexpr int TN = (BN >= 64) ? 4 : ((BN == 32) ? 2 : 1);
  constexpr int TM = (BM * BN) / (256 * TN);
  constexpr int NTX = BN / TN;  // threads along N
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  int kbeg = 0, kend = k;
  if (ksplit > 1) {
    kbeg = blockIdx.z * kchunk;
    kend = min(k, kbeg + kchunk);
    C += (long long)blockIdx.z * m * ldc;
  } else {
    const long long b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
  }
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  T acc[TM][TN];
#pragma unroll
  for (int x = 0; x < TM; ++x)
#pragma unroll
    for (int y = 0; y < TN; ++y) acc[x][y] = T(0);
  for (int l0 = kbeg; l0 < kend; l0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int ii, ll;
      if (!ta) { ii = e / BK; ll = e % BK; } else { ll = e / BM; ii = e % BM; }
      const int gi = i0 + ii, gl = l0 + ll;
      T v = T(0);
      if (gi < m && gl < kend) v = ta ? A[(long long)gl * lda + gi] : A[(long long)gi * lda + gl];
      As[ll][ii] = v;
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      int ll, jj;
      if (!tb) { ll = e / BN; jj = e % BN; } else { jj = e / BK; ll = e % BK; }
      const int gl = l0 + ll, gj = j0 + jj;
      T v = T(0);
      if (gl < kend && gj < n) v = tb ? B[(long long)gj * ldb + gl] : B[(long long)gl * ldb + gj];
      Bs[ll][jj] = v;
    }
    __syncthreads();
    const int kk = min(BK, kend - l0);
#pragma unroll 4
    for (int ll = 0; ll < kk; ++ll) {
      T av[TM], bv[TN];
#pragma unroll
      for (int x = 0; x < TM; ++x) av[x] = As[ll][ty + (BM / TM) * x];
#pragma unroll
      for (int y = 0; y < TN; ++y) bv[y] = Bs[ll][tx + NTX * y];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    const int gi = i0 + ty + (BM / TM) * x;
    if (gi >= m) continue;
#pragma unroll
    for (int y = 0; y < TN; ++y) {
      const int gj = j0 + tx + NTX * y;
      if (gj >= n) continue;
      T *cp = C + (long long)gi * ldc + gj;
      if (ksplit > 1) *cp = acc[x][y];
      else *cp = (beta == T(0)) ? alpha * acc[x][y] : alpha * acc[x][y] + beta * (*cp);
    }
  }
}

// C = alpha sum_s W[s] + beta C over the split-K partials (fixed order: deterministic).
template <typename T>
__global__ void k_splitk_reduce(const T *__restrict__ W, int ksplit, int m, int n, T alpha, T beta, T *C,
                                long long ldc) {
  const long long tot = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    T acc = T(0);
    for (int s = 0; s < ksplit; ++s) acc += W[((long long)s * m + i) * n + j];
    T *cp = C + i * ldc + j;
    *cp = (beta == T(0)) ? alpha * acc : alpha * acc + beta * (*cp);
  }
}

// The same with one warp per output: lanes stride over the partials and combine them by a
// fixed shuffle tree (deterministic), for few outputs over many partials, where a thread per
// output would walk all ksplit partials serially.
template <typename T>
__global__ void __launch_bounds__(256) k_splitk_reduce_warp(const T *__restrict__ W, int ksplit, int m, int n,
                                                            T alpha, T beta, T *C, long long ldc) {
  const long long e = blockIdx.x * 8LL + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= (long long)m * n) return;  // the whole warp leaves together
  const long long i = e / n, j = e % n;
  T acc = T(0);
  for (int s = lane; s < ksplit; s += 32) acc += W[((long long)s * m + i) * n + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    T *cp = C + i * ldc + j;
    *cp = (beta == T(0)) ? alpha * acc : alpha * acc + beta * (*cp);
  }
}

template <typename T>
__global__ void k_scale_mat(T *C, int m, int n, long long ldc, long long sC, T beta) {
  const long long b = blockIdx.y;
  T *Cb = C + b * sC;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * n;
       e += (long long)gridDim.x * blockDim.x) {
    T *cp = Cb + (e / n) * ldc + (e % n);
    *cp = (beta == T(0)) ? T(0) : beta * (*cp);
  }
}

template <typename T>
void gemm(Ctx *c, bool ta, bool tb, int m, int n, int k, T alpha, const T *A, long long lda,
          long long sA, const T *B, long long ldb, long long sB, T beta, T *C, long long ldc,
          long long sC, int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return;
  if (k <= 0) {
    for (int b0 = 0; b0 < batch; b0 += 65535) {
      int nb = std::min(65535, batch - b0);
      k_scale_mat<T><<<dim3(grid1d((long long)m * n, 256, 1024), nb), 256, 0, c->stream>>>(
          C + b0 * sC, m, n, ldc, sC, beta);
      TTI_LAUNCH();
    }
    return;
  }
  // Tile shape by CTA count.  GB300 executes about 2 FP64 FMAs per clock per SM,
  // so a GEMM of this path is as fast as the number of SMs its FMAs are spread
  // over: the largest tile that still gives every SM about two CTAs, down to
  // 16 x 16 (one output per thread).  FP32 (mixed precision) uses the same rule.
  const long long batch_tiles = batch;
  auto ntiles = [&](int bm, int bn) { return (long long)cdiv(n, bn) * cdiv(m, bm) * batch_tiles; };
  const long long want = 2LL * c->num_sms;
  int shape;  // 0: 64x64, 1: 128x16, 2: 16x128, 3: 32x32, 4: 16x16
  if (ntiles(64, 64) >= want && m > 32 && n > 32) shape = 0;
  else if (ntiles(32, 32) >= want && m > 16 && n > 16) shape = 3;
  else if (n <= 16 && ntiles(128, 16) >= want) shape = 1;
  else if (m <= 16 && ntiles(16, 128) >= want) shape = 2;
  else shape = 4;
  const int BMs[5] = {64, 128, 16, 32, 16}, BNs[5] = {64, 16, 128, 32, 16};
  const int BM = BMs[shape], BN = BNs[shape];
  auto launch = [&](dim3 grid, const T *A_, const T *B_, T beta_, T *C_, long long ldc_, long long sA_, long long sB_,
                    long long sC_, int ksplit, int kchunk) {
    switch (shape) {
      case 0:
        k_gemm<T, 64, 64><<<grid, 256, 0, c->stream>>>(ta, tb, m, n, k, alpha, A_, lda, sA_, B_, ldb, sB_, beta_, C_,
                                                        ldc_, sC_, ksplit, kchunk);
        break;
      case 1:
        k_gemm<T, 128, 16><<<grid, 256, 0, c->stream>>>(ta, tb, m, n, k, alpha, A_, lda, sA_, B_, ldb, sB_, beta_, C_,
                                                         ldc_, sC_, ksplit, kchunk);
        break;
      case 2:
        k_gemm<T, 16, 128><<<grid, 256, 0, c->stream>>>(ta, tb, m, n, k, alpha, A_, lda, sA_, B_, ldb, sB_, beta_, C_,
                                                         ldc_, sC_, ksplit, kchunk);
        break;
      case 3:
        k_gemm<T, 32, 32><<<grid, 256, 0, c->stream>>>(ta, tb, m, n, k, alpha, A_, lda, sA_, B_, ldb, sB_, beta_, C_,
                                                        ldc_, sC_, ksplit, kchunk);
        break;
      default:
        k_gemm<T, 16, 16><<<grid, 256, 0, c->stream>>>(ta, tb, m, n, k, alpha, A_, lda, sA_, B_, ldb, sB_, beta_, C_,
                                                        ldc_, sC_, ksplit, kchunk);
        break;
    }
    TTI_LAUNCH();
  };
  const long long tiles = (long long)cdiv(n, BN) * cdiv(m, BM);
  if (batch == 1 && tiles * 2 < c->num_sms && k >= 64) {
    // few output tiles but a long K: split K over CTAs (chunks of at least 32), then reduce the partials
    int ksplit = (int)std::min<long long>(std::max<long long>(1, want / tiles), (k + 31) / 32);
    ksplit = std::max(2, std::min(ksplit, 256));
    const int kchunk = ((k + ksplit - 1) / ksplit + 15) / 16 * 16;
    ksplit = (k + kchunk - 1) / kchunk;
    DBuf W(c, (size_t)ksplit * m * n * sizeof(T));
    {
      ProfScope ps(c, sizeof(T) == 8 ? PROF_GEMM64 : PROF_OFF, 2.0 * m * (double)n * k);
      launch(dim3(cdiv(n, BN), cdiv(m, BM), ksplit), A, B, T(0), W.as<T>(), n, 0, 0, 0, ksplit, kchunk);
    }
    const long long outs = (long long)m * n;
    if (outs <= 64LL * c->num_sms)  // up to 8 CTAs of 8 warps per SM
      k_splitk_reduce_warp<T><<<(unsigned)cdiv(outs, 8), 256, 0, c->stream>>>(W.as<T>(), ksplit, m, n, alpha, beta,
                                                                             C, ldc);
    else
      k_splitk_reduce<T><<<grid1d(outs, 256), 256, 0, c->stream>>>(W.as<T>(), ksplit, m, n, alpha, beta, C, ldc);
    TTI_LAUNCH();
    return;
  }
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    int nb = std::min(65535, batch - b0);
    dim3 grid(cdiv(n, BN), cdiv(m, BM), nb);
    TTI_CHECK_ARG(grid.y <= 65535, "gemm: m=%d too large", m);
    ProfScope ps(c, sizeof(T) == 8 ? PROF_GEMM64 : PROF_OFF, 2.0 * m * (double)n * k * nb);
    launch(grid, A + b0 * sA, B + b0 * sB, beta, C + b0 * sC, ldc, sA, sB, sC, 1, k);
  }
}

template void gemm<double>(Ctx *, bool, bool, int, int, int, double, const double *, long long, long long,
                           const double *, long long, long long, double, double *, long long, long long, int);
template void gemm<float>(Ctx *, bool, bool, int, int, int, float, const float *, long long, long long,
                          const float *, long long, long long, float, float *, long long, long long, int);

// ------------------------------------------------------------- reductions

constexpr int kRedBlocks = 256;

__global__ void k_partial_dot(const double *x, const double *y, long long n, double *part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * (y ? y[i] : x[i]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_final_sum(const double *part, int np, double *out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

void dev_dot(Ctx *c, const double *x, const double *y, long long n, double *out) {
  int nb = (int)std::min<long long>(kRedBlocks, std::max<long long>(1, (n + 255) / 256));
  double *part = c->dscratch + 4096;
  k_partial_dot<<<nb, 256, 0, c->stream>>>(x, y, n, part);
  TTI_LAUNCH();
  k_final_sum<<<1, 256, 0, c->stream>>>(part, nb, out);
  TTI_LAUNCH();
}
void dev_sumsq(Ctx *c, const double *x, long long n, double *out) { dev_dot(c, x, nullptr, n, out); }

double host_dot(Ctx *c, const double *x, const double *y, long long n) {
  dev_dot(c, x, y, n, c->dscratch);
  double v;
  c->d2h(&v, c->dscratch, sizeof v);
  return v;
}
double host_nrm2(Ctx *c, const double *x, long long n) { return sqrt(std::max(0.0, host_dot(c, x, x, n))); }

// ------------------------------------------------------- elementwise helpers

template <typename T>
__global__ void k_scale(T *x, long long n, T a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= a;
}
template <typename T>
__global__ void k_axpy(long long n, T a, const T *x, T *y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
template <typename T> void scale(Ctx *c, T *x, long long n, T a) {
  if (n <= 0) return;
  k_scale<T><<<grid1d(n, 256), 256, 0, c->stream>>>(x, n, a);
  TTI_LAUNCH();
}
template <typename T> void axpy(Ctx *c, long long n, T a, const T *x, T *y) {
  if (n <= 0) return;
  k_axpy<T><<<grid1d(n, 256), 256, 0, c->stream>>>(n, a, x, y);
  TTI_LAUNCH();
}
template void scale<double>(Ctx *, double *, long long, double);
template void scale<float>(Ctx *, float *, long long, float);
template void axpy<double>(Ctx *, long long, double, const double *, double *);
template void axpy<float>(Ctx *, long long, float, const float *, float *);

__global__ void k_d2f(const double *x, float *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_f2d(const float *x, double *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
void convert_f64_to_f32(Ctx *c, const double *x, float *y, long long n) {
  if (n <= 0) return;
  k_d2f<<<grid1d(n, 256), 256, 0, c->stream>>>(x, y, n);
  TTI_LAUNCH();
}
void convert_f32_to_f64(Ctx *c, const float *x, double *y, long long n) {
  if (n <= 0) return;
  k_f2d<<<grid1d(n, 256), 256, 0, c->stream>>>(x, y, n);
  TTI_LAUNCH();
}

__global__ void k_copy2d(double *dst, long long ldd, const double *src, long long lds, int rows, int cols) {
  long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / cols, j = e % cols;
    dst[i * ldd + j] = src[i * lds + j];
  }
}
void copy2d(Ctx *c, double *dst, long long ldd, const double *src, long long lds, int rows, int cols) {
  if ((long long)rows * cols <= 0) return;
  k_copy2d<<<grid1d((long long)rows * cols, 256), 256, 0, c->stream>>>(dst, ldd, src, lds, rows, cols);
  TTI_LAUNCH();
}

__global__ void k_permute3(const double *in, double *out, int d0, int d1, int d2, int p0, int p1, int p2) {
  const int dims[3] = {d0, d1, d2};
  const int od1 = dims[p1], od2 = dims[p2];
  long long tot = (long long)d0 * d1 * d2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long o2 = e % od2, t = e / od2;
    long long o1 = t % od1, o0 = t / od1;
    long long src[3];
    src[p0] = o0;
    src[p1] = o1;
    src[p2] = o2;
    out[e] = in[(src[0] * d1 + src[1]) * d2 + src[2]];
  }
}
void permute3(Ctx *c, const double *in, double *out, int d0, int d1, int d2, int p0, int p1, int p2) {
  long long tot = (long long)d0 * d1 * d2;
  if (tot <= 0) return;
  k_permute3<<<grid1d(tot, 256), 256, 0, c->stream>>>(in, out, d0, d1, d2, p0, p1, p2);
  TTI_LAUNCH();
}

// ------------------------------------------------------------ TSQR (FP64)
//
// Level-0 blocks of mb rows are copied into block-column-major workspaces and
// factorised by Householder reflections, one CTA per block; the stacked k x k
// R factors form the input of the next level until one block remains.  The
// explicit Q is built top-down: each block applies its reflectors to the
// k x k slice of the level above padded with zeros.

__global__ void k_qr_load(const double *__restrict__ A, long long lda, long long rows, int k, int mb,
                          double *__restrict__ W) {
  const long long blk = blockIdx.x;
  double *Wb = W + blk * (long long)mb * k;
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int i = e / k, cc = e % k;
    const long long gr = blk * mb + i;
    Wb[(long long)cc * mb + i] = (gr < rows) ? A[gr * lda + cc] : 0.0;
  }
}

// Y <- H_0 H_1 ... H_{k-1} Y for the reflectors of one block (Wb: column j holds v_j below
// the diagonal, the unit entry implied; tb: the k tau), applied backwards, one warp per
// column of Y.  With `ident` Y starts as the first k columns of the identity: H_j then leaves
// the columns cc < j unchanged (v_j is zero above row j and e_cc is zero from row j on), so
// only columns j .. k-1 are touched, half the work of a general Y.
__device__ __forceinline__ void qr_apply_back(const double *Wb, const double *tb, int mb, int k, double *Yb,
                                              bool ident) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = k - 1; j >= 0; --j) {
    const double tj = tb[j];
    if (tj == 0.0) continue;  // uniform over the CTA
    const double *v = Wb + (long long)j * mb;
    for (int cc = (ident ? j : 0) + warp; cc < k; cc += nw) {
      double *yc = Yb + (long long)cc * mb;
      double w = (lane == 0) ? yc[j] : 0.0, w2 = 0.0;
      int i = j + 1 + lane;
      for (; i + 32 < mb; i += 64) {
        w += v[i] * yc[i];
        w2 += v[i + 32] * yc[i + 32];
      }
      if (i < mb) w += v[i] * yc[i];
      w = warp_sum(w + w2) * tj;
      if (lane == 0) yc[j] -= w;
      for (int i2 = j + 1 + lane; i2 < mb; i2 += 32) yc[i2] -= w * v[i2];
    }
    __syncthreads();
  }
}

// Y (block-column-major, mb x k) <- Cin's k x k slice of this block stacked on zeros, or the
// identity when Cin is null.
__device__ __forceinline__ void qr_init_y(double *Yb, int mb, int k, const double *Cin, long long blk) {
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int cc = e / mb, i = e % mb;
    double v = 0.0;
    if (i < k) v = Cin ? Cin[(blk * k + i) * k + cc] : (i == cc ? 1.0 : 0.0);
    Yb[(long long)cc * mb + i] = v;
  }
}

// Rows blk*mb .. of Out (row-major, k columns, out_rows rows) <- Y.
__device__ __forceinline__ void qr_store_y(const double *Yb, int mb, int k, double *Out, long long out_rows,
                                           long long blk) {
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int i = e / k, cc = e % k;
    const long long row = blk * mb + i;
    if (row < out_rows) Out[row * k + cc] = Yb[(long long)cc * mb + i];
  }
}

// Householder QR of each mb x k block.  With use_smem the block is read straight from
// the source matrix (row-major, ld, `rows` rows; rows past the end read as zero) into a
// shared-memory copy, so no separate layout pass is needed, and the reflectors are
// written back to W at the end; otherwise W already holds the block (k_qr_load).  With
// Qout (one block, use_smem, room for a second mb x k panel) the block's explicit Q is
// formed here from the reflectors still in shared memory and stored to Qout's first
// out_rows rows, which saves the separate Q-formation launch of a single-block level.
__global__ void __launch_bounds__(256) k_qr_panel(double *__restrict__ W, int mb, int k, double *__restrict__ tau,
                                                  double *__restrict__ Rout, int use_smem,
                                                  const double *__restrict__ src, long long ld, long long rows,
                                                  double *__restrict__ Qout, long long out_rows) {
  extern __shared__ double qsm[];
  __shared__ double tsh[256];
  const long long blk = blockIdx.x;
  double *Wg = W + blk * (long long)mb * k;
  double *Wb = Wg;
  if (use_smem) {  // work on a shared-memory copy of the block, write the reflectors back at the end
    for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
      const int i = e / k, cc = e % k;
      const long long gr = blk * mb + i;
      qsm[(long long)cc * mb + i] = (gr < rows) ? src[gr * ld + cc] : 0.0;
    }
    Wb = qsm;
    __syncthreads();
  }
  double *tb = tau + blk * k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // Reflector of column c, run by one warp from s (its sum of squares below the diagonal,
  // the same value in every lane) and its diagonal entry: every lane forms the same
  // scalars, the warp scales the column below the diagonal, lane 0 stores tau and R's
  // diagonal.  beta = -sign(x0) sqrt(h), h = x0^2 + s; with y = 1/sqrt(h): |beta| = h y,
  // tau = (beta - x0) / beta = 1 + |x0| y, and 1/(x0 - beta) = sign(x0) / (|x0| + h y).
  auto make_reflector = [&](int c, double s) {
    double *col = Wb + (long long)c * mb;
    const double x0 = col[c];
    double t = 0.0, beta = x0, sc = 0.0;
    if (s != 0.0) {
      const double h = x0 * x0 + s, y = rsqrt(h), ab = h * y;
      t = 1.0 + fabs(x0) * y;
      beta = -copysign(ab, x0);
      sc = copysign(1.0, x0) / (fabs(x0) + ab);
      for (int i = c + 1 + lane; i < mb; i += 32) col[i] *= sc;
    }
    if (lane == 0) {
      col[c] = beta;
      tb[c] = t;
      tsh[c] = t;
    }
  };
  // Look-ahead: warp 0 applies reflector j to column j + 1 only, summing the squares of the
  // updated entries as it goes, and forms reflector j + 1 at once; warps 1.. update the
  // other trailing columns meanwhile.  One barrier per column, no CTA-wide reduction.
  // (Launched with 256 threads: warps 1..7 exist.)
  if (warp == 0) {
    double sq = 0.0;
    for (int i = 1 + lane; i < mb; i += 32) sq += Wb[i] * Wb[i];
    sq = warp_sum(sq);
    __syncwarp();
    make_reflector(0, sq);
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const double tj = tsh[j];
    const double *v = Wb + (long long)j * mb;
    if (warp == 0) {
      if (j + 1 < k) {
        double *cn = Wb + (long long)(j + 1) * mb;
        double sq = 0.0;
        if (tj != 0.0) {
          double w = (lane == 0) ? cn[j] : 0.0, w2 = 0.0;
          int i = j + 1 + lane;
          for (; i + 32 < mb; i += 64) {
            w += v[i] * cn[i];
            w2 += v[i + 32] * cn[i + 32];
          }
          if (i < mb) w += v[i] * cn[i];
          w = warp_sum(w + w2) * tj;
          if (lane == 0) cn[j] -= w;
          for (int i2 = j + 1 + lane; i2 < mb; i2 += 32) {
            const double y = cn[i2] - w * v[i2];
            cn[i2] = y;
            if (i2 > j + 1) sq += y * y;
          }
        } else {
          for (int i2 = j + 2 + lane; i2 < mb; i2 += 32) sq += cn[i2] * cn[i2];
        }
        sq = warp_sum(sq);
        __syncwarp();
        make_reflector(j + 1, sq);
      }
    } else if (tj != 0.0) {
      for (int cc = j + 1 + warp; cc < k; cc += nw - 1) {
        double *ccol = Wb + (long long)cc * mb;
        double w = (lane == 0) ? ccol[j] : 0.0, w2 = 0.0;
        int i = j + 1 + lane;
        for (; i + 32 < mb; i += 64) {
          w += v[i] * ccol[i];
          w2 += v[i + 32] * ccol[i + 32];
        }
        if (i < mb) w += v[i] * ccol[i];
        w = warp_sum(w + w2) * tj;
        if (lane == 0) ccol[j] -= w;
        for (int i2 = j + 1 + lane; i2 < mb; i2 += 32) ccol[i2] -= w * v[i2];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int row = e / k, cc = e % k;
    Rout[(blk * k + row) * k + cc] = (cc >= row && row < mb) ? Wb[(long long)cc * mb + row] : 0.0;
  }
  if (Qout) {  // one block: Q = H_0 ... H_{k-1} I from the reflectors in shared memory
    double *Yb = qsm + (long long)mb * k;
    qr_init_y(Yb, mb, k, nullptr, 0);
    __syncthreads();
    qr_apply_back(Wb, tsh, mb, k, Yb, true);
    qr_store_y(Yb, mb, k, Qout, out_rows, 0);
    return;  // the reflectors are not needed again
  }
  if (use_smem)
    for (int e = tid; e < mb * k; e += blockDim.x) Wg[e] = Wb[e];
}

// Q of one tree level: each block applies its reflectors to the k x k slice of the level
// above (Cin, or the identity at the top) stacked on zeros.  use_smem: 0 works in global
// memory (Y), 1 keeps Y in shared memory, 2 also stages the reflectors there.
__global__ void __launch_bounds__(256) k_qr_formq(const double *__restrict__ W, const double *__restrict__ tau,
                                                  int mb, int k, const double *__restrict__ Cin,
                                                  double *__restrict__ Y, double *__restrict__ Out,
                                                  long long out_rows, int use_smem) {
  extern __shared__ double qsm[];
  __shared__ double tsh[256];
  const long long blk = blockIdx.x;
  const double *Wb = W + blk * (long long)mb * k;
  double *Yb = use_smem ? qsm : Y + blk * (long long)mb * k;
  if (use_smem == 2) {
    double *Ws = qsm + (long long)mb * k;
    for (int e = threadIdx.x; e < mb * k; e += blockDim.x) Ws[e] = Wb[e];
    Wb = Ws;
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) tsh[j] = tau[blk * k + j];
  qr_init_y(Yb, mb, k, Cin, blk);
  __syncthreads();
  qr_apply_back(Wb, tsh, mb, k, Yb, Cin == nullptr);
  qr_store_y(Yb, mb, k, Out, out_rows, blk);
}

// Rows per TSQR block: 128-row blocks (4k for wide panels), or the whole matrix as one
// block when it has at most 512 rows and little FP64 work (rows k^2 <= 32k FMAs): the
// upper levels of a tree over narrow panels then take one launch instead of two or three.
// Taller single blocks lose: one CTA's column chain grows with the rows.
static int qr_block_rows(long long rows, int k) {
  int mb = std::max(4 * k, 128);
  mb = (mb + 31) / 32 * 32;
  if (rows > mb && rows <= 512 && rows * k * (long long)k <= 32768) mb = (int)((rows + 31) / 32 * 32);
  if (rows <= mb) {
    long long r = std::max<long long>(rows, k);
    mb = (int)((r + 31) / 32 * 32);
  }
  return mb;
}

constexpr size_t kQrSmemBytes = 160 * 1024;

void qr(Ctx *c, int m, int k, const double *A, long long lda, double *Q, double *R) {
  TTI_CHECK_ARG(m >= 1 && k >= 1 && k <= 256, "qr: bad sizes m=%d k=%d", m, k);
  set_smem_limit_once((const void *)k_qr_panel, (int)kQrSmemBytes);
  set_smem_limit_once((const void *)k_qr_formq, (int)kQrSmemBytes);
  struct Level {
    long long rows;
    int mb, nblk;
    DBuf W, tau, Rs;
  };
  std::vector<Level> lv;
  const double *src = A;
  long long ld = lda, rows = m;
  DBuf top_q;           // Q of the top block, formed by its panel launch (the next level's Cin)
  bool fused = false;   // the top level's Q is already formed
  for (;;) {
    Level L;
    L.rows = rows;
    L.mb = qr_block_rows(rows, k);
    L.nblk = cdiv(rows, L.mb);
    L.W = DBuf(c, (size_t)L.nblk * L.mb * k * sizeof(double));
    L.tau = DBuf(c, (size_t)L.nblk * k * sizeof(double));
    L.Rs = DBuf(c, (size_t)L.nblk * k * k * sizeof(double));
    const size_t sm = (size_t)L.mb * k * sizeof(double);
    const int use = sm <= kQrSmemBytes;
    if (!use) {
      k_qr_load<<<L.nblk, 256, 0, c->stream>>>(src, ld, rows, k, L.mb, L.W.d());
      TTI_LAUNCH();
    }
    // a single block with room for a second panel forms its Q in the same launch
    fused = Q && L.nblk == 1 && 2 * sm <= kQrSmemBytes;
    double *qout = nullptr;
    long long out_rows = 0;
    if (fused) {
      if (lv.empty()) {
        qout = Q;
        out_rows = m;
      } else {
        out_rows = (long long)lv.back().nblk * k;
        top_q = DBuf(c, (size_t)out_rows * k * sizeof(double));
        qout = top_q.d();
      }
    }
    {
      ProfScope ps(c, PROF_QR, (fused ? 3.0 : 2.0) * L.nblk * (double)L.mb * k * k);
      k_qr_panel<<<L.nblk, 256, fused ? 2 * sm : (use ? sm : 0), c->stream>>>(
          L.W.d(), L.mb, k, L.tau.d(), L.Rs.d(), use, src, ld, rows, qout, out_rows);
      TTI_LAUNCH();
    }
    lv.push_back(std::move(L));
    Level &top = lv.back();
    if (top.nblk == 1) break;
    src = top.Rs.d();
    ld = k;
    rows = (long long)top.nblk * k;
  }
  TTI_CUDA(cudaMemcpyAsync(R, lv.back().Rs.d(), (size_t)k * k * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (!Q) return;  // R only: the orthogonal factor is not formed
  DBuf Cbuf = std::move(top_q);
  const double *Cin = fused ? Cbuf.d() : nullptr;
  for (int L = (int)lv.size() - (fused ? 2 : 1); L >= 0; --L) {
    Level &l = lv[L];
    DBuf Out;
    double *outp;
    long long out_rows;
    if (L == 0) {
      outp = Q;
      out_rows = m;
    } else {
      out_rows = (long long)lv[L - 1].nblk * k;
      Out = DBuf(c, (size_t)out_rows * k * sizeof(double));
      outp = Out.d();
    }
    const size_t sm = (size_t)l.mb * k * sizeof(double);
    const int use = 2 * sm <= kQrSmemBytes ? 2 : (sm <= kQrSmemBytes ? 1 : 0);
    DBuf Y;
    if (!use) Y = DBuf(c, (size_t)l.nblk * l.mb * k * sizeof(double));
    k_qr_formq<<<l.nblk, 256, use * sm, c->stream>>>(l.W.d(), l.tau.d(), l.mb, k, Cin, Y.d(), outp, out_rows, use);
    TTI_LAUNCH();
    Cbuf = std::move(Out);
    Cin = Cbuf.d();
  }
}

// ------------------------------------------------------- one-sided Jacobi SVD

// One-sided Jacobi SVD of a k x k matrix (k <= 256), one CTA, run on the
// columns of A^T (the rows of A): with A^T J = W converged to orthogonal
// columns, A = J diag(|w_j|) (w_j / |w_j|)^T, so U is the accumulated rotation
// J, exactly orthonormal, and V the normalised columns of W.  The inputs of the
// TT algorithms are triangular factors of tall QRs with graded singular
// values, for which the rows converge in about half the sweeps of the columns,
// and the left factor they need comes out orthonormal to FP64 precision (a
// column of V is orthogonal to the others to about eps s_0 / s_j).  Each pair
// of columns is handled by a group of G lanes (G = 4, 8, 16 or 32, the
// smallest power of two >= k, 32 beyond): the product reduces in log2(G)
// shuffle levels, and all kp/2 pairs of a round run at once when the CTA is
// large enough (for k <= 8 a single warp, synchronised with __syncwarp).  The
// rotation angle is computed in FP32 from the FP64 dot products and cos/sin are
// then formed in FP64 from that tangent, so every rotation is orthogonal to FP64
// precision; an angle that is only FP32-accurate leaves a relative 1e-7 of the
// off-diagonal entry, which later sweeps remove (convergence is tested in FP64:
// g^2 <= tol^2 a b).  A tangent that FP32 cannot represent is computed in FP64.
// Non-convergence after 60 sweeps raises DS_BREAKDOWN in *status (may be null)
// and writes 1 to *info (may be null; 0 when the sweeps converged).
template <int G>
__global__ void __launch_bounds__(1024) k_jacobi_svd(int k, const double *__restrict__ A, double *__restrict__ U,
                                                    double *__restrict__ S, double *__restrict__ V,
                                                    double *Wg, double *Vg, int use_smem, int *status, int *info) {
  extern __shared__ double smem[];
  __shared__ int perm[256];
  __shared__ double nrm[256];
  __shared__ double cn[256];
  const int kp = k + (k & 1);
  double *W = use_smem ? smem : Wg;           // W[c * k + i]: column c, row i
  double *Vw = use_smem ? smem + (size_t)kp * k : Vg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const bool one_warp = blockDim.x == 32;
  auto sync = [&] {
    if (one_warp) __syncwarp();
    else __syncthreads();
  };
  __shared__ double red[32];
  double fro = 0.0;
  for (int e = tid; e < kp * k; e += blockDim.x) {
    const int cc = e / k, i = e % k;
    const double v = (cc < k) ? A[(long long)cc * k + i] : 0.0;  // column cc of A^T
    W[e] = v;
    fro += v * v;
    Vw[e] = (cc == i) ? 1.0 : 0.0;
  }
  fro = warp_sum(fro);
  if (!one_warp) {
    if (lane == 0) red[warp] = fro;
    __syncthreads();
    fro = 0.0;
    for (int w = 0; w < nw; ++w) fro += red[w];
  }
  // columns whose squared norm is below this are roundoff: rotating them changes nothing
  const double tiny = fro * 1e-32 + 1e-300;
  const double tol = 4.0 * k * DBL_EPSILON, tol2 = tol * tol;
  sync();
  const int li = tid % G, grp = tid / G, ngrp = blockDim.x / G;
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    int rotated = 0;
    // squared column norms, exact at the start of each sweep and updated by every rotation
    // (a' = a - t g, b' = b + t g for the pair's squared norms a, b and product g), so a
    // round reduces only the product: one shuffle tree instead of three
    for (int base = 0; base < kp; base += ngrp) {
      const int cc = base + grp;
      double a = 0.0;
      if (cc < kp)
        for (int i = li; i < k; i += G) a += W[(size_t)cc * k + i] * W[(size_t)cc * k + i];
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (cc < kp && li == 0) cn[cc] = a;
    }
    sync();
    for (int rd = 0; rd < kp - 1; ++rd) {
      // every lane runs the same number of passes (the shuffles below need the whole
      // warp); a group without a pair in this pass contributes zeros and rotates nothing
      for (int base = 0; base < kp / 2; base += ngrp) {
        const int pi = base + grp;
        const bool act = pi < kp / 2;
        int p = 0, q = 1;
        if (act) {
          p = (rd + pi) % (kp - 1);
          q = (pi == 0) ? kp - 1 : (rd - pi + kp - 1) % (kp - 1);
          if (p > q) { int t = p; p = q; q = t; }
        }
        double *wp = W + (size_t)p * k, *wq = W + (size_t)q * k;
        double g = 0.0;
        if (act)
          for (int i = li; i < k; i += G) g += wp[i] * wq[i];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        const double a = act ? cn[p] : 0.0, b = act ? cn[q] : 0.0;
        bool renorm = false;
        if (act && g != 0.0 && a > tiny && b > tiny && g * g > tol2 * a * b) {
          const double num = b - a, den = 2.0 * g;
          const float zf = (float)num / (float)den;
          double t;
          if (isfinite(zf) && fabsf(zf) < 1e15f && fabsf(zf) > 1e-15f) {
            t = (double)(copysignf(1.f, zf) / (fabsf(zf) + sqrtf(1.f + zf * zf)));
          } else {
            const double zeta = num / den;
            t = (fabs(zeta) > 1e100) ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          }
          const double cs = rsqrt(1.0 + t * t), sn = cs * t;
          for (int i = li; i < k; i += G) {
            const double x = wp[i], y = wq[i];
            wp[i] = cs * x - sn * y;
            wq[i] = sn * x + cs * y;
          }
          double *vp = Vw + (size_t)p * k, *vq = Vw + (size_t)q * k;
          for (int i = li; i < k; i += G) {
            const double x = vp[i], y = vq[i];
            vp[i] = cs * x - sn * y;
            vq[i] = sn * x + cs * y;
          }
          const double an = a - t * g, bn = b + t * g;
          // a norm that drops by two orders has lost its relative accuracy to cancellation:
          // recompute both from the rotated columns instead (the group agrees on the test)
          renorm = an < 0.01 * a || bn < 0.01 * b;
          if (li == 0) {
            cn[p] = an;
            cn[q] = bn;
          }
          rotated = 1;
        }
        if (__any_sync(0xffffffffu, renorm)) {
          double a2 = 0.0, b2 = 0.0;
          if (renorm)
            for (int i = li; i < k; i += G) {
              a2 += wp[i] * wp[i];
              b2 += wq[i] * wq[i];
            }
#pragma unroll
          for (int o = G / 2; o > 0; o >>= 1) {
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            b2 += __shfl_xor_sync(0xffffffffu, b2, o);
          }
          if (renorm && li == 0) {
            cn[p] = a2;
            cn[q] = b2;
          }
        }
      }
      sync();
    }
    const int any = one_warp ? __any_sync(0xffffffffu, rotated) : __syncthreads_or(rotated);
    if (!any) break;
  }
  if (sweep == 60 && tid == 0 && status) atomicMax(status, (int)DS_BREAKDOWN);
  if (tid == 0 && info) *info = (sweep == 60) ? 1 : 0;
  for (int cc = warp; cc < k; cc += nw) {
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s += W[(size_t)cc * k + i] * W[(size_t)cc * k + i];
    s = warp_sum(s);
    if (lane == 0) nrm[cc] = sqrt(s);
  }
  sync();
  if (tid == 0) {
    for (int i = 0; i < k; ++i) perm[i] = i;
    for (int i = 1; i < k; ++i) {  // insertion sort, descending, stable
      int v = perm[i], j = i - 1;
      while (j >= 0 && nrm[perm[j]] < nrm[v]) { perm[j + 1] = perm[j]; --j; }
      perm[j + 1] = v;
    }
  }
  sync();
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    const int src = perm[j];
    const double sv = nrm[src];
    U[e] = Vw[(size_t)src * k + i];
    V[e] = (sv > 0.0) ? W[(size_t)src * k + i] / sv : 0.0;
  }
  for (int j = tid; j < k; j += blockDim.x) S[j] = nrm[perm[j]];
}

constexpr size_t kSvdSmemMax = 200 * 1024;  // W and V panels in shared memory up to this size

// Lane group and CTA size for a k x k SVD: every pair of a round gets a group.
// Returns the launch's own error code (cudaLaunchKernel), so a caller never
// reports an error left behind by unrelated earlier work on the thread.
static cudaError_t svd_launch(cudaStream_t st, int k, const double *A, double *U, double *s, double *V, double *Wg,
                              double *Vg, int use_smem, size_t bytes, int *status, int *info) {
  const int kp = k + (k & 1), pairs = kp / 2;
  const int G = k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : 32));
  const int threads = std::min(1024, std::max(32, (pairs * G + 31) / 32 * 32));
  const void *fn;
  switch (G) {
    case 4: fn = (const void *)k_jacobi_svd<4>; break;
    case 8: fn = (const void *)k_jacobi_svd<8>; break;
    case 16: fn = (const void *)k_jacobi_svd<16>; break;
    default:
      // the limit is raised once to the largest size any call uses: a per-call value could
      // be lowered by a concurrent call on another thread between its setting and this launch;
      // raised whenever shared memory is used, since the kernel's static arrays count against
      // the default 48 KB too
      fn = (const void *)k_jacobi_svd<32>;
      if (bytes > 0) set_smem_limit_once(fn, (int)kSvdSmemMax);
      break;
  }
  void *args[] = {&k, &A, &U, &s, &V, &Wg, &Vg, &use_smem, &status, &info};
  return cudaLaunchKernel(fn, dim3(1), dim3(threads), args, bytes, st);
}

void svd_small(Ctx *c, int k, const double *A, double *U, double *s, double *V) {
  TTI_CHECK_ARG(k >= 1 && k <= 256, "svd_small: k=%d out of range", k);
  const int kp = k + (k & 1);
  size_t bytes = 2 * (size_t)kp * k * sizeof(double);
  int use_smem = bytes <= kSvdSmemMax;
  DBuf Wg, Vg;
  if (!use_smem) {
    Wg = DBuf(c, (size_t)kp * k * sizeof(double));
    Vg = DBuf(c, (size_t)kp * k * sizeof(double));
    bytes = 0;
  }
  const cudaError_t e = svd_launch(c->stream, k, A, U, s, V, Wg.d(), Vg.d(), use_smem, bytes, c->dstatus, nullptr);
  if (e != cudaSuccess) {
    const int kp2 = k + (k & 1), G = k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : 32));
    fail(TT_IGA_ERR_CUDA, "svd_small launch (k=%d, lanes per pair %d, threads %d, shared bytes %zu): %s", k, G,
         std::min(1024, std::max(32, (kp2 / 2 * G + 31) / 32 * 32)), bytes, cudaGetErrorString(e));
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// ------------------------------------------- allocation-free SVD entry point
//
// Fixed scratch of the one-sided Jacobi SVD for callers that cannot allocate
// device memory: two 256 x 256 FP64 panels (1 MiB) resident on every device
// that loads the library, shared by all calls.  Each call overwrites both
// panels before reading them (the kernel copies A into W and sets V to the
// identity first), so nothing needs clearing between calls; the convergence
// flag goes to the caller's own `info` word, not to the shared array.

static __device__ __align__(256) double g_svd_scratch[2 * 256 * 256];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

int svd_small_noalloc(cudaStream_t stream, int k, const double *A, double *U, double *s, double *V, int *info) {
  if (k < 1 || k > 256) return TT_IGA_ERR_TOO_LARGE;
  if (!A || !U || !s || !V) return TT_IGA_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TT_IGA_ERR_CUDA;
  double *scratch;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      // set-up, once per device with that device current: host code only holds a
      // stand-in for the symbol, so ask the runtime for the array's device address
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_svd_scratch) != cudaSuccess || !p) return TT_IGA_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  // the launch's own return code: an error left by someone else's earlier work is
  // neither reported as ours nor cleared
  const cudaError_t e = svd_launch(stream, k, A, U, s, V, scratch, scratch + 256 * 256, 0, 0, nullptr, info);
  if (e != cudaSuccess) return TT_IGA_ERR_CUDA;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return TT_IGA_OK;
}

// ----------------------------------------------------------------- maxvol

// Deterministic block argmax of |x| over candidates; ties go to the smallest index.
__device__ void block_argmax(double v, long long idx, double *sv, long long *si, double *out_v, long long *out_i) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    long long oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { sv[warp] = v; si[warp] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = sv[0];
    long long bi = si[0];
    for (int w = 1; w < nw; ++w)
      if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
    *out_v = bv;
    *out_i = bi;
  }
  __syncthreads();
}

// Phase 1 (one CTA per matrix): pivot rows by Gaussian elimination with
// partial pivoting on a copy, then the inverse of U[rows, :] by Gauss-Jordan.
__global__ void __launch_bounds__(1024) k_maxvol_init(const int *__restrict__ mm, const int *__restrict__ rr,
                                                      const long long *__restrict__ off, const double *__restrict__ U,
                                                      double *__restrict__ Wk, int *__restrict__ mask,
                                                      const long long *__restrict__ moff, int *__restrict__ rows,
                                                      const long long *__restrict__ roff, double *__restrict__ inv,
                                                      const long long *__restrict__ ioff, int *status) {
  __shared__ double sv[32];
  __shared__ long long si[32];
  __shared__ double bv;
  __shared__ long long bi;
  const int b = blockIdx.x;
  const int m = mm[b], r = rr[b];
  const double *Ub = U + off[b];
  double *W = Wk + off[b];
  int *mk = mask + moff[b];
  int *rw = rows + roff[b];
  double *G = inv + ioff[b];  // [r][2r] augmented matrix
  for (long long e = threadIdx.x; e < (long long)m * r; e += blockDim.x) W[e] = Ub[e];
  for (int i = threadIdx.x; i < m; i += blockDim.x) mk[i] = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    double v = -1.0;
    long long idx = 0x7fffffffffffffffLL;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (mk[i]) continue;
      const double a = fabs(W[(long long)i * r + j]);
      if (a > v || (a == v && i < idx)) { v = a; idx = i; }
    }
    block_argmax(v, idx, sv, si, &bv, &bi);
    if (threadIdx.x == 0) {
      if (bi < 0 || bi >= m) {  // no finite candidate (NaN column): take the first unused row
        bi = 0;
        while (bi < m - 1 && mk[bi]) ++bi;
        if (status) atomicMax(status, (int)DS_NONFINITE);
      }
      rw[j] = (int)bi;
      mk[bi] = 1;
      if (!(bv > 0.0) && status) atomicMax(status, (int)DS_BREAKDOWN);
    }
    __syncthreads();
    const int piv = (int)bi;
    const double pv = W[(long long)piv * r + j];
    if (pv != 0.0) {
      for (long long e = threadIdx.x; e < (long long)m * (r - j - 1); e += blockDim.x) {
        const int i = (int)(e / (r - j - 1)), cc = j + 1 + (int)(e % (r - j - 1));
        if (mk[i]) continue;
        W[(long long)i * r + cc] -= W[(long long)i * r + j] / pv * W[(long long)piv * r + cc];
      }
    }
    __syncthreads();
  }
  // Gauss-Jordan inverse of A = U[rows, :] with partial pivoting.
  for (int e = threadIdx.x; e < r * 2 * r; e += blockDim.x) {
    const int i = e / (2 * r), cc = e % (2 * r);
    G[e] = (cc < r) ? Ub[(long long)rw[i] * r + cc] : ((cc - r) == i ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      int p = j;
      double best = fabs(G[j * 2 * r + j]);
      for (int i = j + 1; i < r; ++i)
        if (fabs(G[i * 2 * r + j]) > best) { best = fabs(G[i * 2 * r + j]); p = i; }
      if (p != j)
        for (int cc = 0; cc < 2 * r; ++cc) {
          double t = G[j * 2 * r + cc];
          G[j * 2 * r + cc] = G[p * 2 * r + cc];
          G[p * 2 * r + cc] = t;
        }
      const double d = G[j * 2 * r + j];
      if (d == 0.0) {
        if (status) atomicMax(status, (int)DS_BREAKDOWN);
      } else {
        for (int cc = 0; cc < 2 * r; ++cc) G[j * 2 * r + cc] /= d;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * 2 * r; e += blockDim.x) {
      const int i = e / (2 * r), cc = e % (2 * r);
      if (i == j || cc == j) continue;
      G[e] -= G[i * 2 * r + j] * G[j * 2 * r + cc];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      if (i != j) G[i * 2 * r + j] = 0.0;
    __syncthreads();
  }
}

// Phase 3 (one CTA per matrix): greedy row swaps while max |B| > 1 + delta.
__global__ void __launch_bounds__(1024) k_maxvol_swap(const int *__restrict__ mm, const int *__restrict__ rr,
                                                      const long long *__restrict__ off, double *__restrict__ B,
                                                      double *__restrict__ colbuf, int *__restrict__ rows,
                                                      const long long *__restrict__ roff, double delta, int maxit) {
  __shared__ double sv[32];
  __shared__ long long si[32];
  __shared__ double bv;
  __shared__ long long bi;
  __shared__ double rowi[256];
  const int b = blockIdx.x;
  const int m = mm[b], r = rr[b];
  double *Bb = B + off[b];
  double *cb = colbuf + off[b];
  int *rw = rows + roff[b];
  for (int it = 0; it < maxit; ++it) {
    double v = -1.0;
    long long idx = 0x7fffffffffffffffLL;
    for (long long e = threadIdx.x; e < (long long)m * r; e += blockDim.x) {
      const double a = fabs(Bb[e]);
      if (a > v || (a == v && e < idx)) { v = a; idx = e; }
    }
    block_argmax(v, idx, sv, si, &bv, &bi);
    if (!(bv > 1.0 + delta)) break;
    const int i = (int)(bi / r), j = (int)(bi % r);
    for (int cc = threadIdx.x; cc < r; cc += blockDim.x) rowi[cc] = Bb[(long long)i * r + cc];
    for (int x = threadIdx.x; x < m; x += blockDim.x) cb[x] = Bb[(long long)x * r + j];
    __syncthreads();
    const double piv = rowi[j];
    for (long long e = threadIdx.x; e < (long long)m * r; e += blockDim.x) {
      const int x = (int)(e / r), cc = (int)(e % r);
      Bb[e] -= cb[x] * (rowi[cc] - (cc == j ? 1.0 : 0.0)) / piv;
    }
    if (threadIdx.x == 0) rw[j] = i;
    __syncthreads();
  }
}

void maxvol_batched(Ctx *c, int count, const int *m, const int *r, const long long *off, const double *U,
                    double *B, int *rows, const long long *rows_off, double delta, int maxit) {
  if (count <= 0) return;
  std::vector<long long> moff(count), ioff(count);
  long long mt = 0, it = 0, tot = 0;
  for (int b = 0; b < count; ++b) {
    TTI_CHECK_ARG(r[b] >= 1 && r[b] <= 256 && m[b] >= r[b], "maxvol: bad sizes m=%d r=%d", m[b], r[b]);
    moff[b] = mt;
    mt += m[b];
    ioff[b] = it;
    it += (long long)r[b] * 2 * r[b];
    tot = std::max(tot, off[b] + (long long)m[b] * r[b]);
  }
  std::vector<int> meta_i(2 * count);
  std::vector<long long> meta_l(4 * count);
  for (int b = 0; b < count; ++b) {
    meta_i[b] = m[b];
    meta_i[count + b] = r[b];
    meta_l[b] = off[b];
    meta_l[count + b] = moff[b];
    meta_l[2 * count + b] = rows_off[b];
    meta_l[3 * count + b] = ioff[b];
  }
  DBuf dmi(c, meta_i.size() * sizeof(int)), dml(c, meta_l.size() * sizeof(long long));
  c->h2d(dmi.get(), meta_i.data(), meta_i.size() * sizeof(int));
  c->h2d(dml.get(), meta_l.data(), meta_l.size() * sizeof(long long));
  const int *dm = dmi.as<int>(), *dr = dm + count;
  const long long *doff = dml.as<long long>(), *dmoff = doff + count, *droff = doff + 2 * count,
                  *dioff = doff + 3 * count;
  DBuf work(c, (size_t)tot * sizeof(double)), mask(c, (size_t)mt * sizeof(int)), inv(c, (size_t)it * sizeof(double));
  k_maxvol_init<<<count, 1024, 0, c->stream>>>(dm, dr, doff, U, work.d(), mask.as<int>(), dmoff, rows, droff,
                                               inv.d(), dioff, c->dstatus);
  TTI_LAUNCH();
  // B = U * inv(U[rows, :]) on the whole GPU (inverse sits in the right half of the augmented matrix)
  for (int b = 0; b < count; ++b)
    gemm<double>(c, false, false, m[b], r[b], r[b], 1.0, U + off[b], r[b], 0, inv.d() + ioff[b] + r[b], 2 * r[b], 0,
                 0.0, B + off[b], r[b], 0, 1);
  k_maxvol_swap<<<count, 1024, 0, c->stream>>>(dm, dr, doff, B, work.d(), rows, droff, delta, maxit);
  TTI_LAUNCH();
}

}  // namespace ttiga
