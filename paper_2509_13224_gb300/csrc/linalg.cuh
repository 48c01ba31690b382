// Dense linear algebra on the device used by TT rounding, TT-cross and AMEn:
// strided-batched GEMM (FP64 / FP32), tall-skinny Householder QR, one-sided
// Jacobi SVD, maximum-volume row selection and deterministic reductions.
#pragma once
#include "common.cuh"

namespace ttiga {

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], row-major, op(X) = X or X^T.
// op(A) is m x k: element (i, l) is A[i*lda + l] (ta = false) or A[l*lda + i] (ta = true).
template <typename T>
void gemm(Ctx *c, bool ta, bool tb, int m, int n, int k, T alpha, const T *A, long long lda,
          long long sA, const T *B, long long ldb, long long sB, T beta, T *C, long long ldc,
          long long sC, int batch = 1);

// Sum of squares / dot product of n doubles, written to device *out (deterministic).
void dev_sumsq(Ctx *c, const double *x, long long n, double *out);
void dev_dot(Ctx *c, const double *x, const double *y, long long n, double *out);
double host_nrm2(Ctx *c, const double *x, long long n);
double host_dot(Ctx *c, const double *x, const double *y, long long n);

// Tall-skinny QR: A (m x k, row-major, lda) = Q (m x k, ld k) R (k x k upper).
// For m < k the columns m..k-1 of Q and rows m..k-1 of R are zero.  Q may be
// null: then only R is computed (the form-Q tree is skipped).
void qr(Ctx *c, int m, int k, const double *A, long long lda, double *Q, double *R);

// SVD of a k x k row-major matrix: A = U diag(s) V^T, s descending (k <= 256).
void svd_small(Ctx *c, int k, const double *A, double *U, double *s, double *V);

// Allocation-free variant of svd_small on `stream` (k <= 256) using the
// library's fixed device scratch; *info (device, may be null) receives 0 when the
// Jacobi sweeps converged, 1 otherwise.  Returns a tt_iga_status.
int svd_small_noalloc(cudaStream_t stream, int k, const double *A, double *U, double *s, double *V, int *info);

// Batched maxvol on `count` tall matrices U_b (m_b x r_b, row-major, ld r_b,
// contiguous at offsets off[b] in doubles): rows_b[r_b] and B_b = U_b U_b[rows]^{-1}.
// All pointers device; m, r, off are host arrays.
void maxvol_batched(Ctx *c, int count, const int *m, const int *r, const long long *off,
                    const double *U, double *B, int *rows, const long long *rows_off, double delta,
                    int maxit);

// Elementwise helpers.
template <typename T> void scale(Ctx *c, T *x, long long n, T a);
template <typename T> void axpy(Ctx *c, long long n, T a, const T *x, T *y);  // y += a x
void convert_f64_to_f32(Ctx *c, const double *x, float *y, long long n);
void convert_f32_to_f64(Ctx *c, const float *x, double *y, long long n);
void copy2d(Ctx *c, double *dst, long long ldd, const double *src, long long lds, int rows, int cols);
// out[i][j][k] = in[perm-mapped] for a 3D array in[d0][d1][d2]; perm gives the
// source axis of each destination axis.
void permute3(Ctx *c, const double *in, double *out, int d0, int d1, int d2, int p0, int p1, int p2);

}  // namespace ttiga
