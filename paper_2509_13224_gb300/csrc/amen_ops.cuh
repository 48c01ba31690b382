// Contractions of the AMEn local systems (Section 4.1.2, TT linear solver).
//
// Shapes (row-major, last index fastest):
//   TT core          X[rl][n][rr]
//   band TT-matrix   A[Rl][n][b][Rr]   (entry (i, j) at slot o = j - i + p)
//   left interface   PhiL[ol][Rl][il]  (test rank, operator rank, trial rank)
//   right interface  PhiR[or][Rr][ir]
//   load interfaces  PsiL[ol][fl], PsiR[or][fr]
#pragma once
#include "common.cuh"

namespace ttiga {

struct BandCore {
  const double *A;
  const float *A32;  // FP32 copy (mixed precision), may be null
  int Rl, n, b, p, Rr;
};

template <typename T> struct Work {
  Ctx *c;
  DBuf t1, t2;
  T *get1(size_t elems) { return ensure(t1, elems); }
  T *get2(size_t elems) { return ensure(t2, elems); }
  T *ensure(DBuf &d, size_t elems) {
    if (d.bytes() < elems * sizeof(T)) d = DBuf(c, elems * sizeof(T));
    return d.as<T>();
  }
};

// y[ol][n][or] = sum PhiL[ol][g][il] A[g][i][o][d] PhiR[or][d][ir] x[il][i+o-p][ir]
template <typename T>
void apply_local(Ctx *c, Work<T> &w, const T *PhiL, int ol, int il, const BandCore &A, const T *Ak, const T *PhiR,
                 int orr, int ir, const T *x, T *y);
// Left interface update: out[tr][Rr][ur] = sum Z[tl][i][tr] PhiL[tl][g][ul] A[g][i][o][d] U[ul][i+o-p][ur]
void left_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const double *PhiL, const BandCore &A,
                 const double *U, int ul, int ur, double *out);
// Right interface update: out[tl][Rl][ul] = sum Z[tl][i][tr] A[g][i][o][d] PhiR[tr][d][ur] U[ul][i+o-p][ur]
void right_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const BandCore &A, const double *PhiR,
                  const double *U, int ul, int ur, double *out);
// Local right-hand side: y[ol][n][or] = sum PsiL[ol][fl] F[fl][i][fr] PsiR[or][fr]
void rhs_local(Ctx *c, Work<double> &w, const double *PsiL, int ol, const double *F, int fl, int n, int fr,
               const double *PsiR, int orr, double *y);
void rhs_left_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const double *PsiL, const double *F,
                     int fl, int n, int fr, double *out);  // out[tr][fr]
void rhs_right_update(Ctx *c, Work<double> &w, const double *Z, int tl, int tr, const double *F, int fl, int n, int fr,
                      const double *PsiR, double *out);  // out[tl][fl]

// Band block-Jacobi preconditioner of the local system: for every (alpha, beta)
// the n x n band matrix sum_{g,d} PhiL[a][g][a] A[g][.][.][d] PhiR[b][d][b],
// factorised by band Cholesky.  L layout: [n][p+1][rl*rr] (pair index fastest).
template <typename T>
void precond_build(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, T *L);

// Matrix-vector product of the band TT-matrix with a TT core: out[(g,a)][i][(d,b)].
void tt_matvec_core(Ctx *c, const BandCore &A, const double *U, int ul, int ur, double *out);

}  // namespace ttiga
