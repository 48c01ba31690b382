// Order-3 tensor-train operations on the device (Section 4.1.1).
#pragma once
#include <vector>
#include "common.cuh"

namespace ttiga {

// Deep copy.
void tt_copy(Ctx *c, const TT3 &x, TT3 &y);
// y = a x + b y as a TT of rank r_x + r_y (block cores); a is applied to core 1.
void tt_sum(Ctx *c, const TT3 &x, double a, const TT3 &y, double b, TT3 &out);
// out = sum of the terms, unrounded: ranks add up (block-diagonal inner cores).
void tt_sum_many(Ctx *c, const std::vector<const TT3 *> &xs, TT3 &out);
// In-place TT rounding to relative accuracy eps (Oseledets 2011): right-to-left
// QR orthogonalisation, left-to-right truncated SVD with threshold
// eps ||X|| / sqrt(2).  Ranks capped at max_rank (0: none).  Returns ||X||_F.
double tt_round(Ctx *c, TT3 &x, double eps, int max_rank);
// Right-orthogonalise core k (1 or 2): core_k = L Q, Q with orthonormal rows
// replaces core_k and L is merged into core_{k-1}.
void orth_right_step(Ctx *c, TT3 &x, int k);
// Right-to-left orthogonalisation only (cores 2, 3 get orthonormal rows);
// returns ||X||_F (norm of core 1).
double tt_orth_rl(Ctx *c, TT3 &x);
// Frobenius norm by orthogonalisation of a copy.
double tt_norm(Ctx *c, const TT3 &x);
// Values at m index triples idx[m][3] (device) into out[m] (device).
void tt_eval_points(Ctx *c, const TT3 &x, int m, const int *idx, double *out);
// Dense tensor out[i3][i2][i1] (i1 fastest; device) of a small TT.
void tt_full(Ctx *c, const TT3 &x, double *out);
// Dense tensor out[i1][i2][i3] (i3 fastest; device) by two GEMMs: cost m1 r1 m2 r2 + m1 m2 r2 m3,
// for TTs whose ranks are too large for the per-entry kernel of tt_full.
void tt_dense(Ctx *c, const TT3 &x, double *out);
// W[j][l] = S[j] V[l][j] for j < r: the first r rows of diag(S) V^T (V is k x k).
void svt(Ctx *c, const double *S, const double *V, int k, int r, double *W);
// Transposes of a core (row-major r0 x (m r1) <-> (m r1) x r0).
void transpose(Ctx *c, const double *in, double *out, long long rows, long long cols);

}  // namespace ttiga
