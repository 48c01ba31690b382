// Exact block-band preconditioner for AMEn local systems whose interface block
// m = rl * rr is small (Section 4.1.2, local solves of the TT linear solver).
//
// With the unknowns of a local system x[a][i][c] taken mode-index-major, the
// local matrix B = sum_{g,d} PhiL_g (x) A_k[g, d] (x) PhiR_d is block banded:
// n block rows of m unknowns (padded to M = 4 or 8, padding carries the
// identity), half-bandwidth p blocks, because the operator core A_k is banded in
// the mode index.  Grouping p consecutive block rows into a super-row of
// q = p M unknowns makes B block tridiagonal over S = ceil(n / p) super-rows
// (padding super-rows past n carry the identity): diagonal blocks D_J and
// couplings C_J = B(super-row J, super-row J - 1).
//
// B is factorised by odd-even (cyclic) reduction, in FP32.  At level l
// (h = 2^l) the active super-rows are the multiples of h, and those that are
// odd multiples are eliminated, all at once:
//   L_j L_j^T = D_j,   Ul_j = L_j^{-1} C_j,   Ur_j = L_j^{-1} C_{j+h}^T,
// and the Schur complements update the rows left for level l + 1:
//   D_{j-h} -= Ul_j^T Ul_j,   D_{j+h} -= Ur_j^T Ur_j,   C_{j+h} <- -Ur_j^T Ul_j
// (the last is the new coupling of j + h with j - h).  Super-row 0 is left at
// the top and factored last.  This is the block Cholesky factor of B with its
// super-rows in odd-even order, so the preconditioner is B^{-1} up to FP32
// rounding and PCG on these systems converges in one or two iterations, but the
// factorisation and the substitutions are log2(S) levels deep instead of n
// sequential block steps.  Stored per super-row (FP32, [S][q][q] row-major):
//   Linv[J] = L_J^{-1},  Ul[J],  Ur[J]  (zero where the neighbour does not exist).
// Solving B z = r:
//   forward   for l = 0 .. top-1: y_j = Linv_j b_j for the rows eliminated at l,
//             then each row active at l + 1: b_J -= Ur_{J-h}^T y_{J-h} + Ul_{J+h}^T y_{J+h};
//             y_0 = Linv_0 b_0
//   backward  z_0 = Linv_0^T y_0; for l = top-1 .. 0:
//             z_j = Linv_j^T (y_j - Ul_j z_{j-h} - Ur_j z_{j+h}).
#pragma once
#include "amen_ops.cuh"

namespace ttiga {

// Largest interface block handled: past m = 8 the band block-Jacobi iterations
// cost less than the q^3 work per super-row.
constexpr int kBBMaxM = 8;
__host__ __device__ constexpr int bb_pad(int m) { return m <= 4 ? 4 : 8; }

struct BBPrec {
  DBuf Linv, Ul, Ur;  // [S][q][q] each (FP32)
  int n = 0, p = 0, m = 0, M = 0, S = 0, q = 0, levels = 0;
};

// True when the local system of the given shape uses the block-band preconditioner.
bool bb_eligible(int m, int n, int p);

// Build and factor the block-band preconditioner of B = PhiL (x) A (x) PhiR.
void bb_prec_build(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, BBPrec &P);

}  // namespace ttiga
