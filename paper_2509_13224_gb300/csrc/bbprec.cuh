// Exact block-band preconditioner for AMEn local systems whose interface block
// m = rl * rr is small (Section 4.1.2, local solves of the TT linear solver).
//
// With the unknowns of a local system x[a][i][c] taken mode-index-major, the
// local matrix B = sum_{g,d} PhiL_g (x) A_k[g, d] (x) PhiR_d is block banded:
// n block rows of m unknowns (padded to M = 4 or 8), half-bandwidth p
// blocks, because the operator core A_k is banded in the mode index.  Its block
// Cholesky factor B ~ L L^T (FP32) is an exact preconditioner up to FP32
// rounding, so PCG on these systems converges in a few iterations whatever the
// coupling between the interface ranks (the band block-Jacobi preconditioner
// keeps only the interface diagonals).  Stored per block row i (FP32):
//   Linv[i]        = L_ii^{-1}                          [M][M]
//   G[i][k-1]      = L_ii^{-1} L(i, i-k),       k = 1..p  [M][S]  (forward)
//   H[i][k-1]      = L_ii^{-T} L(i+k, i)^T,     k = 1..p  [M][S]  (backward)
// rows padded to the stride S = bb_stride(M) so that the lanes of a warp read
// their rows with conflict-free 16-byte shared loads.  Then
//   y_i = L_ii^{-1} r_i - sum_k G_ik y_{i-k},   z_i = L_ii^{-T} y_i - sum_k H_ik z_{i+k}.
// G and H blocks that reach outside 0..n-1 are zero.
#pragma once
#include "amen_ops.cuh"

namespace ttiga {

// Largest interface block handled: past m = 8 the sequential factorisation costs
// more than the band block-Jacobi iterations it saves.
constexpr int kBBMaxM = 8;
__host__ __device__ constexpr int bb_stride(int M) { return M == 8 ? 12 : 8; }
__host__ __device__ constexpr int bb_pad(int m) { return m <= 4 ? 4 : 8; }

struct BBPrec {
  DBuf Linv, G, H;
  int n = 0, p = 0, m = 0, M = 0;
};

// True when the local system of the given shape uses the block-band preconditioner.
bool bb_eligible(int m, int n, int p);

// Build and factor the block-band preconditioner of B = PhiL (x) A (x) PhiR.
// phase_clk (optional, device, 3 entries): SM cycles of the factorisation's
// diagonal, panel and trailing-update phases.
void bb_prec_build(Ctx *c, const double *PhiL, int rl, const BandCore &A, const double *PhiR, int rr, BBPrec &P,
                   unsigned long long *phase_clk = nullptr);

}  // namespace ttiga
