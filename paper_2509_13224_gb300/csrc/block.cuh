// Several right-hand sides of one system as a single block-TT solve (Section
// 4.1.2, AMEn, applied to the block system).
#pragma once
#include "handles.cuh"

namespace ttiga {

// Mode that carries the right-hand-side index when the caller leaves the choice to the library.
constexpr int kDefaultStackMode = 1;

// Block system of the right-hand sides of s: the right-hand-side index k is
// merged into mode `mode` (g = i + m k with m the mode's size), the operator is
// I_nrhs (x) K (that core replicated per block, no coupling across blocks), and
// the single load is sum_k e_k (x) F_k / ||F_k|| (block-diagonal TT cores),
// rounded to relative accuracy eps.  scale[k] = ||F_k||.
void stack_system(Ctx *c, const tt_iga_system *s, int mode, double eps, tt_iga_system *out,
                  std::vector<double> &scale);
// Block k of a block-system solution, times scale: the solution of right-hand
// side k of the original system.
void unstack_solution(Ctx *c, const tt_iga_solution *ub, int k, double scale, tt_iga_solution *out);

}  // namespace ttiga
