// AMEn TT solver entry points (Section 4.1.2).
#pragma once
#include "handles.cuh"

namespace ttiga {

// Solve K u = F[opts.rhs_index]; returns TT_IGA_OK or TT_IGA_ERR_NOT_CONVERGED
// (the last iterate is stored in *out either way).  start (may be null): initial
// iterate with the system's mode sizes, otherwise a random rank-2 TT.
int amen_solve(Ctx *c, const tt_iga_system *s, const tt_iga_solve_opts &opts, tt_iga_solution *out, tt_iga_stats *st,
               const tt_iga_solution *start = nullptr);
// Exact ||F_k - K u|| / ||F_k||: TT arithmetic while the residual's TT rank allows
// it, dense vectors for small problems beyond that, -1 when neither applies.
double exact_residual(Ctx *c, const tt_iga_system *s, const tt_iga_solution *u, int k);

}  // namespace ttiga
