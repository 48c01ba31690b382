// Solution evaluation and L2 error (Eq. L2norm).
#pragma once
#include "handles.cuh"

namespace ttiga {

void eval_points(Ctx *c, const tt_iga_solution *u, int m, const double *xi, double *out);
double l2_error(Ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_rhs_desc *rhs);

}  // namespace ttiga
