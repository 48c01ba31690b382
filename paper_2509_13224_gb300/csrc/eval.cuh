// Solution evaluation and L2 error (Eq. L2norm).
#pragma once
#include "handles.cuh"

namespace ttiga {

void eval_points(Ctx *c, const tt_iga_solution *u, int m, const double *xi, double *out);
double l2_error(Ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_rhs_desc *rhs);
// sqrt(int (u_h - v_h)^2 / int v_h^2) over the mapped domain with the Gauss rule of the
// discretisation, in TT arithmetic (mass matrix, rounded difference); u and v share the
// discretisation and carry no Dirichlet lift.
double l2_diff(Ctx *c, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_solution *v);

}  // namespace ttiga
