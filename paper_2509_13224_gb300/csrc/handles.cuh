// Library-owned objects behind the opaque C handles.
#pragma once
#include "cross.cuh"
#include "geom.cuh"

// Geometry: discretisation of each direction and the TT cores of the six
// unique entries of R (order R11, R12, R13, R22, R23, R33).
struct tt_iga_geom {
  ttiga::Ctx *ctx = nullptr;
  tt_iga_geom_desc desc{};
  ttiga::GeomParams gp{};
  ttiga::Space s[3];
  ttiga::CrossResult R[6];
  double ms_cross = 0.0;
  ttiga::DBuf nurbs;  // packed NURBS patch (kind TT_IGA_GEOM_NURBS), see GeomParams
};

namespace ttiga {
// Which basis functions are unknowns and the lift of the Dirichlet data:
// direction d keeps functions lo[d] .. nfull[d] - 1 - hi[d]; the lift is
// lift_lo N_0(xi_dir) + lift_hi N_{n-1}(xi_dir) (dir = -1: no lift).
struct BoundaryLayout {
  int lo[3] = {1, 1, 1}, hi[3] = {1, 1, 1}, nfull[3] = {0, 0, 0};
  int lift_dir = -1;
  double lift_lo = 0.0, lift_hi = 0.0;
  double flux[6] = {0, 0, 0, 0, 0, 0};  // outward normal flux of the natural faces
  bool has_flux() const {
    for (double q : flux)
      if (q != 0.0) return true;
    return false;
  }
};
}  // namespace ttiga

// Restricted TT system: band-stored operator with mode sizes n_d(2p+1) and one
// TT load vector per right-hand side with mode sizes n_d (the unknowns).
struct tt_iga_system {
  ttiga::Ctx *ctx = nullptr;
  int n[3] = {0, 0, 0};   // restricted sizes nfull_d - lo_d - hi_d
  int p = 0, b = 0;       // degree and band width 2p + 1
  ttiga::BoundaryLayout bl;
  ttiga::TT3 K;
  std::vector<ttiga::TT3> F;
  std::vector<double> F_norm;
  int stacked = 1;     // > 1: block system of that many right-hand sides merged into one mode
  int stack_mode = 0;  // the mode (0, 1, 2) that carries the right-hand-side index
};

struct tt_iga_solution {
  ttiga::Ctx *ctx = nullptr;
  int n[3] = {0, 0, 0};   // restricted sizes
  int p = 0;
  ttiga::BoundaryLayout bl;
  ttiga::TT3 u;
  int stacked = 1;     // > 1: solution of a block system (slice it with tt_iga_solution_unstack)
  int stack_mode = 0;
};

namespace ttiga {

// Output index of field (i, j), i <= j, in the R array.
inline int field_of(int i, int j) {
  if (i > j) { int t = i; i = j; j = t; }
  static const int map[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return map[i][j];
}

void stiffness_core(Ctx *c, int n, int p, int nq, const double *wts, const double *N, const double *dN,
                    const double *G, int r0, int r1, int test_deriv, int trial_deriv, double *M);
void load_core(Ctx *c, int n, int p, int nq, const double *wts, const double *N, const double *G, int r0, int r1,
               double *F);
// Boundary layout of bc (nullptr: six homogeneous Dirichlet faces); fails with
// TT_IGA_ERR_ARG on the cases tt_iga_assemble_bc rejects.
BoundaryLayout boundary_layout(const tt_iga_bc_desc *bc, const int nfull[3]);
void assemble_system(Ctx *c, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int n_rhs, double round_tol,
                     const BoundaryLayout &bl, tt_iga_system *out);
// Restricted mass matrix M_ab = int N_a N_b det J (band TT-matrix, mode sizes
// (n_d - lo_d - hi_d)(2p+1)); det J by TT-cross to the geometry's tolerance.
void mass_matrix(Ctx *c, const tt_iga_geom *g, const BoundaryLayout &bl, TT3 &M);
// Dense restricted operator entries for (row, col) multi-index pairs (device arrays).
void operator_entries(Ctx *c, const tt_iga_system *s, int m, const int *rows, const int *cols, double *out);

}  // namespace ttiga
