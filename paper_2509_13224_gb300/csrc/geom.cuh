// Discretisation tables and geometry point evaluation (Sections 2 and 3.3).
#pragma once
#include "common.cuh"

namespace ttiga {

// 1D B-spline space of one direction with its Gauss rule, resident on the device.
struct Space {
  int n = 0, p = 0, nq = 0, ne = 0, Q = 0;
  DBuf pts, wts, N, dN;  // [Q], [Q], [Q][p+1], [Q][p+1]
};

// Geometry parameters passed by value to kernels.
struct GeomParams {
  int kind;
  double r_in, r_out, height, twist, swell;
  double lx, ly, lz;
  // NURBS patch (kind TT_IGA_GEOM_NURBS): degrees, control points per direction and
  // the packed device data: knots of directions 0, 1, 2, weights, control points
  // (x, y, z interleaved), control-point index i1 fastest.
  int nd[3], nc[3];
  const double *nurbs;
};

struct RhsParams {
  int kind;
  int n_modes;
  double a[TT_IGA_MAX_MODES], b[TT_IGA_MAX_MODES][3], c[TT_IGA_MAX_MODES];
  double value;
  int has;  // 0: f = 0
};

GeomParams geom_params(const tt_iga_geom_desc &g);
RhsParams rhs_params(const tt_iga_rhs_desc *r);

// Fill a Space on the device (Golub-Welsch Gauss rule, Cox-de Boor tables).
void build_space(Ctx *c, Space &s, int n, int p, int nq);
void basis_tables(Ctx *c, int n, int p, int nq, double *pts, double *wts, double *N, double *dN);

// First cross component beyond the 8 point outputs: component kFaceComp0 + f is the
// area density of face f = 2 d + side (field_value in geom_device.cuh).
constexpr int kFaceComp0 = 8;

// Evaluate the 8 point outputs (R11 R12 R13 R22 R23 R33 detJ f*detJ) at m grid
// points idx[m][3] (device); out[m][8] (device).
void geom_points(Ctx *c, const GeomParams &g, const RhsParams &f, const double *x1, const double *x2,
                 const double *x3, int m, const int *idx, double *out);

// Evaluate one output component `comp` (0..7) at the points of a structured
// sample set described by index generators (see cross.cu).
struct FiberSet;

}  // namespace ttiga
