// TT-cross interpolation of point-evaluated fields on the tensor Gauss grid
// (Section 4.1.2, TT-cross; Sections 4.2.1 and 4.2.2).
#pragma once
#include "geom.cuh"

namespace ttiga {

struct CrossResult {
  TT3 tt;
  bool zero = false;       // field vanishes to the tolerance (rank 0)
  double max_rel_err = 0;  // validated max |TT - f| / scale on random samples
  double scale = 0;        // max |f| over the samples
  bool converged = true;
  long long evaluations = 0;
};

// Cross of output component comp (0..7 of the point evaluator, 8..13 the face
// area densities, see field_value) on the grid of
// spaces s[3].  eps: relative accuracy; zero_scale: fields with max |f| below
// 1e-13 * zero_scale are rank 0 (pass 0 to use the field's own scale).
// zero_ref (optional) replaces zero_scale: it is called once, with max |f| over
// the first fibre sample, and returns the reference (0: the field's own scale);
// it lets concurrent fields exchange their magnitudes.
void cross3(Ctx *c, const Space *s, const GeomParams &g, const RhsParams &f, int comp, double eps, int max_rank,
            uint64_t seed, double zero_scale, CrossResult &out,
            const std::function<double(double)> *zero_ref = nullptr);

// Values of component comp at explicit grid points idx[m][3] (device) -> out[m].
void field_points(Ctx *c, const Space *s, const GeomParams &g, const RhsParams &f, int comp, int m, const int *idx,
                  double *out);

}  // namespace ttiga
