// FP64 instantiation of the fused local PCG (pcg_fused_impl.cuh); the two
// precisions are separate translation units so that they compile in parallel.
#include "pcg_fused_impl.cuh"

namespace ttiga {

template int pcg_fused_grid<double>(Ctx *, PcgArgs<double> &);
template void pcg_fused<double>(Ctx *, PcgArgs<double>, int);
template void bb_solve_once<double>(Ctx *, const BBPrec &, int, int, int, int, const double *, double *);

}  // namespace ttiga
