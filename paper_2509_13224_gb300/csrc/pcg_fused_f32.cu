// FP32 instantiation of the fused local PCG (pcg_fused_impl.cuh); the two
// precisions are separate translation units so that they compile in parallel.
#include "pcg_fused_impl.cuh"

namespace ttiga {

template int pcg_fused_grid<float>(Ctx *, PcgArgs<float> &);
template void pcg_fused<float>(Ctx *, PcgArgs<float>, int);

}  // namespace ttiga
