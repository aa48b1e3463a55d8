// Double-float instantiations: every factor in (hi, lo) float pairs, FP32 units only.
#include "launch.cuh"

namespace lorads {
LORADS_INSTANTIATE_SPMM_C(dfloat, dfloat, dfloat)
LORADS_INSTANTIATE_SPMM_A(dfloat, dfloat)
LORADS_INSTANTIATE_CONS(dfloat, dfloat)
LORADS_INSTANTIATE_DIR(dfloat)
LORADS_INSTANTIATE_STEP(dfloat, dfloat)
LORADS_INSTANTIATE_UPDATE(dfloat, dfloat)
}  // namespace lorads
