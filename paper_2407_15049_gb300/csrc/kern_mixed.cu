// Mixed instantiations: R and C R kept in double-float (feasibility and the
// gradient's cancellation need ~48 bits), direction, C D, gradient and L-BFGS
// history in FP32.  No per-element FP64 arithmetic.
#include "launch.cuh"

namespace lorads {
LORADS_INSTANTIATE_SPMM_C(float, float, dfloat)
LORADS_INSTANTIATE_SPMM_A(dfloat, float)
LORADS_INSTANTIATE_CONS(dfloat, float)
LORADS_INSTANTIATE_STEP(dfloat, float)
LORADS_INSTANTIATE_UPDATE(dfloat, float)
}  // namespace lorads
