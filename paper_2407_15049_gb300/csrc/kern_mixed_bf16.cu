// The mixed form with the search direction D stored in bf16: the direction is
// rounded once when it is formed, and every later use (the C D product and its
// gathers, the line search, the step, the stored pair s = tau D) sees the same
// rounded values, so R, C R and the L-BFGS pairs stay consistent; G, C D and
// the history stay FP32, R and C R double-float.
#include "launch.cuh"

namespace lorads {
LORADS_INSTANTIATE_DIR2(float, bf16)
LORADS_INSTANTIATE_SPMM_C(bf16, float, dfloat)
LORADS_INSTANTIATE_CONS(dfloat, bf16)
LORADS_INSTANTIATE_STEP2(dfloat, float, bf16)
LORADS_INSTANTIATE_UPDATE2(dfloat, float, bf16)
}  // namespace lorads
