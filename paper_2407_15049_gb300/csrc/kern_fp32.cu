// FP32 instantiations: FP32 storage and products, FP64 cross-row reductions.
#include "launch.cuh"

namespace lorads {
LORADS_INSTANTIATE_SPMM_C(float, float, float)
LORADS_INSTANTIATE_SPMM_A(float, float)
LORADS_INSTANTIATE_CONS(float, float)
LORADS_INSTANTIATE_DIR(float)
LORADS_INSTANTIATE_STEP(float, float)
LORADS_INSTANTIATE_UPDATE(float, float)
}  // namespace lorads
