// FP64 instantiations: every factor and every product in double.
#include "launch.cuh"

namespace lorads {
LORADS_INSTANTIATE_SPMM_C(double, double, double)
LORADS_INSTANTIATE_SPMM_A(double, double)
LORADS_INSTANTIATE_CONS(double, double)
LORADS_INSTANTIATE_DIR(double)
LORADS_INSTANTIATE_STEP(double, double)
LORADS_INSTANTIATE_UPDATE(double, double)
}  // namespace lorads
