// BF16-storage instantiations (FP32 arithmetic) of the standalone entry points.
#include "launch.cuh"

namespace lorads {
LORADS_INSTANTIATE_SPMM_C(bf16, float, bf16)
LORADS_INSTANTIATE_SPMM_A(bf16, float)
LORADS_INSTANTIATE_CONS(bf16, bf16)
}  // namespace lorads
