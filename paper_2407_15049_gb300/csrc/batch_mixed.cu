// Persistent batched-solve kernel, mixed storage (dfloat R and C R, float work arrays).
#include "batch_kernel.cuh"

namespace lorads {
namespace batch {
void* kernel_mixed() { return reinterpret_cast<void*>(&k_batch_solve<dfloat, float>); }
}  // namespace batch
}  // namespace lorads
