// Persistent batched-solve kernel, fp32 storage (float R and C R, float work arrays).
#include "batch_kernel.cuh"

namespace lorads {
namespace batch {
void* kernel_fp32() { return reinterpret_cast<void*>(&k_batch_solve<float, float>); }
}  // namespace batch
}  // namespace lorads
