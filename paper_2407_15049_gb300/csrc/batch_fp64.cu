// Persistent batched-solve kernel, fp64 storage (double R and C R, double work arrays).
#include "batch_kernel.cuh"

namespace lorads {
namespace batch {
void* kernel_fp64() { return reinterpret_cast<void*>(&k_batch_solve<double, double>); }
}  // namespace batch
}  // namespace lorads
