// Instantiations of the batched apply kernel for AR_F32.
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_batch_t<AR_F32>(const std::vector<const Plan*>&, const void* const*, void* const*,
                                           long long, cudaStream_t);
}  // namespace hm
