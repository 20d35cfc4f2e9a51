// Instantiations of the general apply kernel and the batched kernel for the
// FP32 vector policy with 4 right-hand sides of one state per element.
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_t<AR_F32V4, false>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);
template cudaError_t launch_batch_t<AR_F32V4>(const std::vector<const Plan*>&, const void* const*, void* const*,
                                             long long, cudaStream_t);
}  // namespace hm
