// Instantiations of the general apply kernel and the batched kernel for the
// double-float vector policy (2 right-hand sides of one state per element).
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_t<AR_DF64V2, false>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);
template cudaError_t launch_batch_t<AR_DF64V2>(const std::vector<const Plan*>&, const void* const*, void* const*,
                                              long long, cudaStream_t);
}  // namespace hm
