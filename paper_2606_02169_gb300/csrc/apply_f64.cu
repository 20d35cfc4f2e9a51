// Instantiations of the apply kernels for one arithmetic policy (AR_F64).
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_t<AR_F64, false>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);
template cudaError_t launch_batch_t<AR_F64>(const std::vector<const Plan*>&, const void* const*, void* const*,
                                           long long, cudaStream_t);
}  // namespace hm
