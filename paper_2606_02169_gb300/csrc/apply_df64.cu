// Instantiations of the general apply kernel for one arithmetic policy
// (AR_DF64); the batched kernel is in apply_batch_df64.cu.
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_t<AR_DF64, false>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);
}  // namespace hm
