// Instantiations of the general apply kernel for one arithmetic policy
// (AR_F32); the batched kernel is in apply_batch_f32.cu.
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_t<AR_F32, false>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);
}  // namespace hm
