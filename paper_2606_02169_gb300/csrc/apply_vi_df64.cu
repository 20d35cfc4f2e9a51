// The general apply kernel with one group factor per thread (VINV), AR_DF64
// (own translation unit so that the units compile in parallel).
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_t<AR_DF64, true>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);
}  // namespace hm
