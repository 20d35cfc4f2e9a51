// The prefetching general apply kernel with one group factor per thread
// (VINV), AR_DF64.
#include "apply_launch.cuh"

namespace hm {
template cudaError_t launch_apply_pf_t<AR_DF64, true>(const KPlan&, const void*, void*, long long, cudaStream_t,
                                                  TuneCfg);
}  // namespace hm
