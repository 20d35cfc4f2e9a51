// Prefetching variant of the general apply kernel, AR_F32 instantiation (own
// translation unit so that the library's units compile in parallel).
#include "apply_launch.cuh"

namespace hm {

template cudaError_t launch_apply_pf_t<AR_F32, false>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);

}  // namespace hm
