// Instantiation of the one-pass complex-H kernel for the native FP64 (two doubles)
// (re, im) element policy.
#include "apply_cx.cuh"

namespace hm {
template cudaError_t launch_apply_cx_t<AR_F64V2>(const KPlan&, const KPlan&, const void*, void*, long long, cudaStream_t,
                                            int, KGate, bool, bool);
}  // namespace hm
