// Staged apply kernel, AR_F32 instantiation (own translation unit so that the
// library's units compile in parallel).
#include "stream_launch.cuh"

namespace hm {

template cudaError_t launch_stream_t<AR_F32>(const KPlan&, const void*, void*, long long, cudaStream_t, TuneCfg);

int stream_status_f32(int* out, bool clear) { return stream_status(out, clear); }

}  // namespace hm
