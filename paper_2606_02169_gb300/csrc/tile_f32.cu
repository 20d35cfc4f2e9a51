// Instantiation of the tile kernel for FP32 storage.
#include "tile_kernel.cuh"

namespace hm {
template cudaError_t launch_tile_t<AR_F32>(const KTile&, const void*, void*, cudaStream_t, TuneCfg);
}  // namespace hm
