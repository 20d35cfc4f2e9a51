// Instantiations of the tile kernel for FP64 storage: double-float
// arithmetic on the split input, and native FP64 (diagnostic variant).
#include "tile_kernel.cuh"

namespace hm {
template cudaError_t launch_tile_t<AR_DF64>(const KTile&, const void*, void*, cudaStream_t, TuneCfg);
template cudaError_t launch_tile_t<AR_F64>(const KTile&, const void*, void*, cudaStream_t, TuneCfg);
}  // namespace hm
