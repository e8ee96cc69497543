// Warp-specialised tile kernel: 5-bit groups, every op.
#include "k_tile_ws_fns.cuh"

namespace qs {
template void ws_config<5, KS_ALL>(int);
template cudaError_t ws_launch<5, KS_ALL>(const TileArgs &, const CUtensorMap &, const CUtensorMap &, int, int,
                                          cudaStream_t);
template cudaError_t ws_attrs<5, KS_ALL>(cudaFuncAttributes *);
}  // namespace qs
