// Warp-specialised tile kernel: 4-bit groups, 1q-layer / diagonal op set.
#include "k_tile_ws_fns.cuh"

namespace qs {
template void ws_config<4, KS_LAYER>(int);
template cudaError_t ws_launch<4, KS_LAYER>(const TileArgs &, const CUtensorMap &, const CUtensorMap &, int, int,
                                          cudaStream_t);
template cudaError_t ws_attrs<4, KS_LAYER>(cudaFuncAttributes *);
}  // namespace qs
