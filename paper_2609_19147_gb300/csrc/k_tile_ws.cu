// Tile-pass kernel instantiations: the warp-specialised kernel (a producer
// warpgroup and two consumer groups of 256 threads), 4-bit register groups, for
// 1q-layer / diagonal passes (KS_LAYER) and the general op set.
#include "k_tile_impl.cuh"

namespace qs {

void tile_smem_config_ws(int bytes) {
    cudaFuncSetAttribute(tile_pass_ws_kernel<4, 256, false, KS_LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
    cudaFuncSetAttribute(tile_pass_ws_kernel<4, 256, false, KS_ALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
}

cudaError_t launch_tile_ws(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md, int grid,
                           int smem_bytes, cudaStream_t st) {
    if (R != 4 || A.dense || !A.use_tma || A.threads != 2 * 256 + 128) return cudaErrorInvalidValue;
    if (A.kset == 1)
        tile_pass_ws_kernel<4, 256, false, KS_LAYER><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    else
        tile_pass_ws_kernel<4, 256, false, KS_ALL><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    return cudaGetLastError();
}

cudaError_t tile_attrs_ws(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R != 4) return cudaErrorInvalidValue;
    if (A.kset == 1) return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<4, 256, false, KS_LAYER>);
    return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<4, 256, false, KS_ALL>);
}

}  // namespace qs
