// Tile-pass kernel instantiations: 1q-layer and diagonal passes (KS_LAYER), 5-bit register groups.
#include "k_tile_impl.cuh"

namespace qs {

void tile_smem_config_layer5(int bytes) {
    cudaFuncSetAttribute(tile_pass_kernel<5, 256, 1, false, KS_LAYER>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(tile_pass_kernel<5, 128, 2, false, KS_LAYER>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tile_layer5(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md,
                          int grid, int smem_bytes, cudaStream_t st) {
    if (R == 5 && A.ctas_per_sm == 2) {
        tile_pass_kernel<5, 128, 2, false, KS_LAYER><<<grid, 128, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    if (R == 5) {
        tile_pass_kernel<5, 256, 1, false, KS_LAYER><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

cudaError_t tile_attrs_layer5(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R == 5 && A.ctas_per_sm == 2) return cudaFuncGetAttributes(fa, tile_pass_kernel<5, 128, 2, false, KS_LAYER>);
    if (R == 5) return cudaFuncGetAttributes(fa, tile_pass_kernel<5, 256, 1, false, KS_LAYER>);
    return cudaErrorInvalidValue;
}

}  // namespace qs
