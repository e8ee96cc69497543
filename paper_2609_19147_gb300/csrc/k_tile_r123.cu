// Tile-pass kernel instantiations: 1-3 bit register groups.
#include "k_tile_impl.cuh"

namespace qs {

void tile_smem_config_r123(int bytes) {
    cudaFuncSetAttribute(tile_pass_kernel<1, 256, 1, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(tile_pass_kernel<2, 256, 1, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(tile_pass_kernel<3, 256, 1, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tile_r123(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md,
                          int grid, int smem_bytes, cudaStream_t st) {
    if (R == 1) {
        tile_pass_kernel<1, 256, 1, false><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    if (R == 2) {
        tile_pass_kernel<2, 256, 1, false><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    if (R == 3) {
        tile_pass_kernel<3, 256, 1, false><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

cudaError_t tile_attrs_r123(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R == 1) return cudaFuncGetAttributes(fa, tile_pass_kernel<1, 256, 1, false>);
    if (R == 2) return cudaFuncGetAttributes(fa, tile_pass_kernel<2, 256, 1, false>);
    if (R == 3) return cudaFuncGetAttributes(fa, tile_pass_kernel<3, 256, 1, false>);
    return cudaErrorInvalidValue;
}

}  // namespace qs
