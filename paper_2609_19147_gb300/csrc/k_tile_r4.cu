// Tile-pass kernel instantiations: 4-bit register groups (512 threads on 13-bit tiles,
// two 256-thread CTAs per SM on 12-bit tiles).
#include "k_tile_impl.cuh"

namespace qs {

void tile_smem_config_r4(int bytes) {
    cudaFuncSetAttribute(tile_pass_kernel<4, 512, 1, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(tile_pass_kernel<4, 256, 2, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(tile_pass_kernel<4, 256, 1, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tile_r4(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md,
                          int grid, int smem_bytes, cudaStream_t st) {
    if (R == 4 && A.threads == 512) {
        tile_pass_kernel<4, 512, 1, false><<<grid, 512, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    if (R == 4 && A.ctas_per_sm == 2) {
        tile_pass_kernel<4, 256, 2, false><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    if (R == 4) {
        tile_pass_kernel<4, 256, 1, false><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

cudaError_t tile_attrs_r4(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R == 4 && A.threads == 512) return cudaFuncGetAttributes(fa, tile_pass_kernel<4, 512, 1, false>);
    if (R == 4 && A.ctas_per_sm == 2) return cudaFuncGetAttributes(fa, tile_pass_kernel<4, 256, 2, false>);
    if (R == 4) return cudaFuncGetAttributes(fa, tile_pass_kernel<4, 256, 1, false>);
    return cudaErrorInvalidValue;
}

}  // namespace qs
