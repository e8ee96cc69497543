// Tile-pass kernel instantiations: passes with dense-block sweeps (5-bit register
// groups).
#include "k_tile_impl.cuh"

namespace qs {

void tile_smem_config_dense(int bytes) {
    cudaFuncSetAttribute(tile_pass_kernel<5, 256, 1, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tile_dense(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md,
                          int grid, int smem_bytes, cudaStream_t st) {
    if (R == 5 && A.dense) {
        tile_pass_kernel<5, 256, 1, true><<<grid, 256, smem_bytes, st>>>(ms, md, A);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

cudaError_t tile_attrs_dense(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R == 5 && A.dense) return cudaFuncGetAttributes(fa, tile_pass_kernel<5, 256, 1, true>);
    return cudaErrorInvalidValue;
}

}  // namespace qs
