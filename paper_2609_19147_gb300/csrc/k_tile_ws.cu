// Tile-pass kernel instantiations: the warp-specialised kernel (a producer
// warpgroup and two consumer groups) -- 4-bit register groups with 256
// threads per group, 5-bit groups with 128 -- for 1q-layer / diagonal passes
// (KS_LAYER) and the general op set.
#include "k_tile_impl.cuh"

namespace qs {

void tile_smem_config_ws(int bytes) {
    cudaFuncSetAttribute(tile_pass_ws_kernel<4, 256, false, KS_LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
    cudaFuncSetAttribute(tile_pass_ws_kernel<4, 256, false, KS_ALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
    cudaFuncSetAttribute(tile_pass_ws_kernel<5, 128, false, KS_LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
    cudaFuncSetAttribute(tile_pass_ws_kernel<5, 128, false, KS_ALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
}

// threads per CTA of the warp-specialised kernel for register group size R
int tile_ws_threads(int R) { return R == 4 ? 2 * 256 + 128 : R == 5 ? 2 * 128 + 128 : 0; }

cudaError_t launch_tile_ws(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md, int grid,
                           int smem_bytes, cudaStream_t st) {
    if (A.dense || !A.use_tma || A.threads != tile_ws_threads(R)) return cudaErrorInvalidValue;
    if (R == 4 && A.kset == 1)
        tile_pass_ws_kernel<4, 256, false, KS_LAYER><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    else if (R == 4)
        tile_pass_ws_kernel<4, 256, false, KS_ALL><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    else if (R == 5 && A.kset == 1)
        tile_pass_ws_kernel<5, 128, false, KS_LAYER><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    else if (R == 5)
        tile_pass_ws_kernel<5, 128, false, KS_ALL><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t tile_attrs_ws(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R == 4 && A.kset == 1) return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<4, 256, false, KS_LAYER>);
    if (R == 4) return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<4, 256, false, KS_ALL>);
    if (R == 5 && A.kset == 1) return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<5, 128, false, KS_LAYER>);
    if (R == 5) return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<5, 128, false, KS_ALL>);
    return cudaErrorInvalidValue;
}

}  // namespace qs
