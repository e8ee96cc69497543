// Tile-pass launcher: picks the kernel instantiation for the pass (register
// group size R, threads, CTAs per SM, dense sweeps, op set); the
// instantiations live in k_tile_r123.cu, k_tile_r4.cu, k_tile_r5.cu,
// k_tile_layer4.cu, k_tile_layer5.cu, k_tile_dense.cu and k_tile_ws.cu.
#include <cuda.h>

#include <string>

#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

#define QS_TILE_TU(sfx)                                                                                    \
    void tile_smem_config_##sfx(int bytes);                                                                \
    cudaError_t launch_tile_##sfx(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md, \
                                  int grid, int smem_bytes, cudaStream_t st);                              \
    cudaError_t tile_attrs_##sfx(int R, const TileArgs &A, cudaFuncAttributes *fa);
QS_TILE_TU(r123)
QS_TILE_TU(r4)
QS_TILE_TU(r5)
QS_TILE_TU(dense)
QS_TILE_TU(layer4)
QS_TILE_TU(layer5)
QS_TILE_TU(ws)
#undef QS_TILE_TU

void tile_kernel_smem_config(int bytes) {
    tile_smem_config_r123(bytes);
    tile_smem_config_r4(bytes);
    tile_smem_config_r5(bytes);
    tile_smem_config_dense(bytes);
    tile_smem_config_layer4(bytes);
    tile_smem_config_layer5(bytes);
    tile_smem_config_ws(bytes);
}

// R = register group size; 4-bit groups on 13-bit tiles run 512 threads (16
// warps per SM); passes with dense sweeps need R = 5
cudaError_t launch_tile_pass(int R, const TileArgs &A, const void *tm_src, const void *tm_dst, int grid,
                             int smem_bytes, cudaStream_t st) {
    const CUtensorMap &ms = *reinterpret_cast<const CUtensorMap *>(tm_src);
    const CUtensorMap &md = *reinterpret_cast<const CUtensorMap *>(tm_dst);
    cudaGetLastError();
    if (A.ws) return launch_tile_ws(R, A, ms, md, grid, smem_bytes, st);
    if (A.dense) return launch_tile_dense(R, A, ms, md, grid, smem_bytes, st);
    if (A.kset == 1 && R == 4) return launch_tile_layer4(R, A, ms, md, grid, smem_bytes, st);
    if (A.kset == 1 && R == 5) return launch_tile_layer5(R, A, ms, md, grid, smem_bytes, st);
    if (R == 5) return launch_tile_r5(R, A, ms, md, grid, smem_bytes, st);
    if (R == 4) return launch_tile_r4(R, A, ms, md, grid, smem_bytes, st);
    return launch_tile_r123(R, A, ms, md, grid, smem_bytes, st);
}

std::string tile_kernel_attrs(int R, const TileArgs &A) {
    cudaFuncAttributes fa;
    cudaError_t e = A.ws                   ? tile_attrs_ws(R, A, &fa)
                    : A.dense              ? tile_attrs_dense(R, A, &fa)
                    : A.kset == 1 && R == 4 ? tile_attrs_layer4(R, A, &fa)
                    : A.kset == 1 && R == 5 ? tile_attrs_layer5(R, A, &fa)
                    : R == 5 ? tile_attrs_r5(R, A, &fa)
                    : R == 4 ? tile_attrs_r4(R, A, &fa)
                             : tile_attrs_r123(R, A, &fa);
    if (e != cudaSuccess) return "attrs unavailable";
    return "regs=" + std::to_string(fa.numRegs) + " maxThreads=" + std::to_string(fa.maxThreadsPerBlock) +
           " maxDynSmem=" + std::to_string(fa.maxDynamicSharedSizeBytes) +
           " staticSmem=" + std::to_string(fa.sharedSizeBytes) + " localBytes=" + std::to_string(fa.localSizeBytes);
}

}  // namespace qs
