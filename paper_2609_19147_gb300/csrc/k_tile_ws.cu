// Dispatch between the warp-specialised tile kernel's instantiations (a
// producer warpgroup and two consumer groups): 4-bit register groups with 256
// threads per group, 5-bit groups with 128, each for 1q-layer / diagonal
// passes (KS_LAYER) and the general op set, compiled in k_tile_ws{5l,5a,4l,4a}.cu.
#include <cuda.h>

#include "qs_kernels.h"

namespace qs {

constexpr int kWsLayer = 1;   // KS_LAYER
constexpr int kWsAll = 0;     // KS_ALL

template <int R, int KS>
void ws_config(int bytes);
template <int R, int KS>
cudaError_t ws_launch(const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md, int grid, int smem_bytes,
                      cudaStream_t st);
template <int R, int KS>
cudaError_t ws_attrs(cudaFuncAttributes *fa);

void tile_smem_config_ws(int bytes) {
    ws_config<4, kWsLayer>(bytes);
    ws_config<4, kWsAll>(bytes);
    ws_config<5, kWsLayer>(bytes);
    ws_config<5, kWsAll>(bytes);
}

// threads per CTA of the warp-specialised kernel for register group size R
int tile_ws_threads(int R) { return R == 4 ? 2 * 256 + 128 : R == 5 ? 2 * 128 + 128 : 0; }

cudaError_t launch_tile_ws(int R, const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md, int grid,
                           int smem_bytes, cudaStream_t st) {
    if (A.dense || !A.use_tma || A.threads != tile_ws_threads(R)) return cudaErrorInvalidValue;
    if (R == 4 && A.kset == 1) return ws_launch<4, kWsLayer>(A, ms, md, grid, smem_bytes, st);
    if (R == 4) return ws_launch<4, kWsAll>(A, ms, md, grid, smem_bytes, st);
    if (R == 5 && A.kset == 1) return ws_launch<5, kWsLayer>(A, ms, md, grid, smem_bytes, st);
    if (R == 5) return ws_launch<5, kWsAll>(A, ms, md, grid, smem_bytes, st);
    return cudaErrorInvalidValue;
}

cudaError_t tile_attrs_ws(int R, const TileArgs &A, cudaFuncAttributes *fa) {
    if (R == 4 && A.kset == 1) return ws_attrs<4, kWsLayer>(fa);
    if (R == 4) return ws_attrs<4, kWsAll>(fa);
    if (R == 5 && A.kset == 1) return ws_attrs<5, kWsLayer>(fa);
    if (R == 5) return ws_attrs<5, kWsAll>(fa);
    return cudaErrorInvalidValue;
}

}  // namespace qs
