// One instantiation of the warp-specialised tile kernel (R-bit register
// groups, op set KS) with its shared-memory attribute, launch and attribute
// query.  Each (R, KS) is instantiated in a unit of its own (k_tile_ws*.cu), so
// that the four compile in parallel; k_tile_ws.cu dispatches between them.
#pragma once
#include "k_tile_impl.cuh"

namespace qs {

// consumer group size: 256 threads with 4-bit groups, 128 with 5-bit groups
template <int R>
constexpr int ws_group_threads() {
    return R == 4 ? 256 : 128;
}

template <int R, int KS>
void ws_config(int bytes) {
    cudaFuncSetAttribute(tile_pass_ws_kernel<R, ws_group_threads<R>(), false, KS>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int R, int KS>
cudaError_t ws_launch(const TileArgs &A, const CUtensorMap &ms, const CUtensorMap &md, int grid, int smem_bytes,
                      cudaStream_t st) {
    tile_pass_ws_kernel<R, ws_group_threads<R>(), false, KS><<<grid, A.threads, smem_bytes, st>>>(ms, md, A);
    return cudaGetLastError();
}

template <int R, int KS>
cudaError_t ws_attrs(cudaFuncAttributes *fa) {
    return cudaFuncGetAttributes(fa, tile_pass_ws_kernel<R, ws_group_threads<R>(), false, KS>);
}

}  // namespace qs
