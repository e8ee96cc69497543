// Launch interfaces of the CUDA kernels (host <-> device argument blocks).
#pragma once

#include <cuda_runtime.h>
#include <string>
#include "qs_internal.h"

namespace qs {

// Tensor-map geometry of a tile pass: up to 5 dims in ascending bit order.
// kind 0: tile range (coordinate 0); kind 1: gap of non-tile bits, coordinate
// = bits [off, off + w) of the tile index (plus batch * 2^w on the top dim);
// kind 2: batch only.
struct TmaGeom {
    int ndims;
    int kind[5];
    int off[5];
    int w[5];
    int batch_dim;          // dim that carries the batch index, -1 if none
};

struct TileArgs {
    const TilePass *pass;      // device copy of the pass descriptor
    const float2 *consts;      // device copy of the pass constants
    const float2 *roots;       // device roots-of-unity tables (kRootsEntries)
    const float2 *src;         // read tiles from
    float2 *dst;               // write tiles to (== src for in-place)
    long long state_elems;     // 2^n
    long long n_tiles;         // tiles per state, 2^(n - T)
    int batch;
    int n_outer;               // number of non-tile index bits
    int outer_pos[kMaxQubits]; // their positions, ascending
    int off_desc, off_consts, off_roots, off_buf0;   // dynamic smem layout
    int n_buf;                 // tile buffers (1..6), each 8 * 2^T bytes from off_buf0
    int prefetch;              // tiles loaded ahead of the one being processed (0..n_buf-1; 0 when n_buf = 1)
    int threads;               // 256, or 512 for 4-bit register groups on 13-bit tiles
    int ctas_per_sm;           // 2: two co-resident CTAs (12-bit tiles, 4-bit groups)
    int l2_prefetch;           // tiles warmed in L2 beyond the shared-memory prefetch
    int use_tma;               // 1: one tensor copy per tile; 0: one bulk copy per row
    int dense;                 // 1: the pass has dense-block sweeps (kernel with the dense paths)
    long long const_stride;    // > 0: batch items differ in constants only; item i's set at
    int const_group;           //   consts + (batch index / const_group) * const_stride
    int kset;                  // 1: every micro-op is a 1q / layer / diagonal op (KS_LAYER kernels)
    int needs_gidx;            // 1: some micro-op reads global indices (controls, diagonals, QFT)
    int ws;                    // 1: warp-specialised kernel (a producer warp and two consumer groups)
    int tmem;                  // 1: dense sweeps on the tcgen05 tensor cores (tensor memory allocated)
    TmaGeom geo;
    int *err;                  // device status word
};

cudaError_t launch_tile_pass(int R, const TileArgs &A, const void *tm_src, const void *tm_dst, int grid,
                             int smem_bytes, cudaStream_t st);
void tile_kernel_smem_config(int bytes);
int tile_ws_threads(int R);   // threads per CTA of the warp-specialised tile kernel (R = 4 or 5)
std::string tile_kernel_attrs(int R, const TileArgs &A);

// per-gate kernels: op per state (op_stride = 1) or shared (op_stride = 0)
struct PgArgs {
    const PgOp *ops;
    int op_stride;
    float2 *psi[2];            // up to two state arrays processed by one launch
    int n_arrays;
    long long state_elems;
    int batch;
    int n;
    int n_fixed;               // fixed (non-enumerated) bit positions, ascending
    int fixed_pos[4];
    long long n_work;          // enumerated indices per state
    int vec2;                  // 1: bit 0 is free -> two consecutive indices per thread
};
cudaError_t launch_pergate(const PgArgs &A, cudaStream_t st);

struct PermArgs {
    const float2 *src;
    float2 *dst;
    long long state_elems;
    int batch;
    int TB;                    // tile bits
    int in_pos[12];            // global input position of input-local bit k
    int out_pos_loc[12];       // global output position of output-local bit k
    int out_to_in[12];         // input-local bit index feeding output-local bit k
    int n_outer;
    int outer_in[kMaxQubits];  // outer input bit positions (ascending)
    int outer_out[kMaxQubits]; // their output positions
    uint64_t xor_outer;        // xor mask on non-tile output bits
    uint32_t xor_loc;          // xor mask in output-local coordinates
};
cudaError_t launch_perm(const PermArgs &A, cudaStream_t st);

struct GatherArgs {
    const GatherPass *g;       // device copy (tables)
    const float2 *src;
    float2 *dst;
    long long state_elems;
    int batch;
};
cudaError_t launch_gather(const GatherArgs &A, cudaStream_t st);

// expectation / reductions (FP64 accumulation)
struct PauliDev {
    double coeff;
    uint64_t x, z;             // index-bit masks
};
struct ExpectArgs {
    const float2 *psi;         // states
    const float2 *lam;         // second states (NULL: <psi|P|psi>)
    long long state_elems;
    long long bstride;         // elements between batch items (0: state_elems)
    int batch;
    uint64_t xmask;            // common x mask of the group
    int n_terms;
    const PauliDev *terms;     // device
    double *partial;           // [batch][grid][n_terms][2]
    int grid;
};
cudaError_t launch_expect_group(const ExpectArgs &A, cudaStream_t st);
// out[b*n_terms + k] (complex, 2 doubles) = sum over blocks of partial
cudaError_t launch_expect_finish(const double *partial, double *out, int batch, int grid, int n_terms,
                                 cudaStream_t st);

// lam = sum_k coeff_k P_k psi  (one launch over all terms; terms sorted by x
// mask share one load per amplitude)
cudaError_t launch_apply_pauli_sum(const float2 *psi, float2 *lam, long long state_elems, int batch,
                                   const PauliDev *terms, int n_terms, cudaStream_t st, long long bstride = 0);

// The same sum over tiles of 2^(4 + H) amplitudes (the 4 low index bits and
// the H <= 8 high bits hb[]) staged in shared memory: every term's x mask lies
// in the tile's bits, so psi[y ^ x] is read from the tile.  A sum whose x
// masks need several bit sets runs as several such passes, the later ones
// adding into lam (accumulate = 1).
constexpr int kPsumMaxTerms = 64;
struct PsumTileArgs {
    const float2 *psi;
    float2 *lam;               // item b at psi + b * bstride, lam + b * bstride
    long long elems, bstride;
    int batch, H;
    int hb[8];                 // ascending high tile bits (>= 4)
    int n_outer;
    int outer[kMaxQubits];     // the other index bits, ascending
    const PauliDev *terms;     // device, <= kPsumMaxTerms, x masks inside the tile
    int n_terms;
    int accumulate;
    int grid;                  // CTAs per item (they stride over the item's tiles)
};
cudaError_t launch_pauli_sum_tile(const PsumTileArgs &A, cudaStream_t st);

// Adjoint-method overlaps of one state pair (psi_b, lam_b) per batch item:
// for the k <= 4 group bits g_j, Im<lam|X_j|psi> and Im<lam|Y_j|psi> (pairs in
// registers) and S_j = sum_{x_gj = 1} Im(conj(lam_x) psi_x); for the bits of
// zmask (outside the group) S_q likewise; and the total sum_x Im(conj(lam_x)
// psi_x), so that Im<lam|Z_q|psi> = total - 2 S_q.
constexpr int kXyzGroup = 4;
constexpr int kXyzZBits = 34;
constexpr int kXyzSlots = 3 * kXyzGroup + kXyzZBits + 2;   // 48: [ImX | ImY | S_g | S_q | total | pad]
struct XyzArgs {
    const float2 *psi, *lam;   // item b at psi + b * bstride, lam + b * bstride
    long long elems, bstride;
    int batch, k;
    int gbit[kXyzGroup];       // ascending index bits
    uint64_t zmask;            // bits outside the group whose S_q is wanted
    double *partial;           // [batch][grid][kXyzSlots]
    int grid;
};
// <psi|D|psi> for D = sum_k coeff_k Z^{z_k} (terms with x = 0), up to 256 terms;
// per-block FP64 sums (states with elems >= 2)
struct DiagExpectArgs {
    const float2 *psi;
    long long elems, bstride;
    int batch, n_terms;
    const PauliDev *terms;     // device, x = 0
    double *partial;           // [batch][grid][2] (re, 0)
    int grid;
};
cudaError_t launch_diag_expect(const DiagExpectArgs &A, cudaStream_t st);

int xyz_grid(long long elems, int k);   // minimum blocks per item
cudaError_t launch_xyz_overlaps(const XyzArgs &A, cudaStream_t st);

// The same overlaps over a tile of 2^(4 + H) amplitudes (the 4 low index bits
// and H <= 8 high bits hb[]) staged in shared memory for psi and lam: X / Y for
// every tile bit in xymask, S_q for the bits of zmask, and the total.
// Slots: [ImX(tile bit t) t < 12 | ImY(t) t < 12 | S_q q < 34 | total | pad].
constexpr int kXyzTileBits = 12;
constexpr int kXyzTSlots = 2 * kXyzTileBits + kXyzZBits + 2;   // 60
struct XyzTileArgs {
    const float2 *psi, *lam;   // item b at psi + b * bstride, lam + b * bstride
    long long elems, bstride;
    int batch, n, H;
    int hb[8];                 // ascending high tile bits (>= 4)
    uint32_t xymask;           // tile bits (0..3 low, 4 + k for hb[k]) whose X / Y are wanted
    uint64_t zmask;            // index bits whose S_q is wanted
    double *partial;           // [batch][grid][kXyzTSlots]
    int grid;                  // CTAs per item (they stride over the item's tiles)
};
cudaError_t launch_xyz_tile(const XyzTileArgs &A, cudaStream_t st);

cudaError_t launch_init_zero(float2 *psi, long long state_elems, int batch, cudaStream_t st);

// batched QAOA MaxCut: one persistent launch over every instance; states with
// n <= 14 in shared memory, n <= 24 in a per-CTA slot of device memory
constexpr int kQaoaMaxSmallN = 14;
constexpr int kQaoaMaxPersistentN = 24;
constexpr int kQaoaMaxEdges = 64;
constexpr int kQaoaMaxP = 16;
struct QaoaItem {
    int n, n_edges;
    int edge_off;      // into edge_masks
    int lut_off;       // into luts: p * (n_edges + 1) entries exp(-i gamma_l k)
    int mix_off;       // into mix: p entries (cos beta_l, -sin beta_l)
    int out_idx;
};
struct QaoaArgs {
    const QaoaItem *items;
    int n_items;
    int p;
    const uint32_t *edge_masks;   // index-bit masks of each edge's two endpoints
    const float2 *luts;
    const float2 *mix;
    double *out;
    int *counter;                 // work queue head (zeroed before launch)
    float2 *slots;                // grid x slot_elems amplitudes (states with n > 14)
    long long slot_elems;         // 2^(largest n above 14), 0 if none
};
int qaoa_smem_bytes();
cudaError_t launch_qaoa(const QaoaArgs &A, int grid, cudaStream_t st);

// message for qs_last_error() on this host thread
void set_last_error(const char *msg);

}  // namespace qs
