// Internal definitions shared by the planner (host C++) and the CUDA kernels.
//
// Plan model.  The detector turns a gate list into an ordered list of fused
// ops (the layer families of Sec. 5.1-5.2), and the scheduler packs them into
// full-state HBM passes:
//   * TILE pass   -- one read + one write of the state.  A CTA stages a tile
//                    of 2^T amplitudes (the L lowest index bits, contiguous,
//                    plus T-L chosen high bits) in shared memory with
//                    bulk-async (TMA engine) copies, runs a list of "sweeps"
//                    over it and writes it back.  A sweep gives every thread
//                    2^r amplitudes that differ in r tile bits (held in
//                    registers) and applies micro-ops to them: 2x2 / 4x4
//                    unitaries on tile bits with optional controls on any
//                    bits, diagonal phase layers, and QFT stages (Hadamard
//                    butterfly + the stage's controlled-phase ladder in closed
//                    form, Sec. 5.1 "Radix-4 butterflies").
//   * PERM pass   -- out-of-place bit permutation plus XOR mask (runs of
//                    SWAP / X; the QFT's final swaps), tile-transposed through
//                    shared memory so that reads and writes are both
//                    row-contiguous.
//   * GATHER pass -- out-of-place GF(2) affine gather out[y] = in[A y ^ c]
//                    (Sec. 5.1 "GF(2) affine permutation gathers").
//   * PERGATE op  -- one launch per gate: the plain per-gate path (Sec. 3.2.2
//                    structured dispatch), used as the baseline and for gates
//                    no family covers.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

#include "qs.h"

namespace qs {

constexpr int kMaxQubits = 33;
constexpr int kMaxTileBits = 14;     // T
constexpr int kMaxGroup = 5;         // r: amplitudes per thread = 2^r
constexpr int kMaxSweeps = 40;
constexpr int kMaxMicro = 320;
constexpr int kMaxConst = 5120;      // complex64 constants per pass (40 KB)
constexpr int kMaxConstDense = 10240; // ... in plans with dense blocks (80 KB: 13-bit tiles, 2 buffers)
constexpr int kMaxDiag = 4;
constexpr int kTileThreads = 256;     // threads per tile CTA
constexpr int kMaxTileBuffers = 8;

// Diagonal phase (Sec. 5.1 "Phase-LUT diagonal layers").  The phase of basis
// index x is
//   gphase * prod_s SLICE_s[(x >> lo_s) & (2^w_s - 1)]
//          * prod_g LUT_g[popcount(f_g(x) & m_g)]
//          * prod_t TW(x_{p_t} * (x & bits[lo_t, p_t)), p_t)
// with f_g(x) = x ^ (x >> d_g) (ZZ-type mismatch count) or x & (x >> d_g)
// (CZ-type both-set count), and TW(u, p) = exp(i pi u / 2^p) (the QFT ladder
// angle).  Tables are built on the host in FP64, reduced mod 2 pi and rounded
// once to complex64.
constexpr int kMaxSlices = 6;
constexpr int kMaxLutGroups = 8;
constexpr int kMaxTwiddles = 4;

struct DiagDesc {
    int32_t n_slices, n_groups, n_tw, pad0;   // pad0: has a global-phase constant
    int32_t gph_off, pad1;                      // constant offset of exp(i g0)
    int32_t slice_lo[kMaxSlices], slice_w[kMaxSlices], slice_off[kMaxSlices];
    int32_t grp_type[kMaxLutGroups], grp_d[kMaxLutGroups], grp_off[kMaxLutGroups];
    uint64_t grp_mask[kMaxLutGroups];
    int32_t tw_p[kMaxTwiddles], tw_lo[kMaxTwiddles];
};

enum MicroKind : int32_t {
    MK_U1 = 0,    // 2x2 on group bit a where (x & cmask) == cval
    MK_U2 = 1,    // 4x4 on group bits (a = matrix MSB, b = LSB) where (x & cmask) == cval
    MK_DIAG = 2,  // diagonal phase, diag index = cst; a = mask of slices and
                  // b = mask of LUT groups that depend on the sweep's group bits
    MK_QFT = 3,   // QFT stage: H on group bit a (= global bit p), then twiddle
                  // exp(i pi x_p (x & bits[lo, p)) / 2^p); group part at cst
    MK_H = 4,     // Hadamard on group bit a (sign-only butterfly)
    MK_RXC = 5,   // [[c, i s], [i s, c]] on group bit a (RX family): consts c, s
    MK_U1R = 6,   // real 2x2 on group bit a (RY family): consts (m00, m00), (m01, m01),
                  // (m10, m10), (m11, m11) at an even offset (two 16-byte loads, each
                  // entry already the packed FP32x2 operand)
    MK_LAYER = 7, // commuting 2x2 ops of one kind (a = MK_RXC / MK_U1R / MK_U1 / MK_H / MK_ROT)
                  // on the group bits in mask b; constants per bit m at cst + m * stride.
                  // A ROT layer of a rotation program has b = all group bits (the others
                  // identities, t = 0) and its own bits in lo
    MK_QFTL = 8,  // QFT stages (ladders down to bit 0) on the group bits in mask b,
                  // applied from the highest group bit down; p of bit m = (p >> 6m) & 63
                  // (p is a packed 64-bit field: use cmask); group table of bit m at cst + m * 2^R
    MK_DIAGQ = 9, // diagonal factored per sweep: the tables of diag cst at the item's base
                  // index (group bits 0), times Q[j] (2^R entries at p: the group bits' own
                  // terms), times prod over set group bits m of the couplings of bit m to
                  // other bits: (cmask >> 6m) & 63 entries at lo + 2 m kMaxCouple, each a
                  // pair (bit index as int bits, exp(i beta)) applied where that bit is set
    MK_DIAGC = 10, // diagonal exp(i (g0 + gamma c1(x) + h c2(x))): c1 = number of edges
                  // (u, v) of an edge set with x_u != x_v (b = 0, ZZ type) or x_u = x_v = 1
                  // (b = 1, CZ type), c2 = popcount(x & Mz); table LUT[c1 + p c2] at cst
                  // (p = |E| + 1).  Per item c1(x_0) (group bits 0) = sum over a = n_cls
                  // distance classes of popcount(f_d(x_0) & M_d); group bit m adds delta_m
                  // (ZZ: deg_m - 2 popcount(x_0 & N_m); CZ: popcount(x_0 & N_m); N_m = its
                  // neighbours outside the group) plus p if it is in Mz; the edges inside
                  // the group add Qc[j] (4 bits per j, packed in cmask for j < 16 and cval
                  // for j >= 16).  Data at lo (uint64 slots): N_m (R slots), the R degrees
                  // (6 bits each), Mz, the R Mz increments (12 bits each), then per class
                  // M_d and d.
    MK_ROT = 11,  // real rotation c [[1, t], [-t, 1]] (|t| <= 1) on group bit a: consts
                  // (t, t), (-t, -t) (packed FP32x2 operands); the factor c is folded into
                  // the sweep scale, so the op is one packed FMA per amplitude
    MK_ZYZ = 12,  // a 2x2 unitary on every group bit, each factored (FP64, on the host) as
                  // U = diag(e^{i a}, e^{i b}) [[c, -s], [s, c]] diag(1, e^{i d}); consts at
                  // cst: PIN[2^R] = prod_m (x_m ? e^{i d_m} : 1), POUT[2^R], then per group
                  // bit m the packed pairs (k0, k0), (k1, k1), then one entry whose x holds
                  // the form mask F as int bits.  Per amplitude vector: a[j] *= PIN[j]; per
                  // bit (a0, a1) <- (a0 + k0 a1, a1 + k1 a0) from the old values; a[j] *=
                  // POUT[j]; the result a[j] is element j ^ F.  Bit m clear: k = -+s/c
                  // (|c| >= |s|); set: k = +-c/s, which leaves the bit's pair exchanged.
                  // POUT holds the output phases and the rotations' factors, permuted by F
};
constexpr int kMaxCouple = 16;
constexpr int kMaxCountClasses = 24;

// item-address tables per sweep (shared memory): item bits 0-4, 5-9, 10-13,
// then the sweep's group bits (kGroupTab entries: shared-memory offset and
// global index bit of group bit m)
constexpr int kGroupTab = 8;
constexpr int kItemTab = 32 + 32 + 16 + kGroupTab;

struct MicroOp {
    int32_t kind;
    int32_t a, b;          // group-local bit indices
    int32_t p, lo;         // QFT: global bit p, lowest ladder bit
    int32_t cst;           // constant offset (complex64 entries) / diag index
    uint64_t cmask, cval;  // control condition on the global index
};

// Dense-block sweeps (qs_dense_prec): out = U X on the 5 group bits, where X
// is the tile viewed as a 32 x 2^(T-5) matrix (row = the group bits, column =
// the item bits).  Constants at dcst:
//   DS_FP32    U as 32 x 32 complex64, row-major (row = output index);
//   DS_TF32X3  32 x 32 pairs (U_hi, U_lo) of complex64, TF32-rounded on the
//              host from FP64: entry (i, j) at pair i * 32 + (j ^ 4 (i & 1)) (the
//              XOR makes the tensor-core operand loads conflict-free);
//   DS_BF16    U in the m16n8k16 B-operand register order: for k-step s < 4,
//              n-tile t < 8 and lane l, one float2 holding 4 packed BF16.
enum DenseKind : int32_t { DS_NONE = 0, DS_FP32 = 1, DS_TF32X3 = 2, DS_BF16 = 3 };

struct Sweep {
    int32_t r;                   // group size (1..kMaxGroup)
    int32_t op_begin, op_end;    // micro-op range [begin, end)
    int32_t vec;                 // group bit 0 is tile-local bit 0: 16-byte pair accesses
    float scale;                 // folded butterfly normalisation, applied once at the end
    int32_t dense;               // DenseKind: a dense-block sweep (r = 5, no micro-ops)
    int32_t dcst;                // dense sweep: constant offset of the block's tables
    int32_t gbit[kMaxGroup];     // tile-local bit of group bit j
    int32_t tbit[kMaxTileBits];  // tile-local bit of item bit i (i < T - r)
};

// One tile pass.  Tile-local bits 0..L-1 are the low index bits; tile-local
// bit L+k is global bit hb[k] (hb ascending).  In shared memory the tile is
// dense in tile-local order, optionally with the 128-byte TMA swizzle; the
// float2 offset of a tile element is the XOR of smem_contrib[] over its set
// tile-local bits.  Tiles are indexed by the remaining n-T bits (ascending).
struct TilePass {
    int32_t n, L, H, T;
    int32_t R;                           // register group size of the micro-op sweeps
    int32_t swizzle;                     // 1: 128-byte swizzle (TMA tensor path)
    int32_t n_sweeps, n_micro, n_const;
    int32_t hb[kMaxTileBits];
    int32_t smem_contrib[kMaxTileBits];
    Sweep sweeps[kMaxSweeps];
    MicroOp micro[kMaxMicro];
    DiagDesc diags[kMaxDiag];
};

// Roots-of-unity tables used by TW(u, p): R_k[c] = exp(i pi c 2^(8k) / 2^32)
// for k = 0..3, c < 256, so that exp(i pi v / 2^32) = prod_k R_k[byte_k(v)].
constexpr int kRootsEntries = 4 * 256;

// ---------------------------------------------------------------------------
// PERM pass: out[pi(x) ^ c] = in[x] for a bit permutation pi (out bit
// out_pos[b] <- in bit b).  Tile = in-bits {0..L-1} U pi^-1({0..L-1}).
// ---------------------------------------------------------------------------
struct PermPass {
    int32_t n, L;
    int32_t out_pos[kMaxQubits];
    uint64_t xor_mask;
};

// ---------------------------------------------------------------------------
// GATHER pass: out[y] = in[c ^ T_0[y & 255] ^ T_1[(y >> 8) & 255] ^ ...]
// with T_k[b] = A (b << 8k) (byte-sliced XOR tables of the inverse map).
// ---------------------------------------------------------------------------
struct GatherPass {
    int32_t n, n_slices;
    uint64_t c;
    uint64_t tab[5][256];
};

// ---------------------------------------------------------------------------
// Per-gate kernels: generic forms of the paper's structured pure tier.
// ---------------------------------------------------------------------------
enum PgKind : int32_t {
    PG_U1 = 0,     // 2x2 on bit t over the subspace (x & cmask) == cval
    PG_U2 = 1,     // 4x4 on bits (t0 msb, t1 lsb) over the subspace
    PG_PHASE = 2,  // amp *= ph[(bit t0 of x) | (bit t1 of x) << 1] over subspace
    PG_SWAP = 3,   // swap bits t0, t1 over the subspace
};

struct PgOp {
    int32_t kind;
    int32_t t0, t1;
    int32_t nbits_phase;   // PG_PHASE: 1 (bit t0) or 2 (t0, t1)
    uint64_t cmask, cval;
    float2 m[16];          // matrix or phases
};

}  // namespace qs
