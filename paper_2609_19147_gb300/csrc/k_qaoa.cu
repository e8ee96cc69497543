// Batched QAOA MaxCut: every instance (graph, angle set) of a batch in one
// persistent launch (Sec. 3.2.3 QAOA: |+>^n, then for l = 1..p the cost phase
// e^{-i gamma_l H_C} and the mixer e^{-i beta_l H_M}, then <C>).
//
// CTAs pull instance indices from a device work counter (atomicAdd; no waits
// on other CTAs).  Per instance:
//   n <= 14: the whole state stays in the CTA's shared memory (128 KiB at
//            n = 14); cut(x) is computed once into shared memory.
//   n <= 24: the state lives in the CTA's own slot of device memory and moves
//            through shared memory in tiles of 2^14 amplitudes, two passes per
//            layer: pass A holds the low 14 index bits (a contiguous block)
//            and applies RX(2 beta) on them; pass B holds the high bits (and
//            enough low bits for 128-byte rows), applies RX on the high bits
//            and then the next layer's cost phase, or, after the last layer,
//            accumulates <C> instead of storing.  The first pass generates
//            |+>^n with the first cost phase instead of reading a state.
//            Each sweep holds 32 amplitudes of an item (5 tile bits) in a
//            thread's registers, two items per thread; the first sweep of a
//            pass reads device memory and the last writes it, the others go
//            through shared memory.
// cut(x) = number of edges whose endpoint bits differ; per thread it is
// formed for x0 (the register group's bits clear) from the vertices' neighbour
// masks and extended over the group by doubling: setting vertex G changes the
// cut by deg(G) - 2 |N(G) & x|.  exp(-i gamma_l k) comes from FP64-built tables.
#include <cuda_runtime.h>

#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

constexpr int kQaoaThreads = 256;   // two items (of 512) per thread in each tile sweep
constexpr int kQaoaTileBits = 14;
constexpr int kQaoaLutStride = kQaoaMaxEdges + 1;

// shared memory: [0, 128 KiB) the state (n <= 14) or a tile; [128, 144 KiB)
// cut counts (n <= 14); then p cost tables, edge masks, neighbour masks
constexpr int kQaoaSmemTile = 8 << kQaoaTileBits;
constexpr int kQaoaSmemCut = 1 << kQaoaTileBits;
constexpr int kQaoaSmemLut = kQaoaMaxP * kQaoaLutStride * 8;
constexpr int kQaoaSmemMasks = kQaoaMaxEdges * 4;
constexpr int kQaoaSmemNbr = 32 * 4;

__device__ __forceinline__ float2 qa_cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// RX(2 beta) = [[c, i s], [i s, c]], c = cos beta, s = -sin beta
__device__ __forceinline__ void qa_rx(float2 &a0, float2 &a1, float2 cs) {
    const float2 b0 = make_float2(fmaf(cs.x, a0.x, -cs.y * a1.y), fmaf(cs.x, a0.y, cs.y * a1.x));
    const float2 b1 = make_float2(fmaf(cs.x, a1.x, -cs.y * a0.y), fmaf(cs.x, a1.y, cs.y * a0.x));
    a0 = b0;
    a1 = b1;
}
// shared-memory position of tile-local index tl: 16-byte chunk bits XORed with
// tl bits 5-8 (the groups of consecutive sweeps then hit distinct banks)
__device__ __forceinline__ int qa_swz(int tl) { return tl ^ (((tl >> 5) & 15) << 1); }

// cut(x) = sum over vertices u in x of deg(u) - |N(u) & x|
__device__ __forceinline__ int qa_cut(uint32_t x, const uint32_t *nbr) {
    int c = 0;
    for (uint32_t r = x; r; r &= r - 1) {
        const int u = __ffs(r) - 1;
        c += __popc(nbr[u]) - __popc(x & nbr[u]);
    }
    return c;
}
// counts of x0 | (group bits of j) for j < 32; gbit[m] = index bit of group
// bit m
__device__ __forceinline__ void qa_cut_group(uint32_t x0, const int (&gbit)[5], const uint32_t *nbr, int (&cnt)[32]) {
    cnt[0] = qa_cut(x0, nbr);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const int G = gbit[m];
        const uint32_t nG = nbr[G];
        const int base = __popc(nG) - 2 * __popc(x0 & nG);
        uint32_t adj = 0;   // group-local bits k < m adjacent to G
#pragma unroll
        for (int k = 0; k < m; ++k) adj |= ((nG >> gbit[k]) & 1u) << k;
#pragma unroll
        for (int j = 0; j < (1 << m); ++j) cnt[j | (1 << m)] = cnt[j] + base - 2 * __popc((uint32_t)j & adj);
    }
}

// RX on the group bits in `mask` of a 32-amplitude register group
__device__ __forceinline__ void qa_rx_group(float2 (&a)[32], uint32_t mask, float2 cs) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        if (!((mask >> m) & 1)) continue;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (!((j >> m) & 1)) qa_rx(a[j], a[j | (1 << m)], cs);
    }
}

__device__ double qa_block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kQaoaThreads / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------------------
// n <= 14: the state in shared memory
// ---------------------------------------------------------------------------
__device__ void qaoa_small_item(const QaoaArgs &A, const QaoaItem &I, unsigned char *smq, const float2 *lut,
                                const uint32_t *emask, double *red) {
    float2 *psi = reinterpret_cast<float2 *>(smq);
    unsigned char *cut = smq + kQaoaSmemTile;
    const int tid = threadIdx.x;
    const int n = I.n, ne = I.n_edges, p = A.p;
    const int dim = 1 << n;
    const float amp0 = rsqrtf((float)dim);
    for (int x = tid; x < dim; x += kQaoaThreads) {
        int c = 0;
        for (int e = 0; e < ne; ++e) c += __popc((uint32_t)x & emask[e]) & 1;
        cut[x] = (unsigned char)c;
        psi[x] = make_float2(amp0, 0.f);
    }
    __syncthreads();
    for (int l = 0; l < p; ++l) {
        const float2 *L = lut + l * kQaoaLutStride;
        for (int x = tid; x < dim; x += kQaoaThreads) psi[x] = qa_cmul(psi[x], L[cut[x]]);
        __syncthreads();
        const float2 cs = A.mix[(size_t)I.mix_off + l];
        for (int q = 0; q < n; ++q) {
            for (int w = tid; w < (dim >> 1); w += kQaoaThreads) {
                const int lo = w & ((1 << q) - 1);
                const int x0 = ((w >> q) << (q + 1)) | lo, x1 = x0 | (1 << q);
                float2 a0 = psi[x0], a1 = psi[x1];
                qa_rx(a0, a1, cs);
                psi[x0] = a0;
                psi[x1] = a1;
            }
            __syncthreads();
        }
    }
    double acc = 0.0;
    for (int x = tid; x < dim; x += kQaoaThreads) {
        const float2 v = psi[x];
        acc += (double)(v.x * v.x + v.y * v.y) * (double)cut[x];
    }
    const double s = qa_block_sum(acc, red);
    if (tid == 0) A.out[I.out_idx] = s;
}

// ---------------------------------------------------------------------------
// 14 < n <= 24: the state in the CTA's device-memory slot, streamed in tiles
// ---------------------------------------------------------------------------
// One sweep over a tile of 2^14 amplitudes: this thread's item (9 tile-local
// bits) comes from its thread index through ibit[]; its 32 amplitudes differ in
// the group bits gbl[] (tile-local); rx_mask says which of them get RX (the
// others ride along).
struct QaSweep {
    int gbl[5];
    int ibit[9];
    uint32_t rx_mask;   // group bits that get RX
};

enum QaIo { QA_SMEM = 0, QA_GLOBAL = 1, QA_GEN = 2, QA_EXPECT = 3 };

// tile-local bit b of a pass is index bit b below lb and index bit b + hb from
// lb on (pass A: lb = 14, hb = 0; pass B: lb = 28 - n, hb = n - 14)
template <int SRC, int DST>
__device__ __forceinline__ void qa_item(const QaSweep &S, int item, int lb, int hb, uint32_t tile_base, float2 *tile,
                                        float2 *state, const uint32_t *nbr, float2 cs, const float2 *phase_lut,
                                        float amp0, double &acc) {
    auto ibit_of = [&](int b) { return b < lb ? b : b + hb; };
    int tl0 = 0;
    uint32_t x0 = tile_base;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        if ((item >> k) & 1) {
            tl0 |= 1 << S.ibit[k];
            x0 |= 1u << ibit_of(S.ibit[k]);
        }
    int go[5];        // tile-local offset of each group bit
    uint32_t gm[5];   // index-bit mask of each group bit
    int gidx[5];      // its index bit
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        go[m] = 1 << S.gbl[m];
        gidx[m] = ibit_of(S.gbl[m]);
        gm[m] = 1u << gidx[m];
    }
    auto tl_of = [&](int j) {
        int t = tl0;
#pragma unroll
        for (int m = 0; m < 5; ++m)
            if ((j >> m) & 1) t |= go[m];
        return t;
    };
    auto x_of = [&](int j) {
        uint32_t x = x0;
#pragma unroll
        for (int m = 0; m < 5; ++m)
            if ((j >> m) & 1) x |= gm[m];
        return x;
    };
    float2 a[32];
    if constexpr (SRC == QA_GEN) {
        int cnt[32];
        qa_cut_group(x0, gidx, nbr, cnt);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float2 w = phase_lut[cnt[j]];
            a[j] = make_float2(amp0 * w.x, amp0 * w.y);
        }
    } else if constexpr (SRC == QA_GLOBAL) {
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = state[x_of(j)];
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = tile[qa_swz(tl_of(j))];
    }
    qa_rx_group(a, S.rx_mask, cs);
    if constexpr (DST == QA_SMEM) {
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[qa_swz(tl_of(j))] = a[j];
    } else if constexpr (DST == QA_GLOBAL) {
        if (phase_lut) {
            int cnt[32];
            qa_cut_group(x0, gidx, nbr, cnt);
#pragma unroll
            for (int j = 0; j < 32; ++j) a[j] = qa_cmul(a[j], phase_lut[cnt[j]]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) state[x_of(j)] = a[j];
    } else {   // QA_EXPECT: sum |a|^2 cut(x), nothing stored
        int cnt[32];
        qa_cut_group(x0, gidx, nbr, cnt);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) s = fmaf(fmaf(a[j].x, a[j].x, a[j].y * a[j].y), (float)cnt[j], s);
        acc += (double)s;
    }
}

// the tile's 512 items, two per thread
template <int SRC, int DST>
__device__ __forceinline__ void qa_sweep(const QaSweep &S, int lb, int hb, uint32_t tile_base, float2 *tile,
                                         float2 *state, const uint32_t *nbr, float2 cs, const float2 *phase_lut,
                                         float amp0, double &acc) {
#pragma unroll 1
    for (int item = threadIdx.x; item < (1 << 9); item += kQaoaThreads)
        qa_item<SRC, DST>(S, item, lb, hb, tile_base, tile, state, nbr, cs, phase_lut, amp0, acc);
}

__device__ void qaoa_large_item(const QaoaArgs &A, const QaoaItem &I, float2 *tile, const float2 *lut,
                                const uint32_t *nbr, double *red) {
    const int n = I.n, p = A.p;
    float2 *state = A.slots + (size_t)blockIdx.x * A.slot_elems;
    const float amp0 = rsqrtf((float)(1u << n));
    double acc = 0.0;
    // pass A: tile-local bit b = index bit b; tiles over the bits 14 .. n-1
    // sweeps of pass A: group bits 0-4 (from device memory, pairs contiguous),
    // 5-9, then 10-13 (to device memory; bit 0 rides along as a padding bit)
    const QaSweep A1 = {{0, 1, 2, 3, 4}, {5, 6, 7, 8, 9, 10, 11, 12, 13}, 31u};
    const QaSweep A2 = {{5, 6, 7, 8, 9}, {0, 1, 2, 3, 4, 10, 11, 12, 13}, 31u};
    const QaSweep A3 = {{10, 11, 12, 13, 0}, {1, 2, 3, 4, 5, 6, 7, 8, 9}, 15u};
    // pass B: tile-local bits 0 .. LB-1 = index bits 0 .. LB-1 (rows of 2^LB
    // amplitudes), LB .. 13 = index bits 14 .. n-1; tiles over the index bits
    // LB .. 13
    const int H = n - kQaoaTileBits, LB = kQaoaTileBits - H;
    // group of the first high sweep: tile-local LB .. LB+min(H,5)-1, items the
    // remaining tile-local bits with the low ones first (coalesced rows)
    QaSweep B1, B2;
    {
        // group bits: the sweep's high bits, then (when fewer than 5) the
        // highest of the remaining tile bits as padding; items: the other 9,
        // low bits first (coalesced rows)
        auto build = [&](QaSweep &S, int g0, int h) {
            int rest[kQaoaTileBits], q = 0;
            for (int b = 0; b < kQaoaTileBits; ++b)
                if (b < g0 || b >= g0 + h) rest[q++] = b;
            for (int m = 0; m < 5; ++m) S.gbl[m] = m < h ? g0 + m : rest[--q];
            for (int k = 0; k < 9; ++k) S.ibit[k] = rest[k];   // q == 9 here
            S.rx_mask = (1u << h) - 1;
        };
        const int h1 = H < 5 ? H : 5;
        build(B1, LB, h1);
        build(B2, LB + h1, H - h1);
    }
    const int nA = 1 << H;            // tiles of pass A
    const int nB = 1 << (kQaoaTileBits - LB);   // tiles of pass B (= 2^H)
    for (int l = 0; l < p; ++l) {
        const float2 cs = A.mix[(size_t)I.mix_off + l];
        const float2 *next_phase = l + 1 < p ? lut + (l + 1) * kQaoaLutStride : nullptr;
        for (int t = 0; t < nA; ++t) {
            const uint32_t base = (uint32_t)t << kQaoaTileBits;
            if (l == 0) qa_sweep<QA_GEN, QA_SMEM>(A1, kQaoaTileBits, 0, base, tile, state, nbr, cs, lut, amp0, acc);
            else qa_sweep<QA_GLOBAL, QA_SMEM>(A1, kQaoaTileBits, 0, base, tile, state, nbr, cs, nullptr, amp0, acc);
            __syncthreads();
            qa_sweep<QA_SMEM, QA_SMEM>(A2, kQaoaTileBits, 0, base, tile, state, nbr, cs, nullptr, amp0, acc);
            __syncthreads();
            qa_sweep<QA_SMEM, QA_GLOBAL>(A3, kQaoaTileBits, 0, base, tile, state, nbr, cs, nullptr, amp0, acc);
            __syncthreads();
        }
        __threadfence_block();
        for (int t = 0; t < nB; ++t) {
            const uint32_t base = (uint32_t)t << LB;
            if (H <= 5) {
                if (next_phase) qa_sweep<QA_GLOBAL, QA_GLOBAL>(B1, LB, H, base, tile, state, nbr, cs, next_phase, amp0, acc);
                else qa_sweep<QA_GLOBAL, QA_EXPECT>(B1, LB, H, base, tile, state, nbr, cs, nullptr, amp0, acc);
            } else {
                qa_sweep<QA_GLOBAL, QA_SMEM>(B1, LB, H, base, tile, state, nbr, cs, nullptr, amp0, acc);
                __syncthreads();
                if (next_phase) qa_sweep<QA_SMEM, QA_GLOBAL>(B2, LB, H, base, tile, state, nbr, cs, next_phase, amp0, acc);
                else qa_sweep<QA_SMEM, QA_EXPECT>(B2, LB, H, base, tile, state, nbr, cs, nullptr, amp0, acc);
                __syncthreads();
            }
        }
        __syncthreads();   // pass B's device-memory writes before the next pass A reads them
    }
    const double s = qa_block_sum(acc, red);
    if (threadIdx.x == 0) A.out[I.out_idx] = s;
}

__global__ void __launch_bounds__(kQaoaThreads, 1) qaoa_kernel(const QaoaArgs A) {
    extern __shared__ __align__(16) unsigned char smq[];
    float2 *lut = reinterpret_cast<float2 *>(smq + kQaoaSmemTile + kQaoaSmemCut);
    uint32_t *emask = reinterpret_cast<uint32_t *>(smq + kQaoaSmemTile + kQaoaSmemCut + kQaoaSmemLut);
    uint32_t *nbr = emask + kQaoaMaxEdges;
    __shared__ int s_item;
    __shared__ double s_red[kQaoaThreads / 32];
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) s_item = atomicAdd(A.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= A.n_items) break;
        const QaoaItem I = A.items[it];
        const int ne = I.n_edges;
        for (int e = tid; e < ne; e += kQaoaThreads) emask[e] = A.edge_masks[I.edge_off + e];
        for (int k = tid; k < A.p * (ne + 1); k += kQaoaThreads) {
            const int l = k / (ne + 1), c = k - l * (ne + 1);
            lut[l * kQaoaLutStride + c] = A.luts[(size_t)I.lut_off + k];
        }
        if (tid < I.n) {   // neighbour mask of index bit tid
            uint32_t m = 0;
            for (int e = 0; e < ne; ++e) {
                const uint32_t em = A.edge_masks[I.edge_off + e];
                if ((em >> tid) & 1) m |= em & ~(1u << tid);
            }
            nbr[tid] = m;
        }
        __syncthreads();
        if (I.n <= kQaoaMaxSmallN) qaoa_small_item(A, I, smq, lut, emask, s_red);
        else qaoa_large_item(A, I, reinterpret_cast<float2 *>(smq), lut, nbr, s_red);
        __syncthreads();
    }
}

int qaoa_smem_bytes() { return kQaoaSmemTile + kQaoaSmemCut + kQaoaSmemLut + kQaoaSmemMasks + kQaoaSmemNbr; }

cudaError_t launch_qaoa(const QaoaArgs &A, int grid, cudaStream_t st) {
    const int smem = qaoa_smem_bytes();
    cudaFuncSetAttribute(qaoa_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    qaoa_kernel<<<grid, kQaoaThreads, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace qs
