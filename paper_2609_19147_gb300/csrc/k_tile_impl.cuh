// Tile-pass engine (sm_103a): the kernel template, included by the
// translation units that instantiate it (k_tile_*.cu) so that they compile in
// parallel.
//
// One launch = one full-state HBM pass.  Each persistent CTA walks its tiles.
// A tile is 2^T amplitudes: the L low index bits plus the pass's high bits
// hb[].  It moves HBM <-> shared memory as ONE multi-dimensional TMA tensor
// copy (cp.async.bulk.tensor, 128-byte swizzle): the state is described to the
// TMA unit as a <=5-D tensor whose dims are the low bits, the contiguous runs
// of tile bits and the gaps of non-tile bits between them (the tile selects a
// box of extent 1 in every gap).  When the bit set needs more than 5 dims the
// pass falls back to one bulk copy per 2^L-amplitude row.
//
// Tiles rotate through 1-6 shared buffers: while the warps process tile k,
// the loads of the next tiles and the stores of the previous ones are in
// flight.  Thread 0 issues the copies; the buffer it refills was stored
// NB - D tiles ago (D = tiles loaded ahead), so waiting for that store to
// have read shared memory rarely stalls.  With one buffer (D = 0, two CTAs
// per SM) a tile is loaded once the previous store has read the buffer, and
// the SM's other CTA computes meanwhile.
//
// Passes with dense-block sweeps and passes whose micro-ops are all 1q-layer
// or diagonal ops run in their own instantiations (DENSE, KS), which keeps
// the code and register budget of each kernel small.
//
// Between load and store the tile goes through "sweeps": every compute thread
// holds 2^R amplitudes that differ in R tile bits (registers) and applies the
// sweep's micro-ops: 2x2 / 4x4 unitaries with controls (with cheaper forms for
// real and RX-type matrices), diagonal phase tables (factored into an item part
// and a group part), and QFT stages (Hadamard butterfly + closed-form ladder
// twiddle; Sec. 5.1).  Butterfly normalisations are folded into one scale per
// sweep.  Shared-memory offsets are XOR-linear in the tile bits, which covers
// the swizzled layout.
//
// All waits are bounded; on expiry the kernel records QS_ERR_TIMEOUT, lets its
// own copies land and returns.
#pragma once

#include <cuda.h>

#include <string>

#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: gives up after ~2 s of wall time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && globaltimer() - t0 > 2000000000ull) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst_gmem, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_5d(void *dst_smem, const CUtensorMap *tm, const int c[5], uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]),
        "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap *tm, const int c[5], const void *src_smem) {
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(tm)),
        "r"(smem_u32(src_smem)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4])
        : "memory");
}
__device__ __forceinline__ void tma_prefetch_l2_5d(const CUtensorMap *tm, const int c[5]) {
    asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4])
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}


// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmad(float2 a, float2 b, float2 c) {   // a*b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// exp(i pi u / 2^p) for 0 <= u < 2^p, p <= 32, from the FP64-built roots
__device__ __forceinline__ float2 twiddle(uint64_t u, int p, const float2 *roots) {
    if (p == 0 || u == 0) return make_float2(1.f, 0.f);
    uint32_t v = (uint32_t)(u << (32 - p));
    float2 w = roots[v & 255];
    w = cmul(w, roots[256 + ((v >> 8) & 255)]);
    w = cmul(w, roots[512 + ((v >> 16) & 255)]);
    w = cmul(w, roots[768 + (v >> 24)]);
    return w;
}

// product of the diagonal's slice/group factors selected by the masks
__device__ __forceinline__ float2 diag_part(const DiagDesc &d, uint64_t x, const float2 *cs, uint32_t smask,
                                            uint32_t gmask, float2 ph) {
    for (int s = 0; s < d.n_slices; ++s)
        if ((smask >> s) & 1)
            ph = cmul(ph, cs[d.slice_off[s] + (int)((x >> d.slice_lo[s]) & ((1u << d.slice_w[s]) - 1))]);
    for (int g = 0; g < d.n_groups; ++g)
        if ((gmask >> g) & 1) {
            uint64_t f = d.grp_type[g] ? (x & (x >> d.grp_d[g])) : (x ^ (x >> d.grp_d[g]));
            ph = cmul(ph, cs[d.grp_off[g] + __popcll(f & d.grp_mask[g])]);
        }
    return ph;
}

// ---------------------------------------------------------------------------
// micro-ops on a register group a[0 .. 2^R)
// ---------------------------------------------------------------------------
template <int R>
struct Grp {
    uint64_t gg[R];   // global-index contribution of each group bit
    __device__ __forceinline__ uint64_t gidx(uint64_t base, int j) const {
        uint64_t x = base;
#pragma unroll
        for (int m = 0; m < R; ++m)
            if ((j >> m) & 1) x |= gg[m];
        return x;
    }
};

template <int R, int M>
__device__ __forceinline__ void op_u1(float2 (&a)[1 << R], const float2 *mat, uint64_t cmask, uint64_t cval,
                                      uint64_t base, const Grp<R> &G) {
    const float2 m00 = mat[0], m01 = mat[1], m10 = mat[2], m11 = mat[3];
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        float2 a0 = a[j], a1 = a[k];
        float2 b0 = cmad(m01, a1, cmul(m00, a0));
        float2 b1 = cmad(m11, a1, cmul(m10, a0));
        if (cmask) {
            const bool c = (G.gidx(base, j) & cmask) == cval;
            b0 = c ? b0 : a0;
            b1 = c ? b1 : a1;
        }
        a[j] = b0;
        a[k] = b1;
    }
}

// [[c, i s], [i s, c]] (RX(t): c = cos t/2, s = -sin t/2): 4 FP32 ops per amplitude
template <int R, int M>
__device__ __forceinline__ void op_rxc(float2 (&a)[1 << R], const float2 *cs) {
    const float c = cs[0].x, s = cs[0].y;
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = make_float2(fmaf(c, a0.x, -s * a1.y), fmaf(c, a0.y, s * a1.x));
        a[k] = make_float2(fmaf(c, a1.x, -s * a0.y), fmaf(c, a1.y, s * a0.x));
    }
}

// real 2x2 (RY family): a real factor scales (re, im) alike, so the packed
// FP32x2 pipe does both halves of an amplitude in one instruction (2 per
// amplitude; the same roundings as the scalar FMUL + FFMA)
template <int R, int M>
__device__ __forceinline__ void op_u1r(float2 (&a)[1 << R], const float2 *cs) {
    // the four entries are stored as packed pairs (m, m): no register moves
    const float2 m00 = cs[0], m01 = cs[1];
    const float2 m10 = cs[2], m11 = cs[3];
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = __ffma2_rn(m00, a0, __fmul2_rn(m01, a1));
        a[k] = __ffma2_rn(m10, a0, __fmul2_rn(m11, a1));
    }
}

// real rotation c [[1, t], [-t, 1]] without its factor c (folded into the
// sweep scale): one packed FMA per amplitude, (t, t) and (-t, -t) stored as
// the FP32x2 operands
template <int R, int M>
__device__ __forceinline__ void op_rot(float2 (&a)[1 << R], const float2 *cs) {
    const float2 t = cs[0], nt = cs[1];
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = __ffma2_rn(t, a1, a0);
        a[k] = __ffma2_rn(nt, a0, a1);
    }
}

// unnormalised Hadamard butterfly (the 1/sqrt 2 is folded into the sweep
// scale): one packed add and one packed a0 - a1 (an exact FMA with -1)
template <int R, int M>
__device__ __forceinline__ void op_h(float2 (&a)[1 << R]) {
    const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = __fadd2_rn(a0, a1);
        a[k] = __ffma2_rn(a1, neg1, a0);
    }
}

// QFT stage: butterfly on bit M, then the ladder phase on the bit-M = 1 half:
// item twiddle w times the group-bit twiddle gtab[k].  The group-bit twiddle
// sees only the group bits below M, so the 2^(R-1) products take 2^M distinct
// values, formed once per item.
template <int R, int M>
__device__ __forceinline__ void op_qft(float2 (&a)[1 << R], const float2 *gtab, float2 w) {
    float2 wk[1 << M];
#pragma unroll
    for (int q = 0; q < (1 << M); ++q) wk[q] = cmul(w, gtab[q | (1 << M)]);
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = __fadd2_rn(a0, a1);
        a[k] = cmul(__ffma2_rn(a1, make_float2(-1.f, -1.f), a0), wk[j & ((1 << M) - 1)]);
    }
}

template <int R, int MA, int MB>
__device__ __forceinline__ void op_u2(float2 (&a)[1 << R], const float2 *mat, uint64_t cmask, uint64_t cval,
                                      uint64_t base, const Grp<R> &G) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if (((j >> MA) & 1) || ((j >> MB) & 1)) continue;
        if (cmask && (G.gidx(base, j) & cmask) != cval) continue;   // control bits are never MA/MB
        const int i0 = j, i1 = j | (1 << MB), i2 = j | (1 << MA), i3 = j | (1 << MA) | (1 << MB);
        const float2 v0 = a[i0], v1 = a[i1], v2 = a[i2], v3 = a[i3];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float2 acc = cmul(mat[r * 4 + 0], v0);
            acc = cmad(mat[r * 4 + 1], v1, acc);
            acc = cmad(mat[r * 4 + 2], v2, acc);
            acc = cmad(mat[r * 4 + 3], v3, acc);
            a[r == 0 ? i0 : r == 1 ? i1 : r == 2 ? i2 : i3] = acc;
        }
    }
}

// runtime group bit -> template dispatch
template <int R, int M = 0>
__device__ __forceinline__ void disp_u1(int m, float2 (&a)[1 << R], const float2 *mat, uint64_t cm, uint64_t cv,
                                        uint64_t base, const Grp<R> &G) {
    if constexpr (M < R) {
        if (m == M) op_u1<R, M>(a, mat, cm, cv, base, G);
        else disp_u1<R, M + 1>(m, a, mat, cm, cv, base, G);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void disp_rxc(int m, float2 (&a)[1 << R], const float2 *cs) {
    if constexpr (M < R) {
        if (m == M) op_rxc<R, M>(a, cs);
        else disp_rxc<R, M + 1>(m, a, cs);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void disp_u1r(int m, float2 (&a)[1 << R], const float2 *cs) {
    if constexpr (M < R) {
        if (m == M) op_u1r<R, M>(a, cs);
        else disp_u1r<R, M + 1>(m, a, cs);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void disp_rot(int m, float2 (&a)[1 << R], const float2 *cs) {
    if constexpr (M < R) {
        if (m == M) op_rot<R, M>(a, cs);
        else disp_rot<R, M + 1>(m, a, cs);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void disp_h(int m, float2 (&a)[1 << R]) {
    if constexpr (M < R) {
        if (m == M) op_h<R, M>(a);
        else disp_h<R, M + 1>(m, a);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void disp_qft(int m, float2 (&a)[1 << R], const float2 *gtab, float2 w) {
    if constexpr (M < R) {
        if (m == M) op_qft<R, M>(a, gtab, w);
        else disp_qft<R, M + 1>(m, a, gtab, w);
    }
}
template <int R, int MA, int MB = 0>
__device__ __forceinline__ void disp_u2b(int mb, float2 (&a)[1 << R], const float2 *mat, uint64_t cm, uint64_t cv,
                                         uint64_t base, const Grp<R> &G) {
    if constexpr (MB < R) {
        if constexpr (MB != MA) {
            if (mb == MB) {
                op_u2<R, MA, MB>(a, mat, cm, cv, base, G);
                return;
            }
        }
        disp_u2b<R, MA, MB + 1>(mb, a, mat, cm, cv, base, G);
    }
}
template <int R, int MA = 0>
__device__ __forceinline__ void disp_u2(int ma, int mb, float2 (&a)[1 << R], const float2 *mat, uint64_t cm,
                                        uint64_t cv, uint64_t base, const Grp<R> &G) {
    if constexpr (MA < R) {
        if (ma == MA) disp_u2b<R, MA>(mb, a, mat, cm, cv, base, G);
        else disp_u2<R, MA + 1>(ma, mb, a, mat, cm, cv, base, G);
    }
}

// layers: the same 2x2 family on every group bit in `mask`; the coefficients
// of group bit M sit at k0 + stride * M (RXC 1, U1R 4, U1 4, ROT 2, H none)
template <int KIND>
struct LayerOp;
template <>
struct LayerOp<MK_RXC> {
    template <int R, int M>
    static __device__ __forceinline__ void run(float2 (&a)[1 << R], const float2 *k0, const Grp<R> &) {
        op_rxc<R, M>(a, k0 + M);
    }
};
template <>
struct LayerOp<MK_U1R> {
    template <int R, int M>
    static __device__ __forceinline__ void run(float2 (&a)[1 << R], const float2 *k0, const Grp<R> &) {
        op_u1r<R, M>(a, k0 + 4 * M);
    }
};
template <>
struct LayerOp<MK_U1> {
    template <int R, int M>
    static __device__ __forceinline__ void run(float2 (&a)[1 << R], const float2 *k0, const Grp<R> &G) {
        op_u1<R, M>(a, k0 + 4 * M, 0ull, 0ull, 0ull, G);
    }
};
template <>
struct LayerOp<MK_ROT> {
    template <int R, int M>
    static __device__ __forceinline__ void run(float2 (&a)[1 << R], const float2 *k0, const Grp<R> &) {
        op_rot<R, M>(a, k0 + 2 * M);
    }
};
template <>
struct LayerOp<MK_H> {
    template <int R, int M>
    static __device__ __forceinline__ void run(float2 (&a)[1 << R], const float2 *, const Grp<R> &) {
        op_h<R, M>(a);
    }
};

// runtime mask: one branch per group bit
template <int KIND, int R, int M = 0>
__device__ __forceinline__ void layer_bits(float2 (&a)[1 << R], const float2 *k0, uint32_t mask, const Grp<R> &G) {
    if constexpr (M < R) {
        if ((mask >> M) & 1) LayerOp<KIND>::template run<R, M>(a, k0, G);
        layer_bits<KIND, R, M + 1>(a, k0, mask, G);
    }
}

// compile-time mask: straight-line code over the set bits
template <int KIND, int R, uint32_t MASK, int M = 0>
__device__ __forceinline__ void layer_fixed(float2 (&a)[1 << R], const float2 *k0, const Grp<R> &G) {
    if constexpr (M < R) {
        if constexpr ((MASK >> M) & 1) LayerOp<KIND>::template run<R, M>(a, k0, G);
        layer_fixed<KIND, R, MASK, M + 1>(a, k0, G);
    }
}

template <int R>
__device__ __forceinline__ void run_layer(int kind, float2 (&a)[1 << R], const float2 *k0, uint32_t mask,
                                          const Grp<R> &G) {
    switch (kind) {
        case MK_RXC: layer_bits<MK_RXC, R>(a, k0, mask, G); break;
        case MK_U1R: layer_bits<MK_U1R, R>(a, k0, mask, G); break;
        case MK_U1: layer_bits<MK_U1, R>(a, k0, mask, G); break;
        case MK_ROT: layer_bits<MK_ROT, R>(a, k0, mask, G); break;
        default: layer_bits<MK_H, R>(a, k0, mask, G); break;
    }
}

// QFT stages from the highest group bit down (the gate stream's order)
template <int R, int M = R - 1>
__device__ __forceinline__ void layer_qft(float2 (&a)[1 << R], const float2 *k0, uint32_t mask, uint64_t ppack,
                                          uint64_t gbase, const float2 *roots) {
    if constexpr (M >= 0) {
        if ((mask >> M) & 1) {
            const int p = (int)((ppack >> (6 * M)) & 63);
            const float2 w = twiddle(gbase & ((1ull << p) - 1), p, roots);
            op_qft<R, M>(a, k0 + M * (1 << R), w);
        }
        layer_qft<R, M - 1>(a, k0, mask, ppack, gbase, roots);
    }
}

// ---------------------------------------------------------------------------
// one sweep over the tile in shared memory
// ---------------------------------------------------------------------------
struct SweepCtx {
    int T;
    const int *contrib;      // smem: XOR offset of each tile-local bit (float2 units)
    const int *hb;           // smem: global bit of tile-local bit L + k
    int L;
    float2 *buf;
    const float2 *cs;
    const float2 *roots;
    const MicroOp *micro;    // smem
    const DiagDesc *diags;   // smem
    const int *tab_s;        // smem: per-sweep item-address tables (shared-memory offsets)
    const uint64_t *tab_g;   // smem: per-sweep item-address tables (global index bits)
    uint64_t tile_gbase;     // global index of tile-local 0 (within the state)
    int lt;                  // thread index within the threads that share the sweeps
    uint32_t tmem;           // tensor-memory base of the dense tensor-core sweeps
    uint64_t *mma_bar;       // smem mbarrier their MMAs complete on
    uint32_t *mma_phase;     // smem: its current phase parity
    int n_const;             // constants staged (device checks)
    int tile_elems;          // 2^T (device checks)
    int *err;                // device status word (device checks)
};

#ifdef QS_DEVICE_CHECKS
#define QS_DCHECK(ctx, cond, code) (((cond)) ? true : (atomicCAS((ctx).err, 0, (code)), false))
#else
#define QS_DCHECK(ctx, cond, code) true
#endif

template <int R>
__device__ __forceinline__ void sweep_load(const SweepCtx &c, bool vec, int saddr, const int (&gs)[R],
                                           float2 (&a)[1 << R]) {
    if (vec) {   // group bit 0 = tile-local bit 0: pairs are adjacent and 16-byte aligned
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2) {
            int o = saddr;
#pragma unroll
            for (int m = 1; m < R; ++m)
                if ((j >> m) & 1) o ^= gs[m];
            if (!QS_DCHECK(c, o >= 0 && o + 1 < c.tile_elems && !(o & 1), 1010)) continue;
            const float4 v = *reinterpret_cast<const float4 *>(c.buf + o);
            a[j] = make_float2(v.x, v.y);
            a[j + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            int o = saddr;
#pragma unroll
            for (int m = 0; m < R; ++m)
                if ((j >> m) & 1) o ^= gs[m];
            if (!QS_DCHECK(c, o >= 0 && o < c.tile_elems, 1011)) continue;
            a[j] = c.buf[o];
        }
    }
}

template <int R>
__device__ __forceinline__ void sweep_store(const SweepCtx &c, bool vec, int saddr, const int (&gs)[R],
                                            const float2 (&a)[1 << R]) {
    if (vec) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2) {
            int o = saddr;
#pragma unroll
            for (int m = 1; m < R; ++m)
                if ((j >> m) & 1) o ^= gs[m];
            if (QS_DCHECK(c, o >= 0 && o + 1 < c.tile_elems && !(o & 1), 1012))
                *reinterpret_cast<float4 *>(c.buf + o) = make_float4(a[j].x, a[j].y, a[j + 1].x, a[j + 1].y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            int o = saddr;
#pragma unroll
            for (int m = 0; m < R; ++m)
                if ((j >> m) & 1) o ^= gs[m];
            if (QS_DCHECK(c, o >= 0 && o < c.tile_elems, 1013)) c.buf[o] = a[j];
        }
    }
}

// the item's element offsets, computed once for both the load and the store
template <int R>
__device__ __forceinline__ void group_offsets(int saddr, const int (&gs)[R], int (&o)[1 << R]) {
    o[0] = saddr;
#pragma unroll
    for (int m = 0; m < R; ++m)
#pragma unroll
        for (int j = 0; j < (1 << m); ++j) o[j | (1 << m)] = o[j] ^ gs[m];
}

template <int R>
__device__ __forceinline__ void load_at(const SweepCtx &c, bool vec, const int (&o)[1 << R], float2 (&a)[1 << R]) {
    if (vec) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2) {
            if (!QS_DCHECK(c, o[j] >= 0 && o[j] + 1 < c.tile_elems && !(o[j] & 1), 1001)) {
                a[j] = a[j + 1] = make_float2(0.f, 0.f);
                continue;
            }
            const float4 v = *reinterpret_cast<const float4 *>(c.buf + o[j]);
            a[j] = make_float2(v.x, v.y);
            a[j + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            if (!QS_DCHECK(c, o[j] >= 0 && o[j] < c.tile_elems, 1002)) {
                a[j] = make_float2(0.f, 0.f);
                continue;
            }
            a[j] = c.buf[o[j]];
        }
    }
}

template <int R>
__device__ __forceinline__ void store_at(const SweepCtx &c, bool vec, const int (&o)[1 << R], const float2 (&a)[1 << R]) {
    if (vec) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2)
            if (QS_DCHECK(c, o[j] >= 0 && o[j] + 1 < c.tile_elems && !(o[j] & 1), 1003))
                *reinterpret_cast<float4 *>(c.buf + o[j]) = make_float4(a[j].x, a[j].y, a[j + 1].x, a[j + 1].y);
    } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j)
            if (QS_DCHECK(c, o[j] >= 0 && o[j] < c.tile_elems, 1004)) c.buf[o[j]] = a[j];
    }
}

// 16-byte pairs written as two 8-byte stores (explicit, so that they are not
// merged back): the results of the packed FMAs sit in register pairs, and one
// 16-byte store would first need each two pairs moved into an aligned quad
__device__ __forceinline__ void st_shared_f2(float2 *p, float2 v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(smem_u32(p)), "f"(v.x), "f"(v.y) : "memory");
}
template <int R>
__device__ __forceinline__ void store_at_pairs(const SweepCtx &c, bool vec, const int (&o)[1 << R],
                                               const float2 (&a)[1 << R]) {
    if (vec) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2)
            if (QS_DCHECK(c, o[j] >= 0 && o[j] + 1 < c.tile_elems && !(o[j] & 1), 1003)) {
                st_shared_f2(c.buf + o[j], a[j]);
                st_shared_f2(c.buf + o[j] + 1, a[j + 1]);
            }
    } else {
        store_at<R>(c, false, o, a);
    }
}

// MK_DIAG on a register group: the static factor (slices / LUT groups that do
// not see the group bits) once per item, the rest per amplitude
template <int R>
__device__ __forceinline__ void apply_diag(const SweepCtx &c, const MicroOp &op, uint64_t gbase, const Grp<R> &G,
                                           float2 (&a)[1 << R]) {
    const DiagDesc &d = c.diags[op.cst];
    const uint32_t dyn_s = (uint32_t)op.a, dyn_g = (uint32_t)op.b;
    float2 stat = d.pad0 ? c.cs[d.gph_off] : make_float2(1.f, 0.f);
    stat = diag_part(d, gbase, c.cs, ~dyn_s, ~dyn_g, stat);
    if (dyn_g == 0 && __popc(dyn_s) <= 2 && dyn_s) {
        // fast path: the varying tables' indices are the item's base
        // index OR the group bits' contributions (disjoint bits)
        const int s0 = __ffs(dyn_s) - 1;
        const int s1 = (dyn_s & (dyn_s - 1)) ? __ffs(dyn_s & (dyn_s - 1)) - 1 : -1;
        const uint32_t m0 = (1u << d.slice_w[s0]) - 1;
        const int lo0 = d.slice_lo[s0];
        const float2 *t0 = c.cs + d.slice_off[s0];
        const uint32_t b0 = (uint32_t)(gbase >> lo0) & m0;
        uint32_t q0[R];
#pragma unroll
        for (int m = 0; m < R; ++m) q0[m] = (uint32_t)(G.gg[m] >> lo0) & m0;
        if (s1 < 0) {
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) {
                uint32_t i0 = b0;
#pragma unroll
                for (int m = 0; m < R; ++m)
                    if ((j >> m) & 1) i0 |= q0[m];
                a[j] = cmul(a[j], cmul(stat, t0[i0]));
            }
        } else {
            const uint32_t m1 = (1u << d.slice_w[s1]) - 1;
            const int lo1 = d.slice_lo[s1];
            const float2 *t1 = c.cs + d.slice_off[s1];
            const uint32_t b1 = (uint32_t)(gbase >> lo1) & m1;
            uint32_t q1[R];
#pragma unroll
            for (int m = 0; m < R; ++m) q1[m] = (uint32_t)(G.gg[m] >> lo1) & m1;
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) {
                uint32_t i0 = b0, i1 = b1;
#pragma unroll
                for (int m = 0; m < R; ++m)
                    if ((j >> m) & 1) {
                        i0 |= q0[m];
                        i1 |= q1[m];
                    }
                a[j] = cmul(a[j], cmul(stat, cmul(t0[i0], t1[i1])));
            }
        }
    } else if (dyn_s | dyn_g) {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j)
            a[j] = cmul(a[j], diag_part(d, G.gidx(gbase, j), c.cs, dyn_s, dyn_g, stat));
    } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) a[j] = cmul(a[j], stat);
    }
}

// MK_DIAGQ: the diagonal's tables at the item's base index (group bits 0),
// times Q[j] for the group bits' own terms, times the couplings of each set
// group bit to the other index bits (products built by doubling over the
// group bits: two complex multiplies per amplitude)
template <int R>
__device__ __forceinline__ void apply_diagq(const SweepCtx &c, const MicroOp &op, uint64_t gbase,
                                            float2 (&a)[1 << R]) {
    const DiagDesc &d = c.diags[op.cst];
    float2 z[1 << R];
    z[0] = d.pad0 ? c.cs[d.gph_off] : make_float2(1.f, 0.f);
    z[0] = diag_part(d, gbase, c.cs, ~0u, ~0u, z[0]);
#pragma unroll
    for (int m = 0; m < R; ++m) {
        float2 e = make_float2(1.f, 0.f);
        const int cnt = (int)((op.cmask >> (6 * m)) & 63);
        const float2 *ent = c.cs + op.lo + 2 * m * kMaxCouple;
        for (int k = 0; k < cnt; ++k) {
            const int b = __float_as_int(ent[2 * k].x);
            if ((gbase >> b) & 1) e = cmul(e, ent[2 * k + 1]);
        }
#pragma unroll
        for (int j = 0; j < (1 << m); ++j) z[j | (1 << m)] = cmul(z[j], e);
    }
    const float2 *q = c.cs + op.p;
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) a[j] = cmul(a[j], cmul(z[j], q[j]));
}

// MK_DIAGC: count-indexed phase table.  The item's counts at group bits 0 are
// popcounts (edge distance classes, the single-bit mask); each set group bit
// adds its increment (from its neighbours outside the group and its own
// single-bit term) and the edges inside the group add Qc[j]; the counts are
// built by doubling over the group bits, so each amplitude costs one table
// read and one complex multiply.
template <int R>
__device__ __forceinline__ void apply_diagc(const SweepCtx &c, const MicroOp &op, uint64_t x0,
                                            float2 (&a)[1 << R]) {
    const float2 *lut = c.cs + op.cst;
    const uint64_t *dat = reinterpret_cast<const uint64_t *>(c.cs + op.lo);
    const bool cz = op.b != 0;
    const uint64_t degs = dat[R], mz = dat[R + 1], zinc = dat[R + 2];
    int c0 = op.p * __popcll(x0 & mz);
    for (int k = 0; k < op.a; ++k) {
        const uint64_t m = dat[R + 3 + 2 * k];
        const int d = (int)dat[R + 4 + 2 * k];
        const uint64_t f = cz ? (x0 & (x0 >> d)) : (x0 ^ (x0 >> d));
        c0 += __popcll(f & m);
    }
    int cnt[1 << R];
    cnt[0] = c0;
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const int s = __popcll(x0 & dat[m]);
        const int dm = (cz ? s : (int)((degs >> (6 * m)) & 63) - 2 * s) + (int)((zinc >> (12 * m)) & 4095);
#pragma unroll
        for (int j = 0; j < (1 << m); ++j) cnt[j | (1 << m)] = cnt[j] + dm;
    }
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        const uint64_t qw = j < 16 ? op.cmask : op.cval;
        const int q = (int)((qw >> (4 * (j & 15))) & 15);
        if (!QS_DCHECK(c, cnt[j] + q >= 0 && op.cst + cnt[j] + q < c.n_const, 1009)) continue;
        a[j] = cmul(a[j], lut[cnt[j] + q]);
    }
}

// Kernel op sets: KS_ALL compiles every micro-op kind; KS_LAYER only those of
// 1q-layer and diagonal passes (Trotter / QAOA / random-layer circuits),
// which keeps the code small and the register allocation tight.
constexpr int KS_ALL = 0;
constexpr int KS_LAYER = 1;

// A sweep whose only micro-op is one layer on every group bit (or on all
// but group bit 0, the pair bit of 16-byte accesses) runs as straight-line
// code from load to store: with no control-flow merge between the bits and
// the store, the amplitudes are not moved back into fixed registers after
// each bit.  Code 1 + 2 * (U1, H, RXC, U1R, ROT) + (all but bit 0); 0: the
// general path.  (Sweeps that pair the layer with a diagonal keep the general
// path: the second inlined copy of the diagonal code cost more than the
// merges it saved.)
template <int R>
__device__ __forceinline__ int straight_code(const SweepCtx &c, int op_begin, int op_end, float scale) {
    if ((R != 4 && R != 5) || op_end - op_begin != 1) return 0;
    const MicroOp &o = c.micro[op_begin];
    if (o.kind != MK_LAYER || (o.a != MK_H && o.a != MK_ROT && scale != 1.f)) return 0;
    const uint32_t full = (1u << R) - 1, mask = (uint32_t)o.b;
    if (mask != full && mask != (full & ~1u)) return 0;
    const int ki = o.a == MK_U1 ? 0 : o.a == MK_H ? 1 : o.a == MK_RXC ? 2 : o.a == MK_U1R ? 3 : 4;
    return 1 + 2 * ki + (mask == full ? 0 : 1);
}

template <int KIND, int R, uint32_t MASK>
__device__ __forceinline__ void layer_store(const SweepCtx &c, bool vec, const int (&o)[1 << R],
                                            float2 (&a)[1 << R], const float2 *k0, const Grp<R> &G, float scale) {
    layer_fixed<KIND, R, MASK>(a, k0, G);
    if constexpr (KIND == MK_H || KIND == MK_ROT) {
        if (scale != 1.f) {
            const float2 sc = make_float2(scale, scale);
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) a[j] = __fmul2_rn(a[j], sc);
        }
    }
    store_at<R>(c, vec, o, a);
}

// ---------------------------------------------------------------------------
// Rotation sweep programs (1q-layer / diagonal passes): a sweep whose
// micro-ops are one of
//   1: ROT layer                 2: DIAGC, ROT layer
//   3: ROT layer, DIAGC          4: ROT layer, DIAGC, ROT layer
// with every ROT layer on all R group bits (the planner pads missing bits with
// t = 0, an exact identity) runs a loop specialised for that program: the
// layers' tangents and the diagonal's per-sweep data sit in registers for the
// whole sweep, and no per-item dispatch remains.
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ int rot_program(const SweepCtx &c, int op_begin, int op_end) {
    constexpr int F = (1 << R) - 1;
    auto rot = [&](int i) { return c.micro[i].kind == MK_LAYER && c.micro[i].a == MK_ROT && c.micro[i].b == F; };
    auto dgc = [&](int i) { return c.micro[i].kind == MK_DIAGC; };
    const int n = op_end - op_begin, b = op_begin;
    if (n == 1 && rot(b)) return 1;
    if (n == 2 && dgc(b) && rot(b + 1)) return 2;
    if (n == 2 && rot(b) && dgc(b + 1)) return 3;
    if (n == 3 && rot(b) && dgc(b + 1) && rot(b + 2)) return 4;
    return 0;
}

// the count-table diagonal of one sweep: its op read once per sweep, its
// data (neighbour masks, degrees, classes) read from shared memory per item
// (held in registers it would crowd out the amplitudes)
template <int R>
struct DiagcRegs {
    const char *lut;   // the count table, addressed in bytes
    const uint64_t *dat;
    int n_cls, stride;
    bool cz;
    int s8;                       // 8 x the weight of a neighbour count (+1 both-set, -2 mismatch)
    int base8[R];                 // 8 x each group bit's increment without its neighbour term
    uint32_t q8[(1 << R) / 4];    // 8 x the intra-group entry of element j, one byte per element
#ifdef QS_DEVICE_CHECKS
    const SweepCtx *ctx;
#endif
    __device__ __forceinline__ void init(const SweepCtx &c, const MicroOp &op) {
#ifdef QS_DEVICE_CHECKS
        ctx = &c;
        QS_DCHECK(c, op.cst >= 0 && op.lo >= 0 && op.lo + R + 3 + 2 * op.a <= c.n_const, 1005);
#endif
        lut = reinterpret_cast<const char *>(c.cs + op.cst);
        dat = reinterpret_cast<const uint64_t *>(c.cs + op.lo);
        n_cls = op.a;
        stride = op.p;
        cz = op.b != 0;
        s8 = cz ? 8 : -16;
        const uint64_t degs = dat[R], zinc = dat[R + 2];
#pragma unroll
        for (int m = 0; m < R; ++m)
            base8[m] = 8 * ((cz ? 0 : (int)((degs >> (6 * m)) & 63)) + (int)((zinc >> (12 * m)) & 4095));
#pragma unroll
        for (int w = 0; w < (1 << R) / 4; ++w) {
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = 4 * w + b;
                const uint32_t q = (uint32_t)(((j < 16 ? op.cmask : op.cval) >> (4 * (j & 15))) & 15);
                v |= (8u * q) << (8 * b);
            }
            q8[w] = v;
        }
    }
    __device__ __forceinline__ void apply(uint64_t x0, float2 (&a)[1 << R]) const {
        const uint64_t mz = dat[R + 1];
        const uint64_t *cls = dat + R + 3;
        int c0 = stride * __popcll(x0 & mz);
        for (int k = 0; k < n_cls; ++k) {
            const uint64_t f = cz ? (x0 & (x0 >> (int)cls[2 * k + 1])) : (x0 ^ (x0 >> (int)cls[2 * k + 1]));
            c0 += __popcll(f & cls[2 * k]);
        }
        int dm8[R];
#pragma unroll
        for (int m = 0; m < R; ++m) dm8[m] = base8[m] + s8 * __popcll(x0 & dat[m]);
        // the group elements in Gray-code order: one running byte offset, one
        // add or subtract per element, plus the element's intra-group entry
        int off = 8 * c0;
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) {
            const int j = i ^ (i >> 1);
            if (i > 0) {
                const int m = __ffs(i) - 1;
                off += ((j >> m) & 1) ? dm8[m] : -dm8[m];
            }
            const int o = off + (int)__byte_perm(q8[j >> 2], 0u, 0x4440u | (uint32_t)(j & 3));
#ifdef QS_DEVICE_CHECKS
            if (!QS_DCHECK(*ctx, o >= 0 && (lut - reinterpret_cast<const char *>(ctx->cs)) + o + 8 <=
                                               8LL * ctx->n_const, 1006))
                continue;
#endif
            a[j] = cmul(a[j], *reinterpret_cast<const float2 *>(lut + o));
        }
    }
};

// a ROT layer on the group bits in MASK with the tangents in registers (the
// other group bits carry t = 0: identities, skipped)
template <int R, uint32_t MASK = (1u << R) - 1, int M = 0>
__device__ __forceinline__ void rot_layer_regs(float2 (&a)[1 << R], const float2 (&t)[R]) {
    if constexpr (M < R && !((MASK >> M) & 1)) {
        rot_layer_regs<R, MASK, M + 1>(a, t);
    } else if constexpr (M < R) {
        const float2 tp = t[M], tn = make_float2(-t[M].x, -t[M].y);
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            if ((j >> M) & 1) continue;
            const int k = j | (1 << M);
            const float2 a0 = a[j], a1 = a[k];
            a[j] = __ffma2_rn(tp, a1, a0);
            a[k] = __ffma2_rn(tn, a0, a1);
        }
        rot_layer_regs<R, MASK, M + 1>(a, t);
    }
}

template <int R, int NT, int PROG, bool VEC, bool SCALED, uint32_t MASK1 = (1u << R) - 1>
__device__ __forceinline__ void rot_sweep(const SweepCtx &c, const Sweep &S, int sidx) {
    const int *ts = c.tab_s + sidx * kItemTab;
    const uint64_t *tg = c.tab_g + sidx * kItemTab;
    int gs[R];
#pragma unroll
    for (int m = 0; m < R; ++m) gs[m] = ts[kItemTab - kGroupTab + m];
    const int b = S.op_begin;
    const int i_l1 = PROG == 2 ? b + 1 : b;
    float2 t1[R], t2[R];
    (void)QS_DCHECK(c, c.micro[i_l1].cst >= 0 && c.micro[i_l1].cst + 2 * R <= c.n_const, 1007);
    if constexpr (PROG == 4)
        (void)QS_DCHECK(c, c.micro[b + 2].cst >= 0 && c.micro[b + 2].cst + 2 * R <= c.n_const, 1008);
#pragma unroll
    for (int m = 0; m < R; ++m) t1[m] = c.cs[c.micro[i_l1].cst + 2 * m];
    if constexpr (PROG == 4) {
#pragma unroll
        for (int m = 0; m < R; ++m) t2[m] = c.cs[c.micro[b + 2].cst + 2 * m];
    }
    DiagcRegs<R> dg;
    if constexpr (PROG >= 2) dg.init(c, c.micro[PROG == 2 ? b : b + 1]);
    const float2 sc = make_float2(S.scale, S.scale);
    const int n_items = 1 << (c.T - R);
    for (int item = c.lt; item < n_items; item += NT) {
        const int i0 = item & 31, i1 = 32 + ((item >> 5) & 31), i2 = 64 + ((item >> 10) & 15);
        const int saddr = ts[i0] ^ ts[i1] ^ ts[i2];
        float2 a[1 << R];
        int o[1 << R];
        group_offsets<R>(saddr, gs, o);
        load_at<R>(c, VEC, o, a);
        uint64_t x0 = 0;
        if constexpr (PROG >= 2) x0 = c.tile_gbase | tg[i0] | tg[i1] | tg[i2];
        if constexpr (PROG == 2) dg.apply(x0, a);
        rot_layer_regs<R, MASK1>(a, t1);
        if constexpr (PROG == 3 || PROG == 4) dg.apply(x0, a);
        if constexpr (PROG == 4) rot_layer_regs<R>(a, t2);
        if constexpr (SCALED) {
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) a[j] = __fmul2_rn(a[j], sc);
        }
        // with 4-bit groups (112 registers) the offsets are formed again
        // rather than held through the ops
        if constexpr (R == 4) group_offsets<R>(saddr, gs, o);
        store_at_pairs<R>(c, VEC, o, a);
    }
}

template <int R, int NT, int PROG, bool VEC, bool SCALED, bool MASKED>
__device__ __forceinline__ void rot_sweep_masked(const SweepCtx &c, const Sweep &S, int sidx, int mc) {
    constexpr uint32_t F = (1u << R) - 1;
    if constexpr (!MASKED) {
        rot_sweep<R, NT, PROG, VEC, SCALED, F>(c, S, sidx);
        return;
    }
    if (mc == 1) rot_sweep<R, NT, PROG, VEC, SCALED, 7u>(c, S, sidx);
    else if (mc == 2) rot_sweep<R, NT, PROG, VEC, SCALED, F & ~1u>(c, S, sidx);
    else if (R == 5 && mc == 3) rot_sweep<R, NT, PROG, VEC, SCALED, 0xfu & F>(c, S, sidx);
    else if (R == 5 && mc == 4) rot_sweep<R, NT, PROG, VEC, SCALED, 0xeu & F>(c, S, sidx);
    else rot_sweep<R, NT, PROG, VEC, SCALED, F>(c, S, sidx);
}

// MASKED: instantiate the programs whose first layer skips padded identities
// (the warp-specialised kernel; the others keep one form per program)
template <int R, int NT, bool MASKED>
__device__ __forceinline__ bool run_rot_program(const SweepCtx &c, const Sweep &S, int sidx) {
    const int prog = rot_program<R>(c, S.op_begin, S.op_end);
    if (!prog) return false;
    // the first layer's own bits: the lowest three or four group positions,
    // or those above position 0, run without the padded identities
    // (programs 1 and 4)
    constexpr uint32_t F = (1u << R) - 1;
    const uint32_t own = (uint32_t)c.micro[prog == 2 ? S.op_begin + 1 : S.op_begin].lo & F;
    const int mc = (!MASKED || (prog != 1 && prog != 4)) ? 0
                   : own == 7u            ? 1
                   : own == (F & ~1u)     ? 2
                   : (R == 5 && own == 0xfu) ? 3
                   : (R == 5 && own == 0xeu) ? 4
                                             : 0;
    const int k = 4 * (prog - 1) + (S.vec ? 2 : 0) + (S.scale != 1.f ? 1 : 0);
    switch (k) {
        case 0: rot_sweep_masked<R, NT, 1, false, false, MASKED>(c, S, sidx, mc); break;
        case 1: rot_sweep_masked<R, NT, 1, false, true, MASKED>(c, S, sidx, mc); break;
        case 2: rot_sweep_masked<R, NT, 1, true, false, MASKED>(c, S, sidx, mc); break;
        case 3: rot_sweep_masked<R, NT, 1, true, true, MASKED>(c, S, sidx, mc); break;
        case 4: rot_sweep<R, NT, 2, false, false>(c, S, sidx); break;
        case 5: rot_sweep<R, NT, 2, false, true>(c, S, sidx); break;
        case 6: rot_sweep<R, NT, 2, true, false>(c, S, sidx); break;
        case 7: rot_sweep<R, NT, 2, true, true>(c, S, sidx); break;
        case 8: rot_sweep<R, NT, 3, false, false>(c, S, sidx); break;
        case 9: rot_sweep<R, NT, 3, false, true>(c, S, sidx); break;
        case 10: rot_sweep<R, NT, 3, true, false>(c, S, sidx); break;
        case 11: rot_sweep<R, NT, 3, true, true>(c, S, sidx); break;
        case 12: rot_sweep_masked<R, NT, 4, false, false, MASKED>(c, S, sidx, mc); break;
        case 13: rot_sweep_masked<R, NT, 4, false, true, MASKED>(c, S, sidx, mc); break;
        case 14: rot_sweep_masked<R, NT, 4, true, false, MASKED>(c, S, sidx, mc); break;
        default: rot_sweep_masked<R, NT, 4, true, true, MASKED>(c, S, sidx, mc); break;
    }
    return true;
}

// ---------------------------------------------------------------------------
// U(2) layer sweeps (MK_ZYZ): every group bit's 2x2 unitary was factored on the
// host into output phases, a real rotation and input phases.  Per item: one
// product with the input-phase table (the phases of all R bits at once), R
// rotation layers at one packed FMA per amplitude and bit, one product with
// the output-phase table.  A bit whose rotation ran in cotangent form leaves
// its pair exchanged; the store undoes the exchange by writing to the
// exchanged offsets (an XOR of the group bits' offsets, formed once per sweep),
// and the planner stored the output-phase table in the exchanged order.
// ---------------------------------------------------------------------------
template <int R, int M = 0>
__device__ __forceinline__ void zyz_rot_regs(float2 (&a)[1 << R], const float2 (&k)[2 * R]) {
    if constexpr (M < R) {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            if ((j >> M) & 1) continue;
            const int q = j | (1 << M);
            const float2 a0 = a[j], a1 = a[q];
            a[j] = __ffma2_rn(k[2 * M], a1, a0);
            a[q] = __ffma2_rn(k[2 * M + 1], a0, a1);
        }
        zyz_rot_regs<R, M + 1>(a, k);
    }
}

// the general path's form (the sweep's last op, after others): the exchange is
// left to the store (zyz_exchange); as any other op it is undone in registers
template <int R>
__device__ __forceinline__ void apply_zyz(const SweepCtx &c, const MicroOp &op, float2 (&a)[1 << R], bool last) {
    constexpr int P = 1 << R;
    if (!QS_DCHECK(c, op.cst >= 0 && op.cst + 2 * P + 2 * R + 1 <= c.n_const, 1014)) return;
    const float2 *pin = c.cs + op.cst, *pout = pin + P, *kk = pout + P;
    float2 k[2 * R];
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) k[m] = kk[m];
    const int form = __float_as_int(kk[2 * R].x);
#pragma unroll
    for (int j = 1; j < P; ++j) a[j] = cmul(a[j], pin[j]);
    zyz_rot_regs<R>(a, k);
#pragma unroll
    for (int j = 0; j < P; ++j) a[j] = cmul(a[j], pout[j]);
    if (last) return;
#pragma unroll
    for (int m = 0; m < R; ++m) {
        if (!((form >> m) & 1)) continue;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if ((j >> m) & 1) continue;
            const float2 t = a[j];
            a[j] = a[j | (1 << m)];
            a[j | (1 << m)] = t;
        }
    }
}

// a sweep that ends with MK_ZYZ: its store goes to the exchanged offsets,
// item base saddr ^ fo (fo over the group bits in the form mask, bit 0 left
// out with 16-byte pairs), and with the pair bit exchanged (sw0) it swaps the
// two halves of each 16-byte store
template <int R>
__device__ __forceinline__ void zyz_exchange(const SweepCtx &c, const Sweep &S, const int (&gs)[R], int &fo,
                                             bool &sw0) {
    fo = 0;
    sw0 = false;
    if (S.op_end <= S.op_begin) return;
    const MicroOp &op = c.micro[S.op_end - 1];
    if (op.kind != MK_ZYZ) return;
    if (!QS_DCHECK(c, op.cst >= 0 && op.cst + 2 * (1 << R) + 2 * R + 1 <= c.n_const, 1014)) return;
    const int form = __float_as_int(c.cs[op.cst + 2 * (1 << R) + 2 * R].x);
#pragma unroll
    for (int m = 0; m < R; ++m)
        if (((form >> m) & 1) && !(m == 0 && S.vec)) fo ^= gs[m];
    sw0 = S.vec && (form & 1);
}

template <int R, int NT, bool VEC, bool SW0>
__device__ __forceinline__ void zyz_sweep(const SweepCtx &c, const Sweep &S, int sidx, const MicroOp &op) {
    constexpr int P = 1 << R;
    const int *ts = c.tab_s + sidx * kItemTab;
    int gs[R];
#pragma unroll
    for (int m = 0; m < R; ++m) gs[m] = ts[kItemTab - kGroupTab + m];
    const float2 *pin = c.cs + op.cst, *pout = pin + P, *kk = pout + P;
    float2 k[2 * R];
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) k[m] = kk[m];
    const int form = __float_as_int(kk[2 * R].x);
    // offset XOR that moves element i to element i ^ form (with 16-byte pairs,
    // bit 0 is the swap inside the pair: SW0)
    int fo = 0;
#pragma unroll
    for (int m = VEC ? 1 : 0; m < R; ++m)
        if ((form >> m) & 1) fo ^= gs[m];
    const int n_items = 1 << (c.T - R);
    for (int item = c.lt; item < n_items; item += NT) {
        const int i0 = item & 31, i1 = 32 + ((item >> 5) & 31), i2 = 64 + ((item >> 10) & 15);
        const int saddr = ts[i0] ^ ts[i1] ^ ts[i2];
        float2 a[P];
        int o[P];
        group_offsets<R>(saddr, gs, o);
        load_at<R>(c, VEC, o, a);
#pragma unroll
        for (int j = 1; j < P; ++j) a[j] = cmul(a[j], pin[j]);
        zyz_rot_regs<R>(a, k);
#pragma unroll
        for (int j = 0; j < P; ++j) a[j] = cmul(a[j], pout[j]);
        // a[i] is element i ^ form: its offset is that of element i from the
        // item base saddr ^ fo
        group_offsets<R>(saddr ^ fo, gs, o);
        if constexpr (VEC) {
#pragma unroll
            for (int j = 0; j < P; j += 2)
                if (QS_DCHECK(c, o[j] >= 0 && o[j] + 1 < c.tile_elems && !(o[j] & 1), 1015)) {
                    const float2 lo = SW0 ? a[j + 1] : a[j], hi = SW0 ? a[j] : a[j + 1];
                    *reinterpret_cast<float4 *>(c.buf + o[j]) = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
        } else {
#pragma unroll
            for (int j = 0; j < P; ++j)
                if (QS_DCHECK(c, o[j] >= 0 && o[j] < c.tile_elems, 1015)) c.buf[o[j]] = a[j];
        }
    }
}

template <int R, int NT>
__device__ __forceinline__ bool run_zyz_program(const SweepCtx &c, const Sweep &S, int sidx) {
    if (S.op_end - S.op_begin != 1 || S.scale != 1.f) return false;
    const MicroOp &op = c.micro[S.op_begin];
    if (op.kind != MK_ZYZ) return false;
    if (!QS_DCHECK(c, op.cst >= 0 && op.cst + 2 * (1 << R) + 2 * R + 1 <= c.n_const, 1014)) return true;
    const bool sw0 = (__float_as_int(c.cs[op.cst + 2 * (1 << R) + 2 * R].x) & 1) != 0;
    if (!S.vec) zyz_sweep<R, NT, false, false>(c, S, sidx, op);
    else if (!sw0) zyz_sweep<R, NT, true, false>(c, S, sidx, op);
    else zyz_sweep<R, NT, true, true>(c, S, sidx, op);
    return true;
}

template <int R, int NT, int KS>
__device__ __forceinline__ void run_sweep_general(const SweepCtx &c, const Sweep &S, int sidx) {
    const int *ts = c.tab_s + sidx * kItemTab;
    const uint64_t *tg = c.tab_g + sidx * kItemTab;
    int gs[R];
    Grp<R> G0;   // global-index bit of each group bit (read by controlled ops and diagonals)
#pragma unroll
    for (int m = 0; m < R; ++m) {
        gs[m] = ts[kItemTab - kGroupTab + m];
        G0.gg[m] = KS == KS_LAYER ? 0ull : tg[kItemTab - kGroupTab + m];
    }
    const int nb = c.T - R;
    const int n_items = 1 << nb;
    const bool vec = S.vec != 0;
    const int op_begin = S.op_begin, op_end = S.op_end;
    const float scale = S.scale;
    const int fast = KS == KS_LAYER ? straight_code<R>(c, op_begin, op_end, scale) : 0;
    const float2 *k0f = c.cs + c.micro[op_begin].cst;
    int zfo;
    bool zsw0;
    zyz_exchange<R>(c, S, gs, zfo, zsw0);
    for (int item = c.lt; item < n_items; item += NT) {
        const int i0 = item & 31, i1 = 32 + ((item >> 5) & 31), i2 = 64 + ((item >> 10) & 15);
        const int saddr = ts[i0] ^ ts[i1] ^ ts[i2];
        // global index of the item's group element 0 (only ops with controls,
        // diagonals and QFT twiddles read it)
        auto gbase = [&]() { return c.tile_gbase | tg[i0] | tg[i1] | tg[i2]; };
        float2 a[1 << R];
        Grp<R> G = G0;
        if constexpr ((R == 4 || R == 5) && KS == KS_LAYER) {
            if (fast) {
                int o[1 << R];
                group_offsets<R>(saddr, gs, o);
                load_at<R>(c, vec, o, a);
                constexpr uint32_t F = (1u << R) - 1, HI = F & ~1u;
                switch (fast) {
                    case 1: layer_store<MK_U1, R, F>(c, vec, o, a, k0f, G, scale); break;
                    case 2: layer_store<MK_U1, R, HI>(c, vec, o, a, k0f, G, scale); break;
                    case 3: layer_store<MK_H, R, F>(c, vec, o, a, k0f, G, scale); break;
                    case 4: layer_store<MK_H, R, HI>(c, vec, o, a, k0f, G, scale); break;
                    case 5: layer_store<MK_RXC, R, F>(c, vec, o, a, k0f, G, scale); break;
                    case 6: layer_store<MK_RXC, R, HI>(c, vec, o, a, k0f, G, scale); break;
                    case 7: layer_store<MK_U1R, R, F>(c, vec, o, a, k0f, G, scale); break;
                    case 8: layer_store<MK_U1R, R, HI>(c, vec, o, a, k0f, G, scale); break;
                    case 9: layer_store<MK_ROT, R, F>(c, vec, o, a, k0f, G, scale); break;
                    default: layer_store<MK_ROT, R, HI>(c, vec, o, a, k0f, G, scale); break;
                }
                continue;
            }
        }
        if constexpr (KS == KS_LAYER) {
            // loaded here: the straight-line layers above never read them
#pragma unroll
            for (int m = 0; m < R; ++m) G.gg[m] = tg[kItemTab - kGroupTab + m];
        }
        sweep_load<R>(c, vec, saddr, gs, a);
        for (int oi = op_begin; oi < op_end; ++oi) {
            const MicroOp &op = c.micro[oi];
            if constexpr (KS == KS_LAYER) {
                switch (op.kind) {
                    case MK_LAYER: run_layer<R>(op.a, a, c.cs + op.cst, (uint32_t)op.b, G); break;
                    case MK_RXC: disp_rxc<R>(op.a, a, c.cs + op.cst); break;
                    case MK_U1R: disp_u1r<R>(op.a, a, c.cs + op.cst); break;
                    case MK_ROT: disp_rot<R>(op.a, a, c.cs + op.cst); break;
                    case MK_H: disp_h<R>(op.a, a); break;
                    case MK_U1: disp_u1<R>(op.a, a, c.cs + op.cst, op.cmask, op.cval, gbase(), G); break;
                    case MK_DIAG: apply_diag<R>(c, op, gbase(), G, a); break;
                    case MK_DIAGQ: apply_diagq<R>(c, op, gbase(), a); break;
                    case MK_DIAGC: apply_diagc<R>(c, op, gbase(), a); break;
                    case MK_ZYZ: apply_zyz<R>(c, op, a, oi == op_end - 1); break;
                    default: break;
                }
            } else {
                switch (op.kind) {
                    case MK_U1:
                        disp_u1<R>(op.a, a, c.cs + op.cst, op.cmask, op.cval, gbase(), G);
                        break;
                    case MK_H:
                        disp_h<R>(op.a, a);
                        break;
                    case MK_RXC:
                        disp_rxc<R>(op.a, a, c.cs + op.cst);
                        break;
                    case MK_U1R:
                        disp_u1r<R>(op.a, a, c.cs + op.cst);
                        break;
                    case MK_ROT:
                        disp_rot<R>(op.a, a, c.cs + op.cst);
                        break;
                    case MK_U2:
                        disp_u2<R>(op.a, op.b, a, c.cs + op.cst, op.cmask, op.cval, gbase(), G);
                        break;
                    case MK_QFT: {
                        const uint64_t Mk = (op.p > op.lo) ? (((1ull << op.p) - 1) & ~((1ull << op.lo) - 1)) : 0ull;
                        const float2 w = twiddle(gbase() & Mk, op.p, c.roots);
                        disp_qft<R>(op.a, a, c.cs + op.cst, w);
                        break;
                    }
                    case MK_LAYER: run_layer<R>(op.a, a, c.cs + op.cst, (uint32_t)op.b, G); break;
                    case MK_QFTL:
                        layer_qft<R>(a, c.cs + op.cst, (uint32_t)op.b, op.cmask, gbase(), c.roots);
                        break;
                    case MK_DIAG:
                        apply_diag<R>(c, op, gbase(), G, a);
                        break;
                    case MK_DIAGQ:
                        apply_diagq<R>(c, op, gbase(), a);
                        break;
                    case MK_DIAGC:
                        apply_diagc<R>(c, op, gbase(), a);
                        break;
                    case MK_ZYZ:
                        apply_zyz<R>(c, op, a, oi == op_end - 1);
                        break;
                    default:
                        break;
                }
            }
        }
        if (scale != 1.f) {
            const float2 sc = make_float2(scale, scale);
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) a[j] = __fmul2_rn(a[j], sc);
        }
        if (zsw0) {
#pragma unroll
            for (int j = 0; j < (1 << R); j += 2) {
                const float2 t = a[j];
                a[j] = a[j + 1];
                a[j + 1] = t;
            }
        }
        sweep_store<R>(c, vec, saddr ^ zfo, gs, a);
    }
}

template <int R, int NT, int KS = KS_ALL, bool WS = false>
__device__ __forceinline__ void run_sweep(const SweepCtx &c, const Sweep &S, int sidx) {
    if constexpr ((R == 4 || R == 5) && KS == KS_LAYER) {
        if (run_rot_program<R, NT, WS>(c, S, sidx)) return;
        if (run_zyz_program<R, NT>(c, S, sidx)) return;
    }
    run_sweep_general<R, NT, KS>(c, S, sidx);
}

// ---------------------------------------------------------------------------
// dense-block sweeps: out = U X, X = the tile as a 32 x 2^(T-5) matrix (row =
// the sweep's 5 group bits, column = its item bits), in place
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dense_coloff(const int *ts, int m) {
    return ts[m & 31] ^ ts[32 + ((m >> 5) & 31)] ^ ts[64 + ((m >> 10) & 15)];
}
// shared-memory offset of block row r: XOR of the group bits' offsets
__device__ __forceinline__ int dense_rowoff(const int (&g)[5], int r) {
    int o = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if ((r >> q) & 1) o ^= g[q];
    return o;
}

// FP32 on the CUDA cores: a thread owns whole columns (32 amplitudes in
// registers); rows of U are read as broadcasts from shared memory
template <int NT>
__device__ __forceinline__ void dense_fp32(const SweepCtx &c, const Sweep &S, int sidx) {
    int g[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) g[q] = c.contrib[S.gbit[q]];
    const int ncols = 1 << (c.T - 5);
    const int *ts = c.tab_s + sidx * kItemTab;
    const float4 *U = reinterpret_cast<const float4 *>(c.cs + S.dcst);
    for (int m = c.lt; m < ncols; m += NT) {
        const int co = dense_coloff(ts, m);
        float2 x[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = c.buf[co ^ dense_rowoff(g, r)];
#pragma unroll 1
        for (int i = 0; i < 32; i += 4) {
            float2 y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) y[e] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4 u = U[((i + e) * 32 + j) >> 1];
                    y[e] = cmad(make_float2(u.x, u.y), x[j], y[e]);
                    y[e] = cmad(make_float2(u.z, u.w), x[j + 1], y[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) c.buf[co ^ dense_rowoff(g, i + e)] = y[e];
        }
    }
}

// x rounded to TF32 (10 explicit mantissa bits, ties away from zero) with
// integer operations; x - hi is then exact in FP32
__device__ __forceinline__ uint32_t tf32_hi(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// (re, im) -> packed BF16 pair, re in the low half
__device__ __forceinline__ uint32_t pack_bf16(float2 v) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(v.y), "f"(v.x));
    return r;
}

// Tensor cores in BF16 (m16n8k16): k = 2 * block row + (re, im) over rows
// 8s..8s+7; U's operand registers come pre-packed from the host.
template <int MT, int NT>
__device__ __forceinline__ void dense_bf16(const SweepCtx &c, const Sweep &S, int sidx) {
    const int lane = c.lt & 31, warp = c.lt >> 5;
    const int q = lane & 3, gq = lane >> 2;
    const int rlo = ((q & 1) ? c.contrib[S.gbit[0]] : 0) ^ ((q & 2) ? c.contrib[S.gbit[1]] : 0);
    const int g2 = c.contrib[S.gbit[2]], g3 = c.contrib[S.gbit[3]], g4 = c.contrib[S.gbit[4]];
    int rhi[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) rhi[s] = ((s & 1) ? g2 : 0) ^ ((s & 2) ? g3 : 0) ^ ((s & 4) ? g4 : 0);
    const uint2 *B = reinterpret_cast<const uint2 *>(c.cs + S.dcst) + lane;
    const int ncols = 1 << (c.T - 5);
    const int *ts = c.tab_s + sidx * kItemTab;
    for (int mb = warp * 16 * MT; mb < ncols; mb += (NT / 32) * 16 * MT) {
        int co[MT][2];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            co[mt][0] = dense_coloff(ts, mb + 16 * mt + gq) ^ rlo;
            co[mt][1] = dense_coloff(ts, mb + 16 * mt + gq + 8) ^ rlo;
        }
        float acc[MT][8][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int t = 0; t < 8; ++t)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][t][e] = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            uint32_t a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                // rows 8s + q (block-row bit 2 clear) and 8s + 4 + q (set)
                a[mt][0] = pack_bf16(c.buf[rhi[2 * s] ^ co[mt][0]]);
                a[mt][1] = pack_bf16(c.buf[rhi[2 * s] ^ co[mt][1]]);
                a[mt][2] = pack_bf16(c.buf[rhi[2 * s + 1] ^ co[mt][0]]);
                a[mt][3] = pack_bf16(c.buf[rhi[2 * s + 1] ^ co[mt][1]]);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const uint2 b = B[(s * 8 + t) * 32];
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) mma_bf16(acc[mt][t], a[mt], b.x, b.y);
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                if (mb + 16 * mt + gq < ncols) c.buf[rhi[t] ^ co[mt][0]] = make_float2(acc[mt][t][0], acc[mt][t][1]);
                if (mb + 16 * mt + gq + 8 < ncols) c.buf[rhi[t] ^ co[mt][1]] = make_float2(acc[mt][t][2], acc[mt][t][3]);
            }
    }
}

// ---------------------------------------------------------------------------
// 3xTF32 dense blocks on the fifth-generation tensor cores (tcgen05)
//
// The block's 32 x 32 complex matrix U times the tile viewed as X, 32 rows (the
// block's 5 group bits) by up to 256 columns (the item bits).  Thread m (of
// 256) gathers column m from shared memory at the sweep's XOR offsets (any
// five tile bits), splits each real and imaginary part into TF32 hi + lo
// (round to nearest) and writes them into tensor memory as the MMA's A
// operand, row m: columns [0, 32) hi re, [32, 64) hi im, [64, 96) lo re,
// [96, 128) lo im, 256 columns per M-tile of 128 rows.  B is U's real and
// imaginary parts (hi and lo, TF32-rounded on the host from FP64), each a
// 32 x 32 K-major matrix in shared memory with the 128-byte swizzle.  One
// thread issues, per M-tile and K-step of 8,
//   Dre += Xre Ure - Xim Uim,   Dim += Xre Uim + Xim Ure
// (the minus sign through the descriptor's negate-B bit), the hi x hi products
// into one pair of accumulators and the two small cross terms (lo x hi, hi x
// lo) into another: the tensor core's FP32 accumulation truncates, so chaining
// the small terms onto the large sum would bias the result toward zero.  The
// accumulators (FP32, in tensor memory) come back with tcgen05.ld, are added
// and stored to the same positions of the tile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 1024-byte
// atoms of 8 rows x 128 bytes (stride 1024 bytes), version 1
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// N and M, optional negation of B
__device__ __forceinline__ constexpr uint32_t tc_idesc_tf32(int M, int N, bool neg_b) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_b ? 1u : 0u) << 14) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
constexpr int kTmemCols = 512;   // two M-tiles x (A hi, A lo, D main, D cross) x (re, im) x 32

// returns false (on every thread) when the MMAs did not complete in time
template <int NT>
__device__ __forceinline__ bool dense_tc_tf32x3(const SweepCtx &c, const Sweep &S, int sidx) {
    static_assert(NT == 256, "two warpgroups: one per M-tile of 128 columns");
    const int m = c.lt, warp = m >> 5, mt = m >> 7;
    const int ncols = 1 << (c.T - 5);
    const int *ts = c.tab_s + sidx * kItemTab;
    int g[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) g[q] = c.contrib[S.gbit[q]];
    const bool mine = m < ncols;
    const int co = mine ? dense_coloff(ts, m) : 0;
    const uint32_t lane_col = c.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * mt);
    {
        uint32_t hr[32], hi[32], lr[32], li[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const float2 x = mine ? c.buf[co ^ dense_rowoff(g, r)] : make_float2(0.f, 0.f);
            hr[r] = tf32_hi(x.x);
            hi[r] = tf32_hi(x.y);
            lr[r] = tf32_hi(x.x - __uint_as_float(hr[r]));
            li[r] = tf32_hi(x.y - __uint_as_float(hi[r]));
        }
        tc_st32(lane_col + 0, hr);
        tc_st32(lane_col + 32, hi);
        tc_st32(lane_col + 64, lr);
        tc_st32(lane_col + 96, li);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (c.lt == 0) {
        tc_fence_after();
        // B matrices 0 Re U hi, 1 Im U hi, 2 Re U lo, 3 Im U lo (4 KB each)
        const uint32_t sb = smem_u32(c.cs + S.dcst);
        constexpr uint32_t id = tc_idesc_tf32(128, 32, false), idn = tc_idesc_tf32(128, 32, true);
        const int n_mt = ncols > 128 ? 2 : 1;
        for (int t = 0; t < n_mt; ++t) {
            const uint32_t b0 = c.tmem + (uint32_t)(256 * t);
            const uint32_t ahr = b0, ahi = b0 + 32, alr = b0 + 64, ali = b0 + 96;
            const uint32_t dmr = b0 + 128, dmi = b0 + 160, dcr = b0 + 192, dci = b0 + 224;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t ko = 8 * k;
                const uint64_t ure = tc_smem_desc(sb + 32 * k), uim = tc_smem_desc(sb + 4096 + 32 * k);
                const uint64_t urel = tc_smem_desc(sb + 8192 + 32 * k), uiml = tc_smem_desc(sb + 12288 + 32 * k);
                const int acc = k > 0;
                tc_mma_tf32(dmr, ahr + ko, ure, id, acc);
                tc_mma_tf32(dmr, ahi + ko, uim, idn, 1);
                tc_mma_tf32(dmi, ahr + ko, uim, id, acc);
                tc_mma_tf32(dmi, ahi + ko, ure, id, 1);
                tc_mma_tf32(dcr, alr + ko, ure, id, acc);
                tc_mma_tf32(dcr, ali + ko, uim, idn, 1);
                tc_mma_tf32(dcr, ahr + ko, urel, id, 1);
                tc_mma_tf32(dcr, ahi + ko, uiml, idn, 1);
                tc_mma_tf32(dci, alr + ko, uim, id, acc);
                tc_mma_tf32(dci, ali + ko, ure, id, 1);
                tc_mma_tf32(dci, ahr + ko, uiml, id, 1);
                tc_mma_tf32(dci, ahi + ko, urel, id, 1);
            }
        }
        tc_commit(c.mma_bar);
    }
    const bool ok = mbar_wait_bounded(c.mma_bar, *c.mma_phase);
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    if (c.lt == 0) *c.mma_phase ^= 1u;   // read by every thread above; written after the barrier
    {
        uint32_t dr[32], di[32], er[32], ei[32];
        tc_ld32(lane_col + 128, dr);
        tc_ld32(lane_col + 160, di);
        tc_ld32(lane_col + 192, er);
        tc_ld32(lane_col + 224, ei);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (mine) {
#pragma unroll
            for (int r = 0; r < 32; ++r)
                c.buf[co ^ dense_rowoff(g, r)] = make_float2(__uint_as_float(dr[r]) + __uint_as_float(er[r]),
                                                             __uint_as_float(di[r]) + __uint_as_float(ei[r]));
        }
    }
    tc_fence_before();
    return true;
}

// tensor memory for the dense sweeps: allocated by warp 0 (all of it: one
// dense CTA per SM), the base address broadcast through shared memory
__device__ __forceinline__ uint32_t tc_alloc(uint32_t *slot) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "n"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *slot;
}
__device__ __forceinline__ void tc_dealloc(uint32_t base) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "n"(kTmemCols));
    }
}

template <int NT>
__device__ __forceinline__ bool run_dense(const SweepCtx &c, const Sweep &S, int sidx) {
    // two m16 tiles per warp when every warp still gets work
    const bool two = (1 << (c.T - 5)) >= 32 * (NT / 32);
    switch (S.dense) {
        case DS_FP32: dense_fp32<NT>(c, S, sidx); break;
        case DS_TF32X3:
            if constexpr (NT == 256) return dense_tc_tf32x3<NT>(c, S, sidx);
            break;
        default:
            if (two) dense_bf16<2, NT>(c, S, sidx);
            else dense_bf16<1, NT>(c, S, sidx);
            break;
    }
    return true;
}

// ---------------------------------------------------------------------------
// the persistent tile kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t row_offset(int r, int H, const int *hb) {
    uint64_t o = 0;
    for (int k = 0; k < H; ++k)
        if ((r >> k) & 1) o |= 1ull << hb[k];
    return o;
}

__device__ __forceinline__ uint64_t tile_base(const TileArgs &A, long long ti) {
    uint64_t g = 0;
    for (int i = 0; i < A.n_outer; ++i)
        if ((ti >> i) & 1) g |= 1ull << A.outer_pos[i];
    return g;
}

__device__ __forceinline__ void tile_coords(const TmaGeom &g, long long ti, long long bi, int c[5]) {
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        long long v = 0;
        if (d < g.ndims) {
            if (g.kind[d] == 1) v = (ti >> g.off[d]) & ((1ll << g.w[d]) - 1);
            if (d == g.batch_dim) v += bi << g.w[d];
        }
        c[d] = (int)v;
    }
}

// Shared-memory layout of a tile pass (base aligned to 1024 bytes for the
// 128-byte swizzle):
//   [0, 64)      full[8]   mbarriers: tile loaded into buffer b
//   [64, 176)    hb[14], contrib[14]
//   [176, 240)   empty[8]  mbarriers: consumers done with buffer b
//   [240, 244)   abort flag
//   [244, 252)   tensor-memory base, phase of the dense sweeps' MMA barrier
//   off_desc     sweeps | micro-ops | diagonals | item tables (global bits, smem offsets)
//   off_consts   constants (cs_copies consecutive copies of n_const entries,
//                each copy 128-byte aligned)
//   off_roots    QFT roots (when used)
//   off_buf0     n_buf tile buffers of 8 * 2^T bytes
struct TileShared {
    uint64_t *full, *empty;
    int *abort_flag;
    uint32_t *tmem_slot, *mma_phase;
    int *s_hb, *s_contrib;
    Sweep *s_sweeps;
    MicroOp *s_micro;
    DiagDesc *s_diags;
    uint64_t *s_tab_g;
    int *s_tab_s;
    float2 *cs, *roots, *buf0;
};

__device__ __forceinline__ int const_copy_stride(int n_const) { return (n_const + 15) & ~15; }

// Stage the pass descriptor, the constants (cs_copies copies of item 0's set)
// and the roots in shared memory, initialise the mbarriers and build the
// item-address tables.  Every thread of the CTA takes part; ends with a
// barrier.
template <int NT>
__device__ __forceinline__ TileShared stage_tile_pass(const TileArgs &A, unsigned char *sm_raw, int cs_copies) {
    TileShared S;
    // the 128-byte swizzle needs 1024-byte aligned tile buffers: align the base
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    S.full = reinterpret_cast<uint64_t *>(sm);
    S.s_hb = reinterpret_cast<int *>(sm + 64);
    S.s_contrib = S.s_hb + kMaxTileBits;
    S.empty = reinterpret_cast<uint64_t *>(sm + 176);
    S.abort_flag = reinterpret_cast<int *>(sm + 240);
    S.tmem_slot = reinterpret_cast<uint32_t *>(sm + 244);
    S.mma_phase = reinterpret_cast<uint32_t *>(sm + 248);
    S.s_sweeps = reinterpret_cast<Sweep *>(sm + A.off_desc);
    const TilePass &P = *A.pass;
    const int n_sweeps = P.n_sweeps, n_micro = P.n_micro;
    S.s_micro = reinterpret_cast<MicroOp *>(S.s_sweeps + n_sweeps);
    S.s_diags = reinterpret_cast<DiagDesc *>(S.s_micro + n_micro);
    S.s_tab_g = reinterpret_cast<uint64_t *>(S.s_diags + kMaxDiag);
    S.s_tab_s = reinterpret_cast<int *>(S.s_tab_g + n_sweeps * kItemTab);
    S.cs = reinterpret_cast<float2 *>(sm + A.off_consts);
    S.roots = reinterpret_cast<float2 *>(sm + A.off_roots);
    S.buf0 = reinterpret_cast<float2 *>(sm + A.off_buf0);
    const int tid = threadIdx.x;
    const int L = P.L, T = P.T;
    Sweep *s_sweeps = S.s_sweeps;
    int *s_hb = S.s_hb, *s_contrib = S.s_contrib;

    // stage the pass descriptor and constants in shared memory
    {
        const int *src = reinterpret_cast<const int *>(P.sweeps);
        int *dst = reinterpret_cast<int *>(s_sweeps);
        const int nw_s = n_sweeps * (int)(sizeof(Sweep) / 4);
        for (int i = tid; i < nw_s; i += NT) dst[i] = src[i];
        src = reinterpret_cast<const int *>(P.micro);
        dst = reinterpret_cast<int *>(S.s_micro);
        const int nw_m = n_micro * (int)(sizeof(MicroOp) / 4);
        for (int i = tid; i < nw_m; i += NT) dst[i] = src[i];
        src = reinterpret_cast<const int *>(P.diags);
        dst = reinterpret_cast<int *>(S.s_diags);
        const int nw_d = kMaxDiag * (int)(sizeof(DiagDesc) / 4);
        for (int i = tid; i < nw_d; i += NT) dst[i] = src[i];
    }
    for (int i = tid; i < P.n_const; i += NT) S.cs[i] = A.consts[i];
    for (int cpy = 1; cpy < cs_copies; ++cpy)
        for (int i = tid; i < P.n_const; i += NT) S.cs[cpy * const_copy_stride(P.n_const) + i] = A.consts[i];
    if (A.off_roots)
        for (int i = tid; i < kRootsEntries; i += NT) S.roots[i] = A.roots[i];
    if (tid < kMaxTileBits) {
        s_hb[tid] = P.hb[tid];
        s_contrib[tid] = P.smem_contrib[tid];
    }
    if (tid == 0) {
        for (int b = 0; b < kMaxTileBuffers; ++b) {
            mbar_init(&S.full[b], 1);
            mbar_init(&S.empty[b], 1);
        }
        *S.abort_flag = 0;
        *S.mma_phase = 0;
        fence_mbar_init();
    }
    __syncthreads();
    // item-address tables: item bits 0-4, 5-9, 10-13 of each sweep -> XOR of the
    // shared-memory offsets and OR of the global index bits of those tile bits
    for (int e = tid; e < n_sweeps * kItemTab; e += NT) {
        const int sw = e / kItemTab, idx = e - sw * kItemTab;
        if (idx >= kItemTab - kGroupTab) {
            // the sweep's group bits
            const int m = idx - (kItemTab - kGroupTab);
            const int tb = m < s_sweeps[sw].r ? s_sweeps[sw].gbit[m] : -1;
            S.s_tab_s[e] = tb < 0 ? 0 : s_contrib[tb];
            S.s_tab_g[e] = tb < 0 ? 0ull : (tb < L ? (1ull << tb) : (1ull << s_hb[tb - L]));
            continue;
        }
        const int part = idx < 32 ? 0 : (idx < 64 ? 1 : 2);
        const int v = idx - 32 * part;
        const int nb = T - s_sweeps[sw].r;
        int so = 0;
        uint64_t go = 0;
        for (int b = 0; b < 5; ++b) {
            const int i = 5 * part + b;
            if (((v >> b) & 1) && i < nb) {
                const int tb = s_sweeps[sw].tbit[i];
                so ^= s_contrib[tb];
                go |= tb < L ? (1ull << tb) : (1ull << s_hb[tb - L]);
            }
        }
        S.s_tab_s[e] = so;
        S.s_tab_g[e] = go;
    }
    fence_proxy_async();
    __syncthreads();
    return S;
}

// DENSE: the pass has dense-block sweeps (a separate instantiation, so that
// the register budget of the other passes does not grow with the dense code)
template <int R, int NT, int MINB = 1, bool DENSE = false, int KS = KS_ALL>
__global__ void __launch_bounds__(NT, MINB)
    tile_pass_kernel(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_dst,
                     const TileArgs A) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const TileShared S = stage_tile_pass<NT>(A, sm_raw, 1);
    uint64_t *full = S.full;
    const int *s_hb = S.s_hb;
    const int *s_contrib = S.s_contrib;
    const Sweep *s_sweeps = S.s_sweeps;
    float2 *cs = S.cs;
    float2 *buf0 = S.buf0;
    const TilePass &P = *A.pass;
    const int n_sweeps = P.n_sweeps;
    const int NB = A.n_buf;
    const int tid = threadIdx.x;
    const int L = P.L, H = P.H, T = P.T;
    const int tile_elems = 1 << T;
    const uint32_t tile_bytes = 8u << T;
    const long long total = A.n_tiles * (long long)A.batch;
    if ((long long)blockIdx.x >= total) return;
    const long long stride = gridDim.x;
    const int n_mine = (int)((total - 1 - blockIdx.x) / stride + 1);   // tiles of this CTA
    const int rows = 1 << H;
    const uint32_t row_bytes = 8u << L;

    // warp 0 issues the copies: with the tensor map its first lane (one
    // instruction per tile); without one (bit sets needing more than 5 tensor
    // dims) all 32 lanes share the tile's row copies, lane 0 posting the
    // expected bytes first.  Every lane commits and later waits on its own
    // bulk store groups.
    const int lane = tid & 31;
    auto load = [&](int k) {
        const int b = k % NB;
        float2 *dstbuf = buf0 + (size_t)b * tile_elems;
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        if (lane == 0) mbar_arrive_expect_tx(&full[b], tile_bytes);
        if (A.use_tma) {
            if (lane == 0) {
                int c[5];
                tile_coords(A.geo, ti, bi, c);
                tma_load_5d(dstbuf, &tm_src, c, &full[b]);
            }
        } else {
            __syncwarp();
            const float2 *src = A.src + bi * A.state_elems + tile_base(A, ti);
            for (int r = lane; r < rows; r += 32)
                bulk_g2s(dstbuf + ((size_t)r << L), src + row_offset(r, H, s_hb), row_bytes, &full[b]);
        }
    };
    auto store = [&](int k) {
        const float2 *srcbuf = buf0 + (size_t)(k % NB) * tile_elems;
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        if (A.use_tma) {
            if (lane == 0) {
                int c[5];
                tile_coords(A.geo, ti, bi, c);
                tma_store_5d(&tm_dst, c, srcbuf);
            }
        } else {
            float2 *dst = A.dst + bi * A.state_elems + tile_base(A, ti);
            for (int r = lane; r < rows; r += 32)
                bulk_s2g(dst + row_offset(r, H, s_hb), srcbuf + ((size_t)r << L), row_bytes);
        }
        bulk_commit();
    };

    const int D = A.prefetch;
    const int PF = A.l2_prefetch;   // tiles beyond the smem prefetch warmed in L2
    auto l2pf = [&](int k) {
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        int c[5];
        tile_coords(A.geo, ti, bi, c);
        tma_prefetch_l2_5d(&tm_src, c);
    };
    if (tid == 0 && A.use_tma)
        for (int k = D; k < D + PF && k < n_mine; ++k) l2pf(k);
    if (tid < 32)
        for (int k = 0; k < D && k < n_mine; ++k) load(k);

    SweepCtx c;
    c.lt = tid;
    c.tmem = 0;
    c.mma_bar = &S.empty[0];   // the empty barriers are unused by this kernel
    c.mma_phase = S.mma_phase;
    if constexpr (DENSE) {
        if (A.tmem) c.tmem = tc_alloc(S.tmem_slot);
    }
    c.n_const = P.n_const;
    c.tile_elems = tile_elems;
    c.err = A.err;
    c.T = T;
    c.L = L;
    c.contrib = s_contrib;
    c.hb = s_hb;
    c.cs = cs;
    c.roots = S.roots;
    c.micro = S.s_micro;
    c.diags = S.s_diags;
    c.tab_s = S.s_tab_s;
    c.tab_g = S.s_tab_g;
    long long cur_item = 0;   // constants of item 0 are staged above
    for (int k = 0; k < n_mine; ++k) {
        if (tid < 32 && k + D < n_mine) {
            // buffer (k+D) % NB last held tile k+D-NB, stored at the end of
            // iteration k+D-NB: allow the NB-D-1 newer stores to stay in flight
            switch (NB - D - 1) {
                case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
                case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
                case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
                default: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
            }
            load(k + D);
        }
        if (tid == 0 && A.use_tma && k + D + PF < n_mine) l2pf(k + D + PF);
        // a bounded wait that ran out (here or in a dense sweep's MMAs): record it,
        // let this CTA's copies in flight land, free the tensor memory, return
        auto abort_pass = [&](bool mma_pending) {
            if (tid == 0) {
                atomicCAS(A.err, 0, (int)QS_ERR_TIMEOUT);
                for (int kk = k + 1; kk < k + D && kk < n_mine; ++kk)
                    mbar_wait_bounded(&full[kk % NB], (uint32_t)((kk / NB) & 1));
                if (mma_pending) mbar_wait_bounded(c.mma_bar, *c.mma_phase);   // the MMAs, once more
            }
            if (tid < 32) bulk_wait_all0();
            if constexpr (DENSE) {
                if (A.tmem) tc_dealloc(c.tmem);
            }
        };
        const bool ok = mbar_wait_bounded(&full[k % NB], (uint32_t)((k / NB) & 1));
        if (__syncthreads_or(!ok)) {
            abort_pass(false);
            return;
        }
        const long long t = blockIdx.x + (long long)k * stride;
        const long long ti = t % A.n_tiles;
        if (A.const_stride) {
            // per-item constants: restage when this tile starts another item (the
            // previous tile's sweeps ended at the barrier before its store)
            const long long item = (t / A.n_tiles) / A.const_group;
            if (item != cur_item) {
                const float2 *src = A.consts + item * A.const_stride;
                for (int i = tid; i < P.n_const; i += NT) cs[i] = src[i];
                __syncthreads();
                cur_item = item;
            }
        }
        c.buf = buf0 + (size_t)(k % NB) * tile_elems;
        c.tile_gbase = A.needs_gidx ? tile_base(A, ti) : 0;
        for (int s = 0; s < n_sweeps; ++s) {
            if (DENSE && s_sweeps[s].dense) {
                if (!run_dense<NT>(c, s_sweeps[s], s)) {   // uniform over the CTA
                    abort_pass(true);
                    return;
                }
            } else {
                run_sweep<R, NT, KS>(c, s_sweeps[s], s);
            }
            if (s + 1 < n_sweeps) __syncthreads();
        }
        fence_proxy_async();   // generic-proxy writes before the async-proxy store
        __syncthreads();
        if (tid < 32) store(k);
    }
    if (tid < 32) bulk_wait_all0();
    if constexpr (DENSE) {
        if (A.tmem) tc_dealloc(c.tmem);
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised tile pass: one CTA per SM, NB (>= 3) tile buffers, a
// producer warpgroup and two consumer groups of NTG threads.
//
// The producer's lane 0 walks this CTA's tiles in order: it loads tile j into
// buffer j % NB as soon as the consumers of tile j - NB are done with that
// buffer and its store has read it out.  Consumer group g takes the tiles
// k = g, g + 2, ... : it waits for the tile's load, runs the sweeps with a
// named barrier of its own between them, and signals the buffer's empty
// barrier.  A load completes on the barrier of its (buffer, group) pair,
// full[2 b + g]: with an odd buffer count a buffer alternates between the
// groups, and a shared barrier would let a group that is one tile ahead take
// the completed phase of a load two uses back (the same parity) while the
// other group's load into that buffer is still in flight.  On its own pair
// barrier a group waits for every phase in order, so parity is exact.  The two groups work on different tiles at different phases of
// their sweeps (the shared-memory, FP32 and TMA work of the SM overlap
// instead of lining up behind one barrier), and the load of a group's next
// tile is issued while the other group still computes, so neither group waits
// for a load issued after its own previous tile.
//
// Every wait is bounded (2 s): a waiter that gives up records QS_ERR_TIMEOUT,
// raises the CTA's abort flag (which ends the other waits) and returns; the
// producer lets the copies it issued land before it returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t *bar, uint32_t parity, const volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && (*abort_flag || globaltimer() - t0 > 2000000000ull)) return false;
    }
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// barrier among the `count` threads that use named barrier `id`
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// the same barrier, returning whether any of them passed p = true
__device__ __forceinline__ bool named_sync_or(int id, int count, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Register split: the CTA launches 2 NTG + 128 threads; the producer
// warpgroup (only its first thread works) drops to 24 registers and the
// consumers rise to ws_consumer_regs(NTG).  The launch total bounds the split
// (setmaxnreg.inc draws on the registers the CTA was launched with):
//   NTG = 256: 640 threads x 96 = 61,440 >= 128 x 24 + 512 x 112 = 60,416;
//              per SM sub-partition 4 x 32 x 112 + 32 x 24 = 15,104 <= 16,384
//   NTG = 128: 384 threads x 168 = 64,512 >= 128 x 24 + 256 x 240 = 64,512;
//              per SM sub-partition 2 x 32 x 240 + 32 x 24 = 16,128 <= 16,384
constexpr int kWsProducerRegs = 24;
constexpr int ws_consumer_regs(int ntg) { return ntg == 256 ? 112 : 240; }

template <int R, int NTG, bool DENSE = false, int KS = KS_ALL>
__global__ void __launch_bounds__(2 * NTG + 128, 1)
    tile_pass_ws_kernel(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_dst,
                        const TileArgs A) {
    constexpr int NT = 2 * NTG + 128;
    static_assert(NTG == 256 || NTG == 128, "the register split is sized for groups of 256 or 128 threads");
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const int per_item = A.const_stride != 0;
    const TileShared S = stage_tile_pass<NT>(A, sm_raw, per_item ? 2 : 1);
    const TilePass &P = *A.pass;
    const int n_sweeps = P.n_sweeps;
    const int NB = A.n_buf;
    const int tid = threadIdx.x;
    const int T = P.T;
    const int tile_elems = 1 << T;
    const uint32_t tile_bytes = 8u << T;
    const long long total = A.n_tiles * (long long)A.batch;
    if ((long long)blockIdx.x >= total) return;
    const long long stride = gridDim.x;
    const int n_mine = (int)((total - 1 - blockIdx.x) / stride + 1);   // tiles of this CTA
    volatile int *abort_flag = S.abort_flag;
    // tiles between two uses of a (buffer, group) barrier: lcm(NB, 2)
    const int pair_period = (NB & 1) ? 2 * NB : NB;

    if (tid >= 2 * NTG) {
        // producer warpgroup: its first thread issues every copy (one tensor
        // copy per tile)
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kWsProducerRegs));
        if (tid != 2 * NTG) return;
        auto coords = [&](int k, int c[5]) {
            const long long t = blockIdx.x + (long long)k * stride;
            const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
            tile_coords(A.geo, ti, bi, c);
        };
        int loaded = 0;
        bool ok = true;
        for (int j = 0; j < n_mine + NB; ++j) {
            const int b = j % NB;
            if (j >= NB) {
                // tile j - NB: its consumers are done; store it from buffer b
                if (!mbar_wait_abortable(&S.empty[b], (uint32_t)(((j - NB) / NB) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                int c[5];
                coords(j - NB, c);
                tma_store_5d(&tm_dst, c, S.buf0 + (size_t)b * tile_elems);
                bulk_commit();
                if (j >= n_mine) continue;
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
            if (j < n_mine) {
                int c[5];
                coords(j, c);
                uint64_t *fb = &S.full[2 * b + (j & 1)];
                mbar_arrive_expect_tx(fb, tile_bytes);
                tma_load_5d(S.buf0 + (size_t)b * tile_elems, &tm_src, c, fb);
                loaded = j + 1;
            }
        }
        if (!ok) {
            atomicCAS(A.err, 0, (int)QS_ERR_TIMEOUT);
            *abort_flag = 1;
            // let the last load of every buffer land before the CTA leaves
            for (int j = loaded - NB < 0 ? 0 : loaded - NB; j < loaded; ++j)
                mbar_wait_bounded(&S.full[2 * (j % NB) + (j & 1)], (uint32_t)((j / pair_period) & 1));
        }
        bulk_wait_all0();
        return;
    }

    // consumer group g
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(ws_consumer_regs(NTG)));
    const int g = tid / NTG;
    const int bar_id = 1 + g;
    float2 *cs = S.cs + (per_item ? g * const_copy_stride(P.n_const) : 0);
    SweepCtx c;
    c.lt = tid - g * NTG;
    c.tmem = 0;
    c.mma_bar = nullptr;
    c.mma_phase = nullptr;
    c.n_const = P.n_const;
    c.tile_elems = tile_elems;
    c.err = A.err;
    c.T = T;
    c.L = P.L;
    c.contrib = S.s_contrib;
    c.hb = S.s_hb;
    c.cs = cs;
    c.roots = S.roots;
    c.micro = S.s_micro;
    c.diags = S.s_diags;
    c.tab_s = S.s_tab_s;
    c.tab_g = S.s_tab_g;
    long long cur_item = 0;   // constants of item 0 are staged above
    for (int k = g; k < n_mine; k += 2) {
        const int b = k % NB;
        const bool ok = mbar_wait_abortable(&S.full[2 * b + g], (uint32_t)((k / pair_period) & 1), abort_flag);
        if (named_sync_or(bar_id, NTG, !ok)) {
            if (c.lt == 0) {
                atomicCAS(A.err, 0, (int)QS_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            return;
        }
        const long long t = blockIdx.x + (long long)k * stride;
        const long long ti = t % A.n_tiles;
        if (per_item) {
            // per-item constants: this group's copy is restaged when its tile
            // starts another item (its previous tile ended at a group barrier)
            const long long item = (t / A.n_tiles) / A.const_group;
            if (item != cur_item) {
                const float2 *src = A.consts + item * A.const_stride;
                for (int i = c.lt; i < P.n_const; i += NTG) cs[i] = src[i];
                named_sync(bar_id, NTG);
                cur_item = item;
            }
        }
        c.buf = S.buf0 + (size_t)b * tile_elems;
        c.tile_gbase = A.needs_gidx ? tile_base(A, ti) : 0;
        for (int s = 0; s < n_sweeps; ++s) {
            if (DENSE && S.s_sweeps[s].dense) run_dense<NTG>(c, S.s_sweeps[s], s);
            else run_sweep<R, NTG, KS, true>(c, S.s_sweeps[s], s);
            if (s + 1 < n_sweeps) named_sync(bar_id, NTG);
        }
        fence_proxy_async();   // generic-proxy writes before the async-proxy store
        named_sync(bar_id, NTG);
        if (c.lt == 0) mbar_arrive(&S.empty[b]);
    }
}

}  // namespace qs
