// Tile-pass engine (sm_103a).
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
// Tiles rotate through 2-3 shared buffers: while the 8 warps process tile k,
// the load of tile k+1 and the stores of tiles k-1 (and k-2) are in flight.
// Thread 0 issues the copies; with 3 buffers the buffer it refills was
// stored two tiles ago, so waiting for that store to have read shared memory
// does not stall.
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
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
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

// real 2x2 (RY family): 4 FP32 ops per amplitude
template <int R, int M>
__device__ __forceinline__ void op_u1r(float2 (&a)[1 << R], const float2 *cs) {
    const float m00 = cs[0].x, m01 = cs[0].y, m10 = cs[1].x, m11 = cs[1].y;
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = make_float2(fmaf(m00, a0.x, m01 * a1.x), fmaf(m00, a0.y, m01 * a1.y));
        a[k] = make_float2(fmaf(m10, a0.x, m11 * a1.x), fmaf(m10, a0.y, m11 * a1.y));
    }
}

// unnormalised Hadamard butterfly (the 1/sqrt 2 is folded into the sweep scale)
template <int R, int M>
__device__ __forceinline__ void op_h(float2 (&a)[1 << R]) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = make_float2(a0.x + a1.x, a0.y + a1.y);
        a[k] = make_float2(a0.x - a1.x, a0.y - a1.y);
    }
}

// QFT stage: butterfly on bit M, then the ladder phase on the bit-M = 1 half:
// item twiddle w times the group-bit twiddle gtab[k]
template <int R, int M>
__device__ __forceinline__ void op_qft(float2 (&a)[1 << R], const float2 *gtab, float2 w) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        const float2 a0 = a[j], a1 = a[k];
        a[j] = make_float2(a0.x + a1.x, a0.y + a1.y);
        a[k] = cmul(make_float2(a0.x - a1.x, a0.y - a1.y), cmul(w, gtab[k]));
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

// layers: the same 2x2 family on every group bit in `mask`, straight-line code
template <int R, int M = 0>
__device__ __forceinline__ void layer_rxc(float2 (&a)[1 << R], const float2 *k0, uint32_t mask) {
    if constexpr (M < R) {
        if ((mask >> M) & 1) op_rxc<R, M>(a, k0 + M);
        layer_rxc<R, M + 1>(a, k0, mask);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void layer_u1r(float2 (&a)[1 << R], const float2 *k0, uint32_t mask) {
    if constexpr (M < R) {
        if ((mask >> M) & 1) op_u1r<R, M>(a, k0 + 2 * M);
        layer_u1r<R, M + 1>(a, k0, mask);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void layer_u1(float2 (&a)[1 << R], const float2 *k0, uint32_t mask, const Grp<R> &G) {
    if constexpr (M < R) {
        if ((mask >> M) & 1) op_u1<R, M>(a, k0 + 4 * M, 0ull, 0ull, 0ull, G);
        layer_u1<R, M + 1>(a, k0, mask, G);
    }
}
template <int R, int M = 0>
__device__ __forceinline__ void layer_h(float2 (&a)[1 << R], uint32_t mask) {
    if constexpr (M < R) {
        if ((mask >> M) & 1) op_h<R, M>(a);
        layer_h<R, M + 1>(a, mask);
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
};

__device__ __forceinline__ uint64_t glob_contrib(const SweepCtx &c, int tb) {
    return tb < c.L ? (1ull << tb) : (1ull << c.hb[tb - c.L]);
}

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
            *reinterpret_cast<float4 *>(c.buf + o) = make_float4(a[j].x, a[j].y, a[j + 1].x, a[j + 1].y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            int o = saddr;
#pragma unroll
            for (int m = 0; m < R; ++m)
                if ((j >> m) & 1) o ^= gs[m];
            c.buf[o] = a[j];
        }
    }
}

template <int R, int NT>
__device__ __forceinline__ void run_sweep(const SweepCtx &c, const Sweep &S, int sidx) {
    int gs[R];
    Grp<R> G;
#pragma unroll
    for (int m = 0; m < R; ++m) {
        gs[m] = c.contrib[S.gbit[m]];
        G.gg[m] = glob_contrib(c, S.gbit[m]);
    }
    const int nb = c.T - R;
    const int n_items = 1 << nb;
    const bool vec = S.vec != 0;
    const int *ts = c.tab_s + sidx * kItemTab;
    const uint64_t *tg = c.tab_g + sidx * kItemTab;
    for (int item = threadIdx.x; item < n_items; item += NT) {
        const int i0 = item & 31, i1 = 32 + ((item >> 5) & 31), i2 = 64 + ((item >> 10) & 15);
        const int saddr = ts[i0] ^ ts[i1] ^ ts[i2];
        const uint64_t gbase = c.tile_gbase | tg[i0] | tg[i1] | tg[i2];
        float2 a[1 << R];
        sweep_load<R>(c, vec, saddr, gs, a);
        for (int oi = S.op_begin; oi < S.op_end; ++oi) {
            const MicroOp &op = c.micro[oi];
            switch (op.kind) {
                case MK_U1:
                    disp_u1<R>(op.a, a, c.cs + op.cst, op.cmask, op.cval, gbase, G);
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
                case MK_U2:
                    disp_u2<R>(op.a, op.b, a, c.cs + op.cst, op.cmask, op.cval, gbase, G);
                    break;
                case MK_QFT: {
                    const uint64_t Mk = (op.p > op.lo) ? (((1ull << op.p) - 1) & ~((1ull << op.lo) - 1)) : 0ull;
                    const float2 w = twiddle(gbase & Mk, op.p, c.roots);
                    disp_qft<R>(op.a, a, c.cs + op.cst, w);
                    break;
                }
                case MK_LAYER: {
                    const float2 *k0 = c.cs + op.cst;
                    const uint32_t mask = (uint32_t)op.b;
                    switch (op.a) {
                        case MK_RXC: layer_rxc<R>(a, k0, mask); break;
                        case MK_U1R: layer_u1r<R>(a, k0, mask); break;
                        case MK_U1: layer_u1<R>(a, k0, mask, G); break;
                        default: layer_h<R>(a, mask); break;
                    }
                    break;
                }
                case MK_QFTL:
                    layer_qft<R>(a, c.cs + op.cst, (uint32_t)op.b, op.cmask, gbase, c.roots);
                    break;
                case MK_DIAG: {
                    const DiagDesc &d = c.diags[op.cst];
                    const uint32_t dyn_s = (uint32_t)op.a, dyn_g = (uint32_t)op.b;
                    float2 stat = d.pad0 ? make_float2(d.gph_re, d.gph_im) : make_float2(1.f, 0.f);
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
                    break;
                }
                default:
                    break;
            }
        }
        if (S.scale != 1.f) {
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) a[j] = make_float2(a[j].x * S.scale, a[j].y * S.scale);
        }
        sweep_store<R>(c, vec, saddr, gs, a);
    }
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

// 16-byte chunk q of a tile (tile-local index 2q, 2q+1): its shared-memory
// float2 offset (XOR-linear layout) and its global offset within the state
__device__ __forceinline__ int chunk_smem(int q, int T, const int *contrib) {
    int o = 0;
    for (int tb = 1; tb < T; ++tb)
        if ((q >> (tb - 1)) & 1) o ^= contrib[tb];
    return o;
}
__device__ __forceinline__ uint64_t chunk_glob(int q, int L, int H, const int *hb) {
    const int t = q << 1;
    uint64_t g = (uint64_t)(t & ((1 << L) - 1));
    const int r = t >> L;
    for (int k = 0; k < H; ++k)
        if ((r >> k) & 1) g |= 1ull << hb[k];
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

template <int R, int NT, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB)
    tile_pass_kernel(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_dst,
                     const TileArgs A) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // the 128-byte swizzle needs 1024-byte aligned tile buffers: align the base
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);          // [kMaxTileBuffers]
    int *s_hb = reinterpret_cast<int *>(sm + 64);
    int *s_contrib = s_hb + kMaxTileBits;
    Sweep *s_sweeps = reinterpret_cast<Sweep *>(sm + A.off_desc);
    const TilePass &P = *A.pass;
    const int n_sweeps = P.n_sweeps, n_micro = P.n_micro;
    MicroOp *s_micro = reinterpret_cast<MicroOp *>(s_sweeps + n_sweeps);
    DiagDesc *s_diags = reinterpret_cast<DiagDesc *>(s_micro + n_micro);
    uint64_t *s_tab_g = reinterpret_cast<uint64_t *>(s_diags + kMaxDiag);
    int *s_tab_s = reinterpret_cast<int *>(s_tab_g + n_sweeps * kItemTab);
    float2 *cs = reinterpret_cast<float2 *>(sm + A.off_consts);
    float2 *roots = reinterpret_cast<float2 *>(sm + A.off_roots);
    float2 *buf0 = reinterpret_cast<float2 *>(sm + A.off_buf0);
    const int NB = A.n_buf;
    const int tid = threadIdx.x;
    const int L = P.L, H = P.H, T = P.T;
    const int tile_elems = 1 << T;
    const uint32_t tile_bytes = 8u << T;
    const long long total = A.n_tiles * (long long)A.batch;

    // stage the pass descriptor and constants in shared memory
    {
        const int *src = reinterpret_cast<const int *>(P.sweeps);
        int *dst = reinterpret_cast<int *>(s_sweeps);
        const int nw_s = n_sweeps * (int)(sizeof(Sweep) / 4);
        for (int i = tid; i < nw_s; i += NT) dst[i] = src[i];
        src = reinterpret_cast<const int *>(P.micro);
        dst = reinterpret_cast<int *>(s_micro);
        const int nw_m = n_micro * (int)(sizeof(MicroOp) / 4);
        for (int i = tid; i < nw_m; i += NT) dst[i] = src[i];
        src = reinterpret_cast<const int *>(P.diags);
        dst = reinterpret_cast<int *>(s_diags);
        const int nw_d = kMaxDiag * (int)(sizeof(DiagDesc) / 4);
        for (int i = tid; i < nw_d; i += NT) dst[i] = src[i];
    }
    for (int i = tid; i < P.n_const; i += NT) cs[i] = A.consts[i];
    if (A.off_roots)
        for (int i = tid; i < kRootsEntries; i += NT) roots[i] = A.roots[i];
    if (tid < kMaxTileBits) {
        s_hb[tid] = P.hb[tid];
        s_contrib[tid] = P.smem_contrib[tid];
    }
    if (tid == 0) {
        for (int b = 0; b < kMaxTileBuffers; ++b) mbar_init(&full[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // item-address tables: item bits 0-4, 5-9, 10-13 of each sweep -> XOR of the
    // shared-memory offsets and OR of the global index bits of those tile bits
    for (int e = tid; e < n_sweeps * kItemTab; e += NT) {
        const int sw = e / kItemTab, idx = e - sw * kItemTab;
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
        s_tab_s[e] = so;
        s_tab_g[e] = go;
    }
    fence_proxy_async();
    __syncthreads();
    if ((long long)blockIdx.x >= total) return;
    const long long stride = gridDim.x;
    const int n_mine = (int)((total - 1 - blockIdx.x) / stride + 1);   // tiles of this CTA
    const int rows = 1 << H;
    const uint32_t row_bytes = 8u << L;

    // thread 0 issues every copy (TMA path: one instruction per tile)
    const int io = A.io_mode;
    const int n_chunks = tile_elems >> 1;
    // 16-byte chunk q = tid + i * NT of a tile: offsets are XOR/OR-linear in the
    // bits of q, so split them into a per-thread part (computed once) and the
    // parts of the (at most 4) loop bits
    int c_smem = 0;
    uint64_t c_glob = 0;
    int i_smem[4] = {0, 0, 0, 0};
    uint64_t i_glob[4] = {0, 0, 0, 0};
    int n_ib = 0;
    if (io != 0) {
        if (tid < n_chunks) {
            c_smem = chunk_smem(tid, T, s_contrib);
            c_glob = chunk_glob(tid, L, H, s_hb);
        }
        for (int m = 0; (NT << m) < n_chunks && m < 4; ++m) {
            i_smem[m] = chunk_smem(NT << m, T, s_contrib);
            i_glob[m] = chunk_glob(NT << m, L, H, s_hb);
            n_ib = m + 1;
        }
    }
    const int per_thread = n_chunks > NT ? n_chunks / NT : 1;
    // cp.async path: every thread copies its 16-byte chunks (coalesced rows)
    auto load_threads = [&](int k) {
        float2 *dstbuf = buf0 + (size_t)(k % NB) * tile_elems;
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        const float2 *src = A.src + bi * A.state_elems + tile_base(A, ti);
        if (tid < n_chunks) {
#pragma unroll 4
            for (int i = 0; i < per_thread; ++i) {
                int so = c_smem;
                uint64_t go = c_glob;
                for (int m = 0; m < n_ib; ++m)
                    if ((i >> m) & 1) {
                        so ^= i_smem[m];
                        go |= i_glob[m];
                    }
                cp_async16(dstbuf + so, src + go);
            }
        }
        cp_async_commit();
    };
    // thread stores: 16-byte chunks straight from shared memory to HBM
    auto store_threads = [&](int k) {
        const float2 *srcbuf = buf0 + (size_t)(k % NB) * tile_elems;
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        float2 *dst = A.dst + bi * A.state_elems + tile_base(A, ti);
        if (tid < n_chunks) {
#pragma unroll 4
            for (int i = 0; i < per_thread; ++i) {
                int so = c_smem;
                uint64_t go = c_glob;
                for (int m = 0; m < n_ib; ++m)
                    if ((i >> m) & 1) {
                        so ^= i_smem[m];
                        go |= i_glob[m];
                    }
                const float4 v = *reinterpret_cast<const float4 *>(srcbuf + so);
                *reinterpret_cast<float4 *>(dst + go) = v;
            }
        }
    };
    auto load = [&](int k) {
        const int b = k % NB;
        float2 *dstbuf = buf0 + (size_t)b * tile_elems;
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        mbar_arrive_expect_tx(&full[b], tile_bytes);
        if (A.use_tma) {
            int c[5];
            tile_coords(A.geo, ti, bi, c);
            tma_load_5d(dstbuf, &tm_src, c, &full[b]);
        } else {
            const float2 *src = A.src + bi * A.state_elems + tile_base(A, ti);
            for (int r = 0; r < rows; ++r)
                bulk_g2s(dstbuf + ((size_t)r << L), src + row_offset(r, H, s_hb), row_bytes, &full[b]);
        }
    };
    auto store = [&](int k) {
        const float2 *srcbuf = buf0 + (size_t)(k % NB) * tile_elems;
        const long long t = blockIdx.x + (long long)k * stride;
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        if (A.use_tma) {
            int c[5];
            tile_coords(A.geo, ti, bi, c);
            tma_store_5d(&tm_dst, c, srcbuf);
        } else {
            float2 *dst = A.dst + bi * A.state_elems + tile_base(A, ti);
            for (int r = 0; r < rows; ++r)
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
    if (tid == 0 && io != 2 && A.use_tma)
        for (int k = D; k < D + PF && k < n_mine; ++k) l2pf(k);
    if (io == 2) {
        for (int k = 0; k < D; ++k) {
            if (k < n_mine) load_threads(k);
            else cp_async_commit();   // keep one group per tile slot
        }
    } else if (tid == 0) {
        for (int k = 0; k < D && k < n_mine; ++k) load(k);
    }

    SweepCtx c;
    c.T = T;
    c.L = L;
    c.contrib = s_contrib;
    c.hb = s_hb;
    c.cs = cs;
    c.roots = roots;
    c.micro = s_micro;
    c.diags = s_diags;
    c.tab_s = s_tab_s;
    c.tab_g = s_tab_g;
    for (int k = 0; k < n_mine; ++k) {
        bool ok = true;
        if (io == 2) {
            // buffer (k+D) % NB held tile k+D-NB <= k-1, already stored by the threads
            if (k + D < n_mine) load_threads(k + D);
            else cp_async_commit();
            // groups are committed per tile in order: tile k is done when at most D remain
            switch (D) {
                case 1: cp_async_wait<1>(); break;
                case 2: cp_async_wait<2>(); break;
                case 3: cp_async_wait<3>(); break;
                default: cp_async_wait<4>(); break;
            }
        } else {
            if (tid == 0 && k + D < n_mine) {
                // buffer (k+D) % NB last held tile k+D-NB, stored at the end of
                // iteration k+D-NB: allow the NB-D-1 newer stores to stay in flight
                if (io == 0) {
                    switch (NB - D - 1) {
                        case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
                        case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
                        case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
                        default: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
                    }
                }
                load(k + D);
            }
            if (tid == 0 && A.use_tma && k + D + PF < n_mine) l2pf(k + D + PF);
            ok = mbar_wait_bounded(&full[k % NB], (uint32_t)((k / NB) & 1));
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(A.err, 0, (int)QS_ERR_TIMEOUT);
                for (int kk = k + 1; kk < k + D && kk < n_mine; ++kk)
                    mbar_wait_bounded(&full[kk % NB], (uint32_t)((kk / NB) & 1));
                bulk_wait_all0();
            }
            return;
        }
        const long long t = blockIdx.x + (long long)k * stride;
        const long long ti = t % A.n_tiles;
        c.buf = buf0 + (size_t)(k % NB) * tile_elems;
        c.tile_gbase = tile_base(A, ti);
        for (int s = 0; s < n_sweeps; ++s) {
            run_sweep<R, NT>(c, s_sweeps[s], s);
            __syncthreads();
        }
        if (io == 0) {
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) store(k);
        } else {
            store_threads(k);
            // the buffer is reloaded D iterations later, after this barrier
            if (io == 2) __syncthreads();
            else {
                fence_proxy_async();   // generic reads before the async-proxy refill
                __syncthreads();
            }
        }
    }
    if (io == 2) cp_async_wait<0>();
    if (tid == 0) bulk_wait_all0();
}

template <int R, int NT, int MINB = 1>
static void set_smem(int bytes) {
    cudaFuncSetAttribute(tile_pass_kernel<R, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void tile_kernel_smem_config(int bytes) {
    set_smem<5, 256>(bytes);
    set_smem<4, 256>(bytes);
    set_smem<4, 512>(bytes);
    set_smem<4, 256, 2>(bytes);
    set_smem<3, 256>(bytes);
    set_smem<2, 256>(bytes);
    set_smem<1, 256>(bytes);
}

// R = register group size; 4-bit groups run 512 threads (16 warps per SM)
cudaError_t launch_tile_pass(int R, const TileArgs &A, const void *tm_src, const void *tm_dst, int grid,
                             int smem_bytes, cudaStream_t st) {
    const CUtensorMap &ms = *reinterpret_cast<const CUtensorMap *>(tm_src);
    const CUtensorMap &md = *reinterpret_cast<const CUtensorMap *>(tm_dst);
    cudaGetLastError();
    switch (R) {
        case 5: tile_pass_kernel<5, 256><<<grid, 256, smem_bytes, st>>>(ms, md, A); break;
        case 4:
            if (A.threads == 512) tile_pass_kernel<4, 512><<<grid, 512, smem_bytes, st>>>(ms, md, A);
            else if (A.ctas_per_sm == 2) tile_pass_kernel<4, 256, 2><<<grid, 256, smem_bytes, st>>>(ms, md, A);
            else tile_pass_kernel<4, 256><<<grid, 256, smem_bytes, st>>>(ms, md, A);
            break;
        case 3: tile_pass_kernel<3, 256><<<grid, 256, smem_bytes, st>>>(ms, md, A); break;
        case 2: tile_pass_kernel<2, 256><<<grid, 256, smem_bytes, st>>>(ms, md, A); break;
        default: tile_pass_kernel<1, 256><<<grid, 256, smem_bytes, st>>>(ms, md, A); break;
    }
    return cudaGetLastError();
}

std::string tile_kernel_attrs(int R) {
    cudaFuncAttributes fa;
    cudaError_t e;
    switch (R) {
        case 5: e = cudaFuncGetAttributes(&fa, tile_pass_kernel<5, 256>); break;
        case 4: e = cudaFuncGetAttributes(&fa, tile_pass_kernel<4, 512>); break;
        case 3: e = cudaFuncGetAttributes(&fa, tile_pass_kernel<3, 256>); break;
        case 2: e = cudaFuncGetAttributes(&fa, tile_pass_kernel<2, 256>); break;
        default: e = cudaFuncGetAttributes(&fa, tile_pass_kernel<1, 256>); break;
    }
    if (e != cudaSuccess) return "attrs unavailable";
    return "regs=" + std::to_string(fa.numRegs) + " maxThreads=" + std::to_string(fa.maxThreadsPerBlock) +
           " maxDynSmem=" + std::to_string(fa.maxDynamicSharedSizeBytes) +
           " staticSmem=" + std::to_string(fa.sharedSizeBytes) + " localBytes=" + std::to_string(fa.localSizeBytes);
}

}  // namespace qs
