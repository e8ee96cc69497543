// Tile-pass engine (sm_103a).
//
// One launch = one full-state HBM pass.  Each persistent CTA walks its tiles:
// a tile is 2^T amplitudes = 2^H rows of 2^L contiguous amplitudes (the L low
// index bits) at the row offsets spanned by the pass's high bits hb[].  Rows
// are moved HBM <-> shared memory with bulk-async copies (cp.async.bulk, the
// TMA engine), double-buffered: the next tile's rows land while the current
// tile is computed, and the previous tile's rows drain asynchronously.
// Between load and store the tile goes through "sweeps": every thread holds
// 2^R amplitudes that differ in R tile bits and applies the sweep's micro-ops
// in registers (2x2 / 4x4 unitaries with controls, diagonal phase tables,
// QFT stages = Hadamard butterfly + closed-form ladder twiddle, Sec. 5.1).
// All waits are bounded; on expiry the kernel records QS_ERR_TIMEOUT, drains
// its own copies and returns.
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
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
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

__device__ __forceinline__ float2 diag_phase(const DiagDesc &d, uint64_t x, const float2 *cs) {
    float2 ph;
    int s0 = 0;
    if (d.n_slices > 0) {
        ph = cs[d.slice_off[0] + (int)((x >> d.slice_lo[0]) & ((1u << d.slice_w[0]) - 1))];
        s0 = 1;
    } else {
        ph = d.pad0 ? make_float2(d.gph_re, d.gph_im) : make_float2(1.f, 0.f);
    }
    for (int s = s0; s < d.n_slices; ++s)
        ph = cmul(ph, cs[d.slice_off[s] + (int)((x >> d.slice_lo[s]) & ((1u << d.slice_w[s]) - 1))]);
    for (int g = 0; g < d.n_groups; ++g) {
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
            bool c = (G.gidx(base, j) & cmask) == cval;
            if (!c) {
                b0 = a0;
                b1 = a1;
            }
        }
        a[j] = b0;
        a[k] = b1;
    }
}

template <int R, int M>
__device__ __forceinline__ void op_h(float2 (&a)[1 << R]) {
    const float s = 0.70710678118654752440f;
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        float2 a0 = a[j], a1 = a[k];
        a[j] = make_float2((a0.x + a1.x) * s, (a0.y + a1.y) * s);
        a[k] = make_float2((a0.x - a1.x) * s, (a0.y - a1.y) * s);
    }
}

template <int R, int M>
__device__ __forceinline__ void op_qft(float2 (&a)[1 << R], const float2 *gtab, float2 w) {
    const float s = 0.70710678118654752440f;
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
        if ((j >> M) & 1) continue;
        const int k = j | (1 << M);
        float2 a0 = a[j], a1 = a[k];
        a[j] = make_float2((a0.x + a1.x) * s, (a0.y + a1.y) * s);
        float2 d = make_float2((a0.x - a1.x) * s, (a0.y - a1.y) * s);
        a[k] = cmul(d, cmul(w, gtab[k]));
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
        float2 v[4] = {a[i0], a[i1], a[i2], a[i3]};
        float2 o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float2 acc = cmul(mat[r * 4 + 0], v[0]);
            acc = cmad(mat[r * 4 + 1], v[1], acc);
            acc = cmad(mat[r * 4 + 2], v[2], acc);
            acc = cmad(mat[r * 4 + 3], v[3], acc);
            o[r] = acc;
        }
        a[i0] = o[0];
        a[i1] = o[1];
        a[i2] = o[2];
        a[i3] = o[3];
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

// ---------------------------------------------------------------------------
// one sweep over the tile in shared memory
// ---------------------------------------------------------------------------
struct SweepCtx {
    int L, T, RS;
    const int *hb;           // smem copy of pass hb
    float2 *buf;
    const float2 *cs;
    const float2 *roots;
    uint64_t tile_gbase;     // global index of tile-local 0
};

__device__ __forceinline__ int smem_contrib(const SweepCtx &c, int tb) {
    return tb < c.L ? (1 << tb) : (c.RS << (tb - c.L));
}
__device__ __forceinline__ uint64_t glob_contrib(const SweepCtx &c, int tb) {
    return tb < c.L ? (1ull << tb) : (1ull << c.hb[tb - c.L]);
}

template <int R>
__device__ void run_sweep(const SweepCtx &c, const Sweep &S, const MicroOp *micro, const DiagDesc *diags) {
    int gs[R];
    Grp<R> G;
#pragma unroll
    for (int m = 0; m < R; ++m) {
        gs[m] = smem_contrib(c, S.gbit[m]);
        G.gg[m] = glob_contrib(c, S.gbit[m]);
    }
    const int nb = c.T - R;
    const int n_items = 1 << nb;
    for (int item = threadIdx.x; item < n_items; item += blockDim.x) {
        int saddr = 0;
        uint64_t gbase = c.tile_gbase;
        for (int i = 0; i < nb; ++i)
            if ((item >> i) & 1) {
                const int tb = S.tbit[i];
                saddr += smem_contrib(c, tb);
                gbase |= glob_contrib(c, tb);
            }
        float2 a[1 << R];
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            int o = saddr;
#pragma unroll
            for (int m = 0; m < R; ++m)
                if ((j >> m) & 1) o += gs[m];
            a[j] = c.buf[o];
        }
        for (int oi = S.op_begin; oi < S.op_end; ++oi) {
            const MicroOp &op = micro[oi];
            switch (op.kind) {
                case MK_U1:
                    disp_u1<R>(op.a, a, c.cs + op.cst, op.cmask, op.cval, gbase, G);
                    break;
                case MK_H:
                    disp_h<R>(op.a, a);
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
                case MK_DIAG: {
                    const DiagDesc &d = diags[op.cst];
#pragma unroll
                    for (int j = 0; j < (1 << R); ++j) a[j] = cmul(a[j], diag_phase(d, G.gidx(gbase, j), c.cs));
                    break;
                }
                default:
                    break;
            }
        }
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) {
            int o = saddr;
#pragma unroll
            for (int m = 0; m < R; ++m)
                if ((j >> m) & 1) o += gs[m];
            c.buf[o] = a[j];
        }
    }
}

__device__ void run_sweep_r(int r, const SweepCtx &c, const Sweep &S, const MicroOp *micro, const DiagDesc *diags) {
    switch (r) {
        case 5: run_sweep<5>(c, S, micro, diags); break;
        case 4: run_sweep<4>(c, S, micro, diags); break;
        case 3: run_sweep<3>(c, S, micro, diags); break;
        case 2: run_sweep<2>(c, S, micro, diags); break;
        default: run_sweep<1>(c, S, micro, diags); break;
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

__global__ void __launch_bounds__(kTileThreads, 1) tile_pass_kernel(const TileArgs A) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    int *s_hb = reinterpret_cast<int *>(sm + 16);
    float2 *cs = reinterpret_cast<float2 *>(sm + A.off_consts);
    float2 *roots = reinterpret_cast<float2 *>(sm + A.off_roots);
    float2 *bufs[2] = {reinterpret_cast<float2 *>(sm + A.off_buf0), reinterpret_cast<float2 *>(sm + A.off_buf1)};
    const TilePass &P = *A.pass;
    const int tid = threadIdx.x;
    const int L = P.L, H = P.H, T = P.T, RS = P.row_stride;
    const int rows = 1 << H;
    const uint32_t row_bytes = 8u << L;
    const long long total = A.n_tiles * (long long)A.batch;

    for (int i = tid; i < P.n_const; i += blockDim.x) cs[i] = A.consts[i];
    if (A.off_roots)
        for (int i = tid; i < kRootsEntries; i += blockDim.x) roots[i] = A.roots[i];
    if (tid < kMaxTileBits) s_hb[tid] = P.hb[tid];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    fence_proxy_async();
    __syncthreads();

    long long tile = blockIdx.x;
    if (tile >= total) return;
    const int warp = tid >> 5, lane = tid & 31;

    auto issue_load = [&](long long t, float2 *dstbuf, uint64_t *b) {
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        const float2 *src = A.src + bi * A.state_elems + tile_base(A, ti);
        if (lane == 0) mbar_arrive_expect_tx(b, (uint32_t)rows * row_bytes);
        __syncwarp();
        for (int r = lane; r < rows; r += 32) bulk_g2s(dstbuf + (size_t)r * RS, src + row_offset(r, H, s_hb), row_bytes, b);
    };
    auto issue_store = [&](long long t, float2 *srcbuf) {
        const long long bi = t / A.n_tiles, ti = t - bi * A.n_tiles;
        float2 *dst = A.dst + bi * A.state_elems + tile_base(A, ti);
        for (int r = lane; r < rows; r += 32) bulk_s2g(dst + row_offset(r, H, s_hb), srcbuf + (size_t)r * RS, row_bytes);
        bulk_commit();
    };

    if (warp == 0) issue_load(tile, bufs[0], &bar[0]);

    bool failed = false;
    int fail_k = 0;
    for (int k = 0; tile < total; tile += gridDim.x, ++k) {
        const int cur = k & 1;
        float2 *B = bufs[cur];
        const long long next = tile + gridDim.x;
        if (next < total && warp == 0) {
            bulk_wait_read0();   // buffer cur^1: its previous tile's stores have read smem
            __syncwarp();
            issue_load(next, bufs[cur ^ 1], &bar[cur ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bar[cur], (uint32_t)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            failed = true;
            fail_k = k;
            break;
        }
        const long long bi = tile / A.n_tiles, ti = tile - bi * A.n_tiles;
        SweepCtx c;
        c.L = L;
        c.T = T;
        c.RS = RS;
        c.hb = s_hb;
        c.buf = B;
        c.cs = cs;
        c.roots = roots;
        c.tile_gbase = tile_base(A, ti);
        for (int s = 0; s < P.n_sweeps; ++s) {
            const Sweep &S = P.sweeps[s];
            run_sweep_r(S.r, c, S, P.micro, P.diags);
            __syncthreads();
        }
        fence_proxy_async();
        __syncthreads();
        if (warp == 0) issue_store(tile, B);
    }
    if (failed) {
        if (tid == 0) atomicCAS(A.err, 0, (int)QS_ERR_TIMEOUT);
        // let this tile's load and the prefetched one land (bounded) before leaving
        if (warp == 0 && lane == 0) {
            mbar_wait_bounded(&bar[fail_k & 1], (uint32_t)((fail_k >> 1) & 1));
            if (tile + gridDim.x < total)
                mbar_wait_bounded(&bar[(fail_k + 1) & 1], (uint32_t)(((fail_k + 1) >> 1) & 1));
        }
    }
    if (warp == 0) bulk_wait_all0();
}

void tile_kernel_smem_config(int bytes) {
    cudaFuncSetAttribute(tile_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tile_pass(const TileArgs &A, int grid, int smem_bytes, cudaStream_t st) {
    tile_pass_kernel<<<grid, kTileThreads, smem_bytes, st>>>(A);
    return cudaGetLastError();
}

}  // namespace qs
