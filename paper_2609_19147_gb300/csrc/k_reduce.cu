// Reductions: Pauli expectation values and adjoint-gradient overlaps, with
// FP64 accumulation (Sec. 3.2.1 "expectation value calculation for Pauli
// observables").
//
// For a group of Pauli terms sharing one x mask xm, one read pass computes
//   S_k = sum_x conj(phi[x ^ xm]) (-1)^popcount(x & zm_k) psi[x]
// for every term k of the group (phi = psi for <psi|P|psi>, phi = lambda for
// the adjoint method's <lambda|G|psi>).  The i^(#Y) factor is applied on the
// host.  Pairs (x, x ^ xm) are visited once, so each amplitude is read once.
// Per-thread sums are kept in FP32 for at most 64 amplitudes and then folded
// into FP64 accumulators; block partials are FP64.
#include <algorithm>

#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

constexpr int kMaxTermsPerGroup = 16;
constexpr int kReduceThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// NT: the group's term count rounded up to a power of two (registers and
// unrolled work scale with it, not with the 16-term maximum)
template <int NT>
__global__ void __launch_bounds__(kReduceThreads) expect_group_kernel(const ExpectArgs A) {
    __shared__ PauliDev terms[kMaxTermsPerGroup];
    __shared__ double red[kReduceThreads / 32][NT][2];
    const int nt = A.n_terms;
    if (threadIdx.x < nt) terms[threadIdx.x] = A.terms[threadIdx.x];
    __syncthreads();
    uint64_t zm[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) zm[k] = k < nt ? terms[k].z : 0;
    const int b = blockIdx.y;
    const long long bs = A.bstride ? A.bstride : A.state_elems;
    const float2 *psi = A.psi + (long long)b * bs;
    const float2 *phi = (A.lam ? A.lam : A.psi) + (long long)b * bs;
    const bool self = A.lam == nullptr;
    const uint64_t xm = A.xmask;
    const int h = xm ? 63 - __clzll(xm) : -1;
    const long long nwork = xm ? (A.state_elems >> 1) : A.state_elems;
    double acc[NT][2];
    float fac[NT][2];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        acc[k][0] = acc[k][1] = 0.0;
        fac[k][0] = fac[k][1] = 0.f;
    }
    int cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        uint64_t x = (uint64_t)w;
        if (h >= 0) x = ((x >> h) << (h + 1)) | (x & ((1ull << h) - 1));   // bit h of x = 0
        const float2 px = psi[x];
        const float2 fx = self ? px : phi[x];
        float2 v1, v2;
        uint64_t y = x ^ xm;
        // v1 = conj(phi[y]) psi[x], v2 = conj(phi[x]) psi[y]
        if (xm) {
            const float2 py = psi[y];
            const float2 fy = self ? py : phi[y];
            v1 = make_float2(fy.x * px.x + fy.y * px.y, fy.x * px.y - fy.y * px.x);
            v2 = make_float2(fx.x * py.x + fx.y * py.y, fx.x * py.y - fx.y * py.x);
        } else {
            v1 = make_float2(fx.x * px.x + fx.y * px.y, fx.x * px.y - fx.y * px.x);
            v2 = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            const float sx = (__popcll(x & zm[k]) & 1) ? -1.f : 1.f;
            const float sy = (__popcll(y & zm[k]) & 1) ? -1.f : 1.f;
            fac[k][0] += sx * v1.x + sy * v2.x;
            fac[k][1] += sx * v1.y + sy * v2.y;
        }
        if (++cnt == 64) {
            cnt = 0;
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                acc[k][0] += (double)fac[k][0];
                acc[k][1] += (double)fac[k][1];
                fac[k][0] = fac[k][1] = 0.f;
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        if (k < nt) {
            double r = warp_sum(acc[k][0] + (double)fac[k][0]);
            double i = warp_sum(acc[k][1] + (double)fac[k][1]);
            if (lane == 0) {
                red[warp][k][0] = r;
                red[warp][k][1] = i;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < nt * 2) {
        const int k = threadIdx.x >> 1, c = threadIdx.x & 1;
        double s = 0.0;
        for (int wi = 0; wi < kReduceThreads / 32; ++wi) s += red[wi][k][c];
        A.partial[(((long long)b * gridDim.x + blockIdx.x) * nt + k) * 2 + c] = s;
    }
}

cudaError_t launch_expect_group(const ExpectArgs &A, cudaStream_t st) {
    if (A.n_terms < 1 || A.n_terms > kMaxTermsPerGroup) return cudaErrorInvalidValue;
    dim3 grid((unsigned)A.grid, (unsigned)A.batch);
    if (A.n_terms == 1) expect_group_kernel<1><<<grid, kReduceThreads, 0, st>>>(A);
    else if (A.n_terms <= 2) expect_group_kernel<2><<<grid, kReduceThreads, 0, st>>>(A);
    else if (A.n_terms <= 4) expect_group_kernel<4><<<grid, kReduceThreads, 0, st>>>(A);
    else if (A.n_terms <= 8) expect_group_kernel<8><<<grid, kReduceThreads, 0, st>>>(A);
    else expect_group_kernel<16><<<grid, kReduceThreads, 0, st>>>(A);
    return cudaGetLastError();
}

__global__ void expect_finish_kernel(const double *partial, double *out, int grid, int n_terms) {
    const int b = blockIdx.x;
    for (int kc = threadIdx.x; kc < n_terms * 2; kc += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < grid; ++g) s += partial[(((long long)b * grid + g) * n_terms) * 2 + kc];
        out[(long long)b * n_terms * 2 + kc] = s;
    }
}

cudaError_t launch_expect_finish(const double *partial, double *out, int batch, int grid, int n_terms,
                                 cudaStream_t st) {
    expect_finish_kernel<<<batch, 64, 0, st>>>(partial, out, grid, n_terms);
    return cudaGetLastError();
}

// lam[y] = sum_k coeff_k i^(#Y_k) (-1)^popcount((y ^ x_k) & z_k) psi[y ^ x_k]
__global__ void __launch_bounds__(256) pauli_sum_kernel(const float2 *psi, float2 *lam, long long elems,
                                                        long long bstride, const PauliDev *terms_g, int n_terms) {
    extern __shared__ PauliDev terms[];
    for (int i = threadIdx.x; i < n_terms; i += blockDim.x) terms[i] = terms_g[i];
    __syncthreads();
    const int b = blockIdx.y;
    const float2 *p = psi + (long long)b * bstride;
    float2 *l = lam + (long long)b * bstride;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long y = (long long)blockIdx.x * blockDim.x + threadIdx.x; y < elems; y += stride) {
        float accr = 0.f, acci = 0.f;
        float2 v = make_float2(0.f, 0.f);
        for (int k = 0; k < n_terms; ++k) {
            const uint64_t x = (uint64_t)y ^ terms[k].x;
            if (k == 0 || terms[k].x != terms[k - 1].x) v = p[x];   // terms come sorted by x mask
            const int ny = __popcll(terms[k].x & terms[k].z) & 3;
            const float s = (__popcll(x & terms[k].z) & 1) ? -1.f : 1.f;
            const float c = (float)terms[k].coeff * s;
            // multiply v by c * i^ny
            float vr = v.x * c, vi = v.y * c;
            switch (ny) {
                case 0: accr += vr; acci += vi; break;
                case 1: accr -= vi; acci += vr; break;
                case 2: accr -= vr; acci -= vi; break;
                default: accr += vi; acci -= vr; break;
            }
        }
        l[y] = make_float2(accr, acci);
    }
}

template <int H>
__global__ void __launch_bounds__(256) pauli_sum_tile_kernel(const PsumTileArgs A) {
    constexpr int TB = 4 + H, TN = 1 << TB, ROWS = 1 << H;
    extern __shared__ float2 tile[];                 // TN amplitudes
    __shared__ uint64_t rowoff[ROWS];                // global bits of each row's high-bit pattern
    __shared__ float2 coef[kPsumMaxTerms];           // coeff_k i^ny_k (-1)^popcount(x_k & z_k), FP32
    __shared__ int xl[kPsumMaxTerms], zl[kPsumMaxTerms];   // x and z masks in tile-local bits
    __shared__ float sgn[kPsumMaxTerms];             // the tile's outer-bit parity of z_k, as a sign
    const int tid = threadIdx.x;
    for (int r = tid; r < ROWS; r += blockDim.x) {
        uint64_t o = 0;
        for (int k = 0; k < H; ++k)
            if ((r >> k) & 1) o |= 1ull << A.hb[k];
        rowoff[r] = o;
    }
    auto to_local = [&](uint64_t m) {
        int v = (int)(m & 15);
        for (int h = 0; h < H; ++h)
            if ((m >> A.hb[h]) & 1) v |= 1 << (4 + h);
        return v;
    };
    for (int k = tid; k < A.n_terms; k += blockDim.x) {
        const PauliDev t = A.terms[k];
        xl[k] = to_local(t.x);
        zl[k] = to_local(t.z);
        // (-1)^popcount((y ^ x) & z) = (-1)^popcount(x & z) (-1)^popcount(y & z)
        const double c = (__popcll(t.x & t.z) & 1) ? -t.coeff : t.coeff;
        const float cf = (float)c;
        switch (__popcll(t.x & t.z) & 3) {   // times i^ny
            case 0: coef[k] = make_float2(cf, 0.f); break;
            case 1: coef[k] = make_float2(0.f, cf); break;
            case 2: coef[k] = make_float2(-cf, 0.f); break;
            default: coef[k] = make_float2(0.f, -cf); break;
        }
    }
    const int b = blockIdx.y;
    const float2 *p = A.psi + (long long)b * A.bstride;
    float2 *l = A.lam + (long long)b * A.bstride;
    const long long n_tiles = A.elems >> TB;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        uint64_t g0 = 0;
        for (int i = 0; i < A.n_outer; ++i)
            if ((t >> i) & 1) g0 |= 1ull << A.outer[i];
        __syncthreads();   // the previous tile's reads are done
        for (int k = tid; k < A.n_terms; k += blockDim.x)
            sgn[k] = (__popcll(g0 & A.terms[k].z) & 1) ? -1.f : 1.f;
        // rows of 16 amplitudes are contiguous: 16-byte loads
        for (int e = tid; e < TN / 2; e += blockDim.x) {
            const int row = e >> 3, col = (e & 7) * 2;
            const float4 v = *reinterpret_cast<const float4 *>(p + (g0 | rowoff[row] | (uint64_t)col));
            tile[row * 16 + col] = make_float2(v.x, v.y);
            tile[row * 16 + col + 1] = make_float2(v.z, v.w);
        }
        __syncthreads();
        for (int j = tid; j < TN; j += blockDim.x) {
            float accr = 0.f, acci = 0.f;
            for (int k = 0; k < A.n_terms; ++k) {
                const float2 v = tile[j ^ xl[k]];
                const float sg = (__popc(j & zl[k]) & 1) ? -sgn[k] : sgn[k];
                const float cr = coef[k].x * sg, ci = coef[k].y * sg;
                accr = fmaf(cr, v.x, fmaf(-ci, v.y, accr));
                acci = fmaf(cr, v.y, fmaf(ci, v.x, acci));
            }
            const uint64_t y = g0 | rowoff[j >> 4] | (uint64_t)(j & 15);
            if (A.accumulate) {
                const float2 o = l[y];
                accr += o.x;
                acci += o.y;
            }
            l[y] = make_float2(accr, acci);
        }
    }
}

template <int H>
static cudaError_t psum_tile_launch(const PsumTileArgs &A, cudaStream_t st) {
    const int smem = (1 << (4 + H)) * (int)sizeof(float2);
    dim3 grid((unsigned)A.grid, (unsigned)A.batch);
    pauli_sum_tile_kernel<H><<<grid, 256, smem, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_pauli_sum_tile(const PsumTileArgs &A, cudaStream_t st) {
    if (A.H < 1 || A.H > 7 || A.grid < 1 || A.batch < 1 || A.n_terms < 1 || A.n_terms > kPsumMaxTerms ||
        (A.elems >> (4 + A.H)) < 1)
        return cudaErrorInvalidValue;
    switch (A.H) {
        case 1: return psum_tile_launch<1>(A, st);
        case 2: return psum_tile_launch<2>(A, st);
        case 3: return psum_tile_launch<3>(A, st);
        case 4: return psum_tile_launch<4>(A, st);
        case 5: return psum_tile_launch<5>(A, st);
        case 6: return psum_tile_launch<6>(A, st);
        default: return psum_tile_launch<7>(A, st);
    }
}

cudaError_t launch_apply_pauli_sum(const float2 *psi, float2 *lam, long long elems, int batch,
                                   const PauliDev *terms, int n_terms, cudaStream_t st, long long bstride) {
    long long blocks = (elems + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    dim3 grid((unsigned)blocks, (unsigned)batch);
    pauli_sum_kernel<<<grid, 256, n_terms * sizeof(PauliDev), st>>>(psi, lam, elems, bstride ? bstride : elems,
                                                                    terms, n_terms);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// X / Y / Z overlaps for the layer-wise adjoint gradient.  A thread takes the
// 2^k amplitudes of psi and lam that differ in the group bits; pairs across a
// group bit give the X and Y overlaps of that bit, single amplitudes the Z
// parts.
// ---------------------------------------------------------------------------
constexpr int kXyzThreads = 256;

template <int K>
__global__ void __launch_bounds__(kXyzThreads) xyz_kernel(const XyzArgs A) {
    constexpr int G = 1 << K;
    const int b = blockIdx.y;
    const float2 *psi = A.psi + (long long)b * A.bstride;
    const float2 *lam = A.lam + (long long)b * A.bstride;
    uint64_t gmask[K];
#pragma unroll
    for (int j = 0; j < K; ++j) gmask[j] = 1ull << A.gbit[j];
    // FP32 per-thread sums (the launch gives a thread at most 64 groups),
    // FP64 from the warp reduction on
    float f[kXyzSlots];
#pragma unroll
    for (int e = 0; e < kXyzSlots; ++e) f[e] = 0.f;
    const long long nwork = A.elems >> K;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        // base index: w with zeros inserted at the (ascending) group bits
        uint64_t x0 = (uint64_t)w;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int gb = A.gbit[j];
            x0 = ((x0 >> gb) << (gb + 1)) | (x0 & ((1ull << gb) - 1));
        }
        float2 p[G], l[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            uint64_t x = x0;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if ((i >> j) & 1) x |= gmask[j];
            p[i] = psi[x];
            l[i] = lam[x];
        }
        float tot = 0.f;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const float im = l[i].x * p[i].y - l[i].y * p[i].x;   // Im(conj(lam) psi)
            tot += im;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if ((i >> j) & 1) f[2 * kXyzGroup + j] += im;
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int i = 0; i < G; ++i) {
                if ((i >> j) & 1) continue;
                const int i1 = i | (1 << j);
                // A = conj(lam_i) psi_i1, B = conj(lam_i1) psi_i: Im<X> += Im A + Im B, Im<Y> += Re B - Re A
                const float are = l[i].x * p[i1].x + l[i].y * p[i1].y, aim = l[i].x * p[i1].y - l[i].y * p[i1].x;
                const float bre = l[i1].x * p[i].x + l[i1].y * p[i].y, bim = l[i1].x * p[i].y - l[i1].y * p[i].x;
                f[j] += aim + bim;
                f[kXyzGroup + j] += bre - are;
            }
#pragma unroll
        for (int q = 0; q < kXyzZBits; ++q)
            if (((A.zmask >> q) & 1) && ((x0 >> q) & 1)) f[3 * kXyzGroup + q] += tot;
        f[3 * kXyzGroup + kXyzZBits] += tot;
    }
    __shared__ double red[kXyzThreads / 32][kXyzSlots];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < kXyzSlots; ++e) {
        const double v = warp_sum((double)f[e]);
        if (lane == 0) red[warp][e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kXyzSlots; e += blockDim.x) {
        double v = 0.0;
        for (int wi = 0; wi < kXyzThreads / 32; ++wi) v += red[wi][e];
        A.partial[((long long)b * gridDim.x + blockIdx.x) * kXyzSlots + e] = v;
    }
}

int xyz_grid(long long elems, int k) {   // blocks per item: at most 64 groups per thread
    const long long per_block = (long long)kXyzThreads * 64;
    return (int)std::max(1ll, ((elems >> k) + per_block - 1) / per_block);
}

cudaError_t launch_xyz_overlaps(const XyzArgs &A, cudaStream_t st) {
    if (A.k < 1 || A.k > kXyzGroup || A.grid < xyz_grid(A.elems, A.k) || A.batch < 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)A.grid, (unsigned)A.batch);
    switch (A.k) {
        case 1: xyz_kernel<1><<<grid, kXyzThreads, 0, st>>>(A); break;
        case 2: xyz_kernel<2><<<grid, kXyzThreads, 0, st>>>(A); break;
        case 3: xyz_kernel<3><<<grid, kXyzThreads, 0, st>>>(A); break;
        default: xyz_kernel<4><<<grid, kXyzThreads, 0, st>>>(A); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// X / Y / Z overlaps over shared-memory tiles: up to 12 pair bits per read of
// the two states (the register-group kernel above takes 4).  A tile holds
// rows of 16 amplitudes (the low index bits) for 2^H combinations of the high
// tile bits; 16-byte chunks of a row are XOR-swizzled with the row's low 3
// bits.  Three sweeps give every thread a 16-amplitude group over 4 tile bits
// (low bits 0-3, high bits 0-3, high bits 4-7); the X / Y sums of a pair are
// 4 FMAs each, chained per thread in FP32 and reduced in FP64 per CTA.
// ---------------------------------------------------------------------------
constexpr int kXyzTThreads = 128;

__device__ __forceinline__ int xt_off(int row, int col) {   // float2 offset of (row, amplitude col)
    return (row << 4) | ((((col >> 1) ^ row) & 7) << 1) | (col & 1);
}
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tiles are double-buffered: the copies of tile k+1 are in flight while tile k
// is reduced.  Every sum stays in FP32 registers of its thread across the
// CTA's tiles (a thread adds a few thousand terms); FP64 starts at the block
// reduction (FP64 arithmetic is slow on this part, FP64 atomics slower).
template <int H>
__global__ void __launch_bounds__(kXyzTThreads) xyz_tile_kernel(const XyzTileArgs A) {
    constexpr int T = 4 + H, E = 1 << T, ROWS = 1 << H;
    extern __shared__ __align__(16) float2 xts[];   // [2 buffers][psi, lam][E]
    const int b = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 *psi = A.psi + (long long)b * A.bstride;
    const float2 *lam = A.lam + (long long)b * A.bstride;
    const long long n_tiles = A.elems >> T;
    int outer[kXyzZBits];
    int n_outer = 0;
    {
        uint64_t tb = 15ull;
        for (int k = 0; k < H; ++k) tb |= 1ull << A.hb[k];
        for (int q = 0; q < A.n; ++q)
            if (!((tb >> q) & 1)) outer[n_outer++] = q;
    }
    int tq[T];   // index bit of each tile bit
#pragma unroll
    for (int t = 0; t < T; ++t) tq[t] = t < 4 ? t : A.hb[t - 4];
    auto tile_base = [&](long long ti) {
        uint64_t g = 0;
        for (int i = 0; i < n_outer; ++i)
            if ((ti >> i) & 1) g |= 1ull << outer[i];
        return g;
    };
    auto issue = [&](long long ti, int buf) {
        const uint64_t base = tile_base(ti);
        float2 *ps = xts + (size_t)buf * 2 * E, *ls = ps + E;
#pragma unroll 4
        for (int e = tid; e < ROWS * 8; e += kXyzTThreads) {
            const int r = e >> 3, c4 = e & 7;
            uint64_t g = base;
#pragma unroll
            for (int k = 0; k < H; ++k)
                if ((r >> k) & 1) g |= 1ull << A.hb[k];
            const int o = xt_off(r, 2 * c4);
            cp_async16(ps + o, psi + g + 2 * c4);
            cp_async16(ls + o, lam + g + 2 * c4);
        }
        cp_async_commit();
    };
    float f[2 * kXyzTileBits], zacc[T], zq[kXyzZBits], ztot = 0.f;
#pragma unroll
    for (int e = 0; e < 2 * kXyzTileBits; ++e) f[e] = 0.f;
#pragma unroll
    for (int t = 0; t < T; ++t) zacc[t] = 0.f;
#pragma unroll
    for (int q = 0; q < kXyzZBits; ++q) zq[q] = 0.f;
    long long ti = blockIdx.x;
    if (ti < n_tiles) issue(ti, 0);
    for (int k = 0; ti < n_tiles; ti += gridDim.x, ++k) {
        const long long nxt = ti + gridDim.x;
        if (nxt < n_tiles) {
            issue(nxt, (k + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();   // tile k is in shared memory for every thread
        const float2 *ps = xts + (size_t)(k & 1) * 2 * E, *ls = ps + E;
        // Z parts (Im(conj(lam) psi) into the total and the set tile bits) come
        // with the first pair sweep, which holds 16 amplitudes per item
        float tot = 0.f;
        float zt[T];
#pragma unroll
        for (int t = 0; t < T; ++t) zt[t] = 0.f;
        // pair sweeps over 4 tile bits at a time
#pragma unroll
        for (int sw = 0; sw < 3; ++sw) {
            if (4 * sw >= T) break;
            const int g0 = 4 * sw, ng = (T - g0) < 4 ? (T - g0) : 4;
            const bool xy = ((A.xymask >> g0) & ((1u << ng) - 1)) != 0;
            if (sw > 0 && !xy) continue;
            const int items = E >> ng;
            for (int it = tid; it < items; it += kXyzTThreads) {
                const int lo = it & ((1 << g0) - 1), hi = it >> g0;
                const int e0 = lo | (hi << (g0 + ng));
                float2 p[16], l[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (j >= (1 << ng)) break;
                    const int e = e0 | (j << g0);
                    const int o = xt_off(e >> 4, e & 15);
                    p[j] = ps[o];
                    l[j] = ls[o];
                }
                if (sw == 0) {   // g0 = 0: j holds tile bits 0..ng-1, the item the rest
                    float im[16], it_sum = 0.f;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j >= (1 << ng)) break;
                        im[j] = l[j].x * p[j].y - l[j].y * p[j].x;
                        it_sum += im[j];
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (m >= ng) break;
                        float z = 0.f;
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j < (1 << ng) && ((j >> m) & 1)) z += im[j];
                        zt[m] += z;
                    }
#pragma unroll
                    for (int t = 4; t < T; ++t)
                        if ((e0 >> t) & 1) zt[t] += it_sum;
                    tot += it_sum;
                    if (!xy) continue;
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (m >= ng) break;
                    float ax = 0.f, ay = 0.f;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j >= (1 << ng) || ((j >> m) & 1)) continue;
                        const int j1 = j | (1 << m);
                        // Im A + Im B, Re B - Re A for A = conj(l_j) p_j1, B = conj(l_j1) p_j
                        ax = fmaf(l[j].x, p[j1].y, ax);
                        ax = fmaf(-l[j].y, p[j1].x, ax);
                        ax = fmaf(l[j1].x, p[j].y, ax);
                        ax = fmaf(-l[j1].y, p[j].x, ax);
                        ay = fmaf(l[j1].x, p[j].x, ay);
                        ay = fmaf(l[j1].y, p[j].y, ay);
                        ay = fmaf(-l[j].x, p[j1].x, ay);
                        ay = fmaf(-l[j].y, p[j1].y, ay);
                    }
                    f[g0 + m] += ax;
                    f[kXyzTileBits + g0 + m] += ay;
                }
            }
        }
        // this tile's Z sums: tile bits from zt; a bit outside the tile (zmask)
        // takes the thread's whole tile sum when the tile's base index has it set
        const uint64_t zb = A.zmask & tile_base(ti);
#pragma unroll
        for (int t = 0; t < T; ++t) zacc[t] += zt[t];
#pragma unroll
        for (int q = 0; q < kXyzZBits; ++q)
            if ((zb >> q) & 1) zq[q] += tot;
        ztot += tot;
        __syncthreads();   // every read of this buffer precedes its refill two tiles on
    }
    // slots: X / Y per tile bit, S_q per index bit (tile bits from zacc, others
    // from zq), total
    __shared__ double red[kXyzTThreads / 32][kXyzTSlots];
    for (int e = tid; e < (kXyzTThreads / 32) * kXyzTSlots; e += kXyzTThreads) (&red[0][0])[e] = 0.0;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 2 * kXyzTileBits; ++e) {
        const double v = warp_sum((double)f[e]);
        if (lane == 0) red[warp][e] = v;
    }
#pragma unroll
    for (int q = 0; q < kXyzZBits; ++q) {
        if (!((A.zmask >> q) & 1)) continue;   // uniform
        const double v = warp_sum((double)zq[q]);
        if (lane == 0) red[warp][2 * kXyzTileBits + q] = v;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const double v = warp_sum((double)zacc[t]);
        if (lane == 0) red[warp][2 * kXyzTileBits + tq[t]] += v;
    }
    {
        const double v = warp_sum((double)ztot);
        if (lane == 0) red[warp][2 * kXyzTileBits + kXyzZBits] = v;
    }
    __syncthreads();
    double *out = A.partial + ((long long)b * gridDim.x + blockIdx.x) * kXyzTSlots;
    for (int e = tid; e < kXyzTSlots; e += kXyzTThreads) {
        double v = 0.0;
        for (int wi = 0; wi < kXyzTThreads / 32; ++wi) v += red[wi][e];
        out[e] = v;
    }
}

template <int H>
static cudaError_t xyz_tile_launch(const XyzTileArgs &A, cudaStream_t st) {
    const int smem = 2 * 2 * (8 << (4 + H));   // two buffers of psi and lam tiles
    cudaFuncSetAttribute(xyz_tile_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 grid((unsigned)A.grid, (unsigned)A.batch);
    xyz_tile_kernel<H><<<grid, kXyzTThreads, smem, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_xyz_tile(const XyzTileArgs &A, cudaStream_t st) {
    if (A.H < 0 || A.H > 8 || A.grid < 1 || A.batch < 1 || (A.elems >> (4 + A.H)) < 1) return cudaErrorInvalidValue;
    switch (A.H) {
        case 0: return xyz_tile_launch<0>(A, st);
        case 1: return xyz_tile_launch<1>(A, st);
        case 2: return xyz_tile_launch<2>(A, st);
        case 3: return xyz_tile_launch<3>(A, st);
        case 4: return xyz_tile_launch<4>(A, st);
        case 5: return xyz_tile_launch<5>(A, st);
        case 6: return xyz_tile_launch<6>(A, st);
        case 7: return xyz_tile_launch<7>(A, st);
        default: return xyz_tile_launch<8>(A, st);
    }
}

// ---------------------------------------------------------------------------
// <psi| D |psi> for a diagonal D = sum_k c_k Z^{z_k}: per amplitude the FP32
// weight w(x) = sum_k c_k (-1)^popcount(x & z_k), one accumulator per thread
// (folded into FP64 every 64 amplitudes), one launch for any number of terms.
// ---------------------------------------------------------------------------
constexpr int kDiagTermsMax = 256;

__global__ void __launch_bounds__(256) diag_expect_kernel(const DiagExpectArgs A) {
    __shared__ uint64_t zs[kDiagTermsMax];
    __shared__ float cs[kDiagTermsMax];
    __shared__ double red[8];
    for (int k = threadIdx.x; k < A.n_terms; k += blockDim.x) {
        zs[k] = A.terms[k].z;
        cs[k] = (float)A.terms[k].coeff;
    }
    __syncthreads();
    const int b = blockIdx.y;
    const float4 *psi = reinterpret_cast<const float4 *>(A.psi + (long long)b * A.bstride);
    const long long npair = A.elems >> 1;   // two amplitudes per 16-byte load
    double acc = 0.0;
    float fac = 0.f;
    int cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < npair; w += stride) {
        const float4 v = psi[w];
        const uint64_t x0 = (uint64_t)w << 1;
        float w0 = 0.f, w1 = 0.f;
        for (int k = 0; k < A.n_terms; ++k) {
            const uint64_t z = zs[k];
            const float c = cs[k];
            w0 += (__popcll(x0 & z) & 1) ? -c : c;
            w1 += (__popcll((x0 | 1) & z) & 1) ? -c : c;
        }
        fac = fmaf(v.x * v.x + v.y * v.y, w0, fac);
        fac = fmaf(v.z * v.z + v.w * v.w, w1, fac);
        if (++cnt == 64) {
            acc += (double)fac;
            fac = 0.f;
            cnt = 0;
        }
    }
    acc = warp_sum(acc + (double)fac);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
        A.partial[((long long)b * gridDim.x + blockIdx.x) * 2] = v;   // (re, im) pairs for the finish kernel
        A.partial[((long long)b * gridDim.x + blockIdx.x) * 2 + 1] = 0.0;
    }
}

cudaError_t launch_diag_expect(const DiagExpectArgs &A, cudaStream_t st) {
    if (A.n_terms < 1 || A.n_terms > kDiagTermsMax || A.elems < 2 || A.grid < 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)A.grid, (unsigned)A.batch);
    diag_expect_kernel<<<grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace qs
