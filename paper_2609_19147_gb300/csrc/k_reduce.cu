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

}  // namespace qs
