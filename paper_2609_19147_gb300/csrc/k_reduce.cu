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

__global__ void __launch_bounds__(kReduceThreads) expect_group_kernel(const ExpectArgs A) {
    __shared__ PauliDev terms[kMaxTermsPerGroup];
    __shared__ double red[kReduceThreads / 32][kMaxTermsPerGroup][2];
    const int nt = A.n_terms;
    if (threadIdx.x < nt) terms[threadIdx.x] = A.terms[threadIdx.x];
    __syncthreads();
    const int b = blockIdx.y;
    const float2 *psi = A.psi + (long long)b * A.state_elems;
    const float2 *phi = (A.lam ? A.lam : A.psi) + (long long)b * A.state_elems;
    const uint64_t xm = A.xmask;
    const int h = xm ? 63 - __clzll(xm) : -1;
    const long long nwork = xm ? (A.state_elems >> 1) : A.state_elems;
    double acc[kMaxTermsPerGroup][2];
    float fac[kMaxTermsPerGroup][2];
#pragma unroll
    for (int k = 0; k < kMaxTermsPerGroup; ++k) {
        acc[k][0] = acc[k][1] = 0.0;
        fac[k][0] = fac[k][1] = 0.f;
    }
    int cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        uint64_t x = (uint64_t)w;
        if (h >= 0) x = ((x >> h) << (h + 1)) | (x & ((1ull << h) - 1));   // bit h of x = 0
        const float2 px = psi[x], fx = phi[x];
        float2 v1, v2;
        uint64_t y = x ^ xm;
        // v1 = conj(phi[y]) psi[x], v2 = conj(phi[x]) psi[y]
        if (xm) {
            const float2 py = psi[y], fy = phi[y];
            v1 = make_float2(fy.x * px.x + fy.y * px.y, fy.x * px.y - fy.y * px.x);
            v2 = make_float2(fx.x * py.x + fx.y * py.y, fx.x * py.y - fx.y * py.x);
        } else {
            v1 = make_float2(fx.x * px.x + fx.y * px.y, fx.x * px.y - fx.y * px.x);
            v2 = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kMaxTermsPerGroup; ++k) {
            if (k < nt) {
                const float sx = (__popcll(x & terms[k].z) & 1) ? -1.f : 1.f;
                const float sy = (__popcll(y & terms[k].z) & 1) ? -1.f : 1.f;
                fac[k][0] += sx * v1.x + sy * v2.x;
                fac[k][1] += sx * v1.y + sy * v2.y;
            }
        }
        if (++cnt == 64) {
            cnt = 0;
#pragma unroll
            for (int k = 0; k < kMaxTermsPerGroup; ++k) {
                acc[k][0] += (double)fac[k][0];
                acc[k][1] += (double)fac[k][1];
                fac[k][0] = fac[k][1] = 0.f;
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kMaxTermsPerGroup; ++k) {
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
    expect_group_kernel<<<grid, kReduceThreads, 0, st>>>(A);
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
                                                        const PauliDev *terms_g, int n_terms) {
    extern __shared__ PauliDev terms[];
    for (int i = threadIdx.x; i < n_terms; i += blockDim.x) terms[i] = terms_g[i];
    __syncthreads();
    const int b = blockIdx.y;
    const float2 *p = psi + (long long)b * elems;
    float2 *l = lam + (long long)b * elems;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long y = (long long)blockIdx.x * blockDim.x + threadIdx.x; y < elems; y += stride) {
        float accr = 0.f, acci = 0.f;
        for (int k = 0; k < n_terms; ++k) {
            const uint64_t x = (uint64_t)y ^ terms[k].x;
            const float2 v = p[x];
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
                                   const PauliDev *terms, int n_terms, cudaStream_t st) {
    long long blocks = (elems + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    dim3 grid((unsigned)blocks, (unsigned)batch);
    pauli_sum_kernel<<<grid, 256, n_terms * sizeof(PauliDev), st>>>(psi, lam, elems, terms, n_terms);
    return cudaGetLastError();
}

}  // namespace qs
