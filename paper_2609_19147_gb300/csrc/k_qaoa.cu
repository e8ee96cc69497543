// Batched QAOA MaxCut for states that fit in one CTA's shared memory
// (n <= 14: 2^14 complex64 = 128 KiB).
//
// One persistent launch covers every small instance: CTAs pull instance
// indices from a device work counter (atomicAdd; no waits).  Per instance the
// CTA keeps the whole state in shared memory:
//   |+>^n  ->  for l = 1..p:  psi_x *= exp(-i gamma_l cut(x))      (Sec. 3.2.3 QAOA,
//                             psi   <- (x)_q RX(2 beta_l) psi       e^{-i gamma H_C}, e^{-i beta H_M})
//   <C> = sum_x |psi_x|^2 cut(x)   (FP64)
// cut(x) = number of edges whose endpoint bits differ, computed once per
// instance into shared memory; exp(-i gamma_l k) comes from FP64-built tables.
#include <cuda_runtime.h>

#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

constexpr int kQaoaThreads = 512;

__global__ void __launch_bounds__(kQaoaThreads, 1) qaoa_small_kernel(const QaoaSmallArgs A) {
    extern __shared__ __align__(16) unsigned char smq[];
    float2 *psi = reinterpret_cast<float2 *>(smq);                         // 2^14
    unsigned char *cut = smq + (8 << 14);                                  // 2^14
    float2 *lut = reinterpret_cast<float2 *>(smq + (8 << 14) + (1 << 14));  // p * (kQaoaMaxEdges + 1)
    uint32_t *emask = reinterpret_cast<uint32_t *>(lut + kQaoaMaxP * (kQaoaMaxEdges + 1));
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
        const int n = I.n, ne = I.n_edges, p = A.p;
        const int dim = 1 << n;
        for (int e = tid; e < ne; e += kQaoaThreads) emask[e] = A.edge_masks[I.edge_off + e];
        for (int k = tid; k < p * (ne + 1); k += kQaoaThreads) {
            const int l = k / (ne + 1), c = k - l * (ne + 1);
            lut[l * (kQaoaMaxEdges + 1) + c] = A.luts[(size_t)I.lut_off + k];
        }
        __syncthreads();
        const float amp0 = rsqrtf((float)dim);
        for (int x = tid; x < dim; x += kQaoaThreads) {
            int c = 0;
            for (int e = 0; e < ne; ++e) c += __popc((uint32_t)x & emask[e]) & 1;
            cut[x] = (unsigned char)c;
            psi[x] = make_float2(amp0, 0.f);
        }
        __syncthreads();
        for (int l = 0; l < p; ++l) {
            const float2 *L = lut + l * (kQaoaMaxEdges + 1);
            for (int x = tid; x < dim; x += kQaoaThreads) {
                const float2 v = psi[x], w = L[cut[x]];
                psi[x] = make_float2(fmaf(v.x, w.x, -v.y * w.y), fmaf(v.x, w.y, v.y * w.x));
            }
            __syncthreads();
            // RX(2 beta) = [[c, i s], [i s, c]] with c = cos beta, s = -sin beta, on every qubit
            const float2 cs = A.mix[(size_t)I.mix_off + l];
            for (int q = 0; q < n; ++q) {
                for (int w = tid; w < (dim >> 1); w += kQaoaThreads) {
                    const int lo = w & ((1 << q) - 1);
                    const int x0 = ((w >> q) << (q + 1)) | lo, x1 = x0 | (1 << q);
                    const float2 a0 = psi[x0], a1 = psi[x1];
                    psi[x0] = make_float2(fmaf(cs.x, a0.x, -cs.y * a1.y), fmaf(cs.x, a0.y, cs.y * a1.x));
                    psi[x1] = make_float2(fmaf(cs.x, a1.x, -cs.y * a0.y), fmaf(cs.x, a1.y, cs.y * a0.x));
                }
                __syncthreads();
            }
        }
        double acc = 0.0;
        for (int x = tid; x < dim; x += kQaoaThreads) {
            const float2 v = psi[x];
            acc += (double)(v.x * v.x + v.y * v.y) * (double)cut[x];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int wi = 0; wi < kQaoaThreads / 32; ++wi) s += s_red[wi];
            A.out[I.out_idx] = s;
        }
        __syncthreads();
    }
}

int qaoa_small_smem_bytes() {
    return (8 << 14) + (1 << 14) + kQaoaMaxP * (kQaoaMaxEdges + 1) * 8 + kQaoaMaxEdges * 4;
}

cudaError_t launch_qaoa_small(const QaoaSmallArgs &A, int grid, cudaStream_t st) {
    const int smem = qaoa_small_smem_bytes();
    cudaFuncSetAttribute(qaoa_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    qaoa_small_kernel<<<grid, kQaoaThreads, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace qs
