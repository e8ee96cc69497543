// GF(2) affine permutation passes (Sec. 5.1 "GF(2) affine permutation
// gathers"): a run of X / CNOT / SWAP gates sends |x> to |M x ^ c>, so the
// whole run is one out-of-place amplitude permutation.
//   * perm_kernel   -- M is a bit permutation (SWAP / X runs, the QFT's final
//                      swaps).  Tile-transposed through shared memory: a tile
//                      spans the input's low bits and the input bits that land
//                      on the output's low bits, so reads and writes are both
//                      row-contiguous (a plain gather would read one 8-byte
//                      amplitude per 32-byte sector for a bit reversal).
//   * gather_kernel -- general invertible M (CNOT ladders, GHZ chains):
//                      out[y] = in[c' ^ XOR_k T_k[byte_k(y)]] with byte-sliced
//                      XOR tables of M^-1 in shared memory (integer-exact).
#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

// A tile is 2^TB input elements (TB <= 12).  Offsets are OR-linear in the
// element's bits, so per-CTA tables of the low 5 and the high TB-5 bits give
// every address in two lookups; the output-to-tile map is linear too, which
// folds the XOR mask into one constant.  Bit 0 is a tile bit on both sides,
// so loads and stores move two amplitudes (16 bytes) at a time.
constexpr int kPermMaxTB = 12;

__global__ void __launch_bounds__(256) perm_kernel(const PermArgs A) {
    __shared__ float2 sm[(1 << kPermMaxTB) + (1 << (kPermMaxTB - 5))];   // one pad slot per 32
    __shared__ uint64_t in_lo[32], in_hi[128], out_lo[32], out_hi[128];
    __shared__ int e_lo[32], e_hi[128];
    const int TB = A.TB, TS = 1 << TB, tid = threadIdx.x;
    if (tid < 32) {
        uint64_t a = 0, b = 0;
        int e = 0;
        for (int k = 0; k < 5 && k < TB; ++k)
            if ((tid >> k) & 1) {
                a |= 1ull << A.in_pos[k];
                b |= 1ull << A.out_pos_loc[k];
                e |= 1 << A.out_to_in[k];
            }
        in_lo[tid] = a;
        out_lo[tid] = b;
        e_lo[tid] = e;
    }
    if (tid < 128) {
        uint64_t a = 0, b = 0;
        int e = 0;
        for (int k = 5; k < TB; ++k)
            if ((tid >> (k - 5)) & 1) {
                a |= 1ull << A.in_pos[k];
                b |= 1ull << A.out_pos_loc[k];
                e |= 1 << A.out_to_in[k];
            }
        in_hi[tid] = a;
        out_hi[tid] = b;
        e_hi[tid] = e;
    }
    int fx = 0;   // tile element of the XOR mask's local part
    for (int k = 0; k < TB; ++k)
        if ((A.xor_loc >> k) & 1) fx |= 1 << A.out_to_in[k];
    __syncthreads();
    const long long tps = 1ll << A.n_outer;
    const long long total = tps * A.batch;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const long long b = t / tps, ti = t - b * tps;
        uint64_t xo = 0, yo = 0;
        for (int i = 0; i < A.n_outer; ++i)
            if ((ti >> i) & 1) {
                xo |= 1ull << A.outer_in[i];
                yo |= 1ull << A.outer_out[i];
            }
        yo ^= A.xor_outer;
        const float2 *src = A.src + b * A.state_elems;
        float2 *dst = A.dst + b * A.state_elems;
#pragma unroll 8
        for (int p = tid; p < (TS >> 1); p += 256) {
            const int e = p << 1;
            const uint64_t x = xo | in_lo[e & 31] | in_hi[e >> 5];
            const float4 v = *reinterpret_cast<const float4 *>(src + x);
            sm[e + (e >> 5)] = make_float2(v.x, v.y);
            sm[e + 1 + (e >> 5)] = make_float2(v.z, v.w);
        }
        __syncthreads();
#pragma unroll 8
        for (int p = tid; p < (TS >> 1); p += 256) {
            const int o = p << 1;
            const uint64_t y = yo | out_lo[o & 31] | out_hi[o >> 5];
            const int e0 = (e_lo[o & 31] | e_hi[o >> 5]) ^ fx;
            const int e1 = (e_lo[(o + 1) & 31] | e_hi[o >> 5]) ^ fx;
            const float2 v0 = sm[e0 + (e0 >> 5)], v1 = sm[e1 + (e1 >> 5)];
            *reinterpret_cast<float4 *>(dst + y) = make_float4(v0.x, v0.y, v1.x, v1.y);
        }
        __syncthreads();
    }
}

cudaError_t launch_perm(const PermArgs &A, cudaStream_t st) {
    long long total = (1ll << A.n_outer) * A.batch;
    long long grid = total < 152 * 8 ? total : 152 * 8;
    if (grid < 1) grid = 1;
    perm_kernel<<<(unsigned)grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) gather_kernel(const GatherArgs A) {
    __shared__ uint64_t tab[5][256];
    __shared__ uint64_t cc;
    const int ns = A.g->n_slices;
    for (int i = threadIdx.x; i < ns * 256; i += blockDim.x) tab[i >> 8][i & 255] = A.g->tab[i >> 8][i & 255];
    if (threadIdx.x == 0) cc = A.g->c;
    __syncthreads();
    const long long half = A.state_elems >> 1;
    const long long total = half * A.batch;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const uint64_t col0 = tab[0][1];
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += stride) {
        const long long b = w / half;
        const uint64_t y = (uint64_t)(w - b * half) << 1;
        uint64_t s0 = cc;
        for (int k = 0; k < ns; ++k) s0 ^= tab[k][(y >> (8 * k)) & 255];
        const uint64_t s1 = s0 ^ col0;
        const float2 *src = A.src + b * A.state_elems;
        const float2 v0 = src[s0], v1 = src[s1];
        *reinterpret_cast<float4 *>(A.dst + b * A.state_elems + y) = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
}

cudaError_t launch_gather(const GatherArgs &A, cudaStream_t st) {
    long long total = (A.state_elems >> 1) * A.batch;
    long long grid = (total + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    gather_kernel<<<(unsigned)grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace qs
