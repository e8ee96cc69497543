// Per-gate kernels: the plain structured per-gate path.
//
// One launch applies one gate, touching only the part of the state the gate
// changes: a general 2x2 on the target bit (optionally restricted to the
// control subspace: the "masked half-state update" of controlled gates), a
// phase multiply on the subspace where it is not 1 (diagonal gates), a swap
// of two quarters (SWAP), a 4x4 on two bits.  These are the GPU analogues of
// the paper's pure-tier structured dispatch (Sec. 3.2.2, Sec. 4.1 dispatch
// ablation): one read and one write of the touched amplitudes per gate.
// Accesses are coalesced; when index bit 0 is free each thread handles two
// consecutive indices with 16-byte loads.
#include "qs_internal.h"
#include "qs_kernels.h"

namespace qs {

__device__ __forceinline__ float2 pg_cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 pg_cmad(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

__device__ __forceinline__ uint64_t expand_index(uint64_t i, const PgArgs &A) {
    // insert a zero at each fixed position (ascending)
    for (int k = 0; k < A.n_fixed; ++k) {
        const int p = A.fixed_pos[k];
        const uint64_t lo = i & ((1ull << p) - 1);
        i = ((i >> p) << (p + 1)) | lo;
    }
    return i;
}

template <int V>
__device__ __forceinline__ void pg_apply(const PgOp &op, float2 *psi, uint64_t x) {
    // V consecutive indices x, x+1 (V = 2 only when bit 0 is free)
    switch (op.kind) {
        case PG_U1: {
            const uint64_t x1 = x | (1ull << op.t0);
            const float2 m0 = op.m[0], m1 = op.m[1], m2 = op.m[2], m3 = op.m[3];
            if (V == 2) {   // x even, bit 0 free: 16-byte accesses
                float4 A0 = *reinterpret_cast<const float4 *>(psi + x);
                float4 A1 = *reinterpret_cast<const float4 *>(psi + x1);
                float2 a0 = make_float2(A0.x, A0.y), b0 = make_float2(A0.z, A0.w);
                float2 a1 = make_float2(A1.x, A1.y), b1 = make_float2(A1.z, A1.w);
                float2 o0 = pg_cmad(m1, a1, pg_cmul(m0, a0)), p0 = pg_cmad(m1, b1, pg_cmul(m0, b0));
                float2 o1 = pg_cmad(m3, a1, pg_cmul(m2, a0)), p1 = pg_cmad(m3, b1, pg_cmul(m2, b0));
                *reinterpret_cast<float4 *>(psi + x) = make_float4(o0.x, o0.y, p0.x, p0.y);
                *reinterpret_cast<float4 *>(psi + x1) = make_float4(o1.x, o1.y, p1.x, p1.y);
            } else {
                float2 a0 = psi[x], a1 = psi[x1];
                psi[x] = pg_cmad(m1, a1, pg_cmul(m0, a0));
                psi[x1] = pg_cmad(m3, a1, pg_cmul(m2, a0));
            }
            break;
        }
        case PG_PHASE: {
            if (V == 2) {
                float4 A0 = *reinterpret_cast<const float4 *>(psi + x);
                int i0 = 0, i1 = 0;
                if (op.nbits_phase >= 1) {
                    i0 |= (int)((x >> op.t0) & 1);
                    i1 |= (int)(((x + 1) >> op.t0) & 1);
                }
                if (op.nbits_phase >= 2) {
                    i0 |= (int)((x >> op.t1) & 1) << 1;
                    i1 |= (int)(((x + 1) >> op.t1) & 1) << 1;
                }
                float2 o0 = pg_cmul(make_float2(A0.x, A0.y), op.m[i0]);
                float2 o1 = pg_cmul(make_float2(A0.z, A0.w), op.m[i1]);
                *reinterpret_cast<float4 *>(psi + x) = make_float4(o0.x, o0.y, o1.x, o1.y);
                break;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint64_t xv = x + v;
                int idx = 0;
                if (op.nbits_phase >= 1) idx |= (int)((xv >> op.t0) & 1);
                if (op.nbits_phase >= 2) idx |= (int)((xv >> op.t1) & 1) << 1;
                psi[xv] = pg_cmul(psi[xv], op.m[idx]);
            }
            break;
        }
        case PG_SWAP: {
            const uint64_t xa = x | (1ull << op.t0), xb = x | (1ull << op.t1);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float2 t = psi[xa + v];
                psi[xa + v] = psi[xb + v];
                psi[xb + v] = t;
            }
            break;
        }
        case PG_U2: {
            const uint64_t i1 = x | (1ull << op.t1), i2 = x | (1ull << op.t0), i3 = i1 | i2;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float2 a[4] = {psi[x + v], psi[i1 + v], psi[i2 + v], psi[i3 + v]};
                float2 o[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float2 acc = pg_cmul(op.m[r * 4], a[0]);
                    acc = pg_cmad(op.m[r * 4 + 1], a[1], acc);
                    acc = pg_cmad(op.m[r * 4 + 2], a[2], acc);
                    acc = pg_cmad(op.m[r * 4 + 3], a[3], acc);
                    o[r] = acc;
                }
                psi[x + v] = o[0];
                psi[i1 + v] = o[1];
                psi[i2 + v] = o[2];
                psi[i3 + v] = o[3];
            }
            break;
        }
        default:
            break;
    }
}

__global__ void __launch_bounds__(256) pergate_kernel(const PgArgs A) {
    const int yi = blockIdx.y;                  // state index over n_arrays * batch
    const int arr = yi / A.batch, b = yi - arr * A.batch;
    const PgOp &op = A.ops[A.op_stride ? b : 0];
    float2 *psi = A.psi[arr] + (long long)b * A.state_elems;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (A.vec2) {
        const long long nw = A.n_work >> 1;
        for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += stride) {
            const uint64_t x = expand_index((uint64_t)w << 1, A) | op.cval;
            pg_apply<2>(op, psi, x);
        }
    } else {
        for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < A.n_work; w += stride) {
            const uint64_t x = expand_index((uint64_t)w, A) | op.cval;
            pg_apply<1>(op, psi, x);
        }
    }
}

cudaError_t launch_pergate(const PgArgs &A, cudaStream_t st) {
    long long work = A.vec2 ? (A.n_work >> 1) : A.n_work;
    long long blocks = (work + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    dim3 grid((unsigned)blocks, (unsigned)(A.batch * A.n_arrays));
    pergate_kernel<<<grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}

__global__ void init_zero_kernel(float2 *psi, long long elems, int batch) {
    const long long total = elems * batch;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const long long r = i % elems;
        psi[i] = make_float2(r == 0 ? 1.f : 0.f, 0.f);
    }
}

cudaError_t launch_init_zero(float2 *psi, long long elems, int batch, cudaStream_t st) {
    long long total = elems * batch;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    init_zero_kernel<<<(unsigned)blocks, 256, 0, st>>>(psi, elems, batch);
    return cudaGetLastError();
}

}  // namespace qs
