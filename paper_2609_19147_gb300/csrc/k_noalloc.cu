// qs_expect_noalloc: Pauli expectation values for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc.  A plug-in that runs inside a host
// application which owns every device allocation (a serving runtime or a
// simulation host with its own arena and memory accounting) is not allowed to
// allocate behind the host's back.  A process that has sized its state vector
// to fill the GPU has no room left for a late allocation, which would fail
// with out-of-memory.  And a real-time loop cannot take the implicit device
// synchronisation of cudaMalloc / cudaFree.  qs_expect needs device scratch
// for its per-block partial sums and allocates it on first use; this entry
// point runs the same reduction kernels with that scratch taken from a fixed
// array compiled into the library instead.
//
// The array is a file-scope static __device__ buffer of 694,272 bytes
// (678 KiB; limits: batch <= 16, n_terms <= 256): every GPU that loads the
// library holds it until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device (per
// CUDA context) looks the address up with cudaGetSymbolAddress, with that
// device current, and keeps it; that first call should come before any
// stream capture.  All calls share the one array and it keeps the previous
// call's contents, so calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it.  Nothing needs clearing
// between calls: every slot a call reads is written earlier in the same
// call.  The call is synchronous: it waits for its stream before it returns
// the sums in host memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "qs.h"
#include "qs_internal.h"
#include "qs_kernels.h"

namespace {

constexpr int kNaGrid = 152;      // reduction blocks per state
constexpr int kNaMaxBatch = 16;
constexpr int kNaMaxTerms = 256;
constexpr int kNaGroupTerms = 16;  // terms per reduction launch (kernel limit)

constexpr size_t kNaPartialDoubles = (size_t)kNaGrid * kNaMaxBatch * kNaGroupTerms * 2;
constexpr size_t kNaOutDoubles = (size_t)kNaMaxBatch * kNaMaxTerms * 2;
constexpr size_t kNaTermsBytes = sizeof(qs::PauliDev) * kNaMaxTerms;
constexpr size_t kNaBytes = (kNaPartialDoubles + kNaOutDoubles) * sizeof(double) + kNaTermsBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// The array's device address, looked up once per (device, context).  The
// module holding the array is loaded once per context, so a context created
// after cudaDeviceReset, or a caller's own non-primary context, can place it
// elsewhere: the address is kept per context, not only per device.
struct NaAddr {
    int dev;
    CUcontext ctx;
    unsigned char *addr;
};
std::mutex g_na_mu;
NaAddr g_na_addr[64];
int g_na_count = 0;
PFN_cuCtxGetCurrent_v4000 g_na_get_ctx = nullptr;

bool na_current_ctx(CUcontext *out) {
    if (!g_na_get_ctx) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        g_na_get_ctx = (PFN_cuCtxGetCurrent_v4000)fn;
    }
    return g_na_get_ctx(out) == CUDA_SUCCESS;
}

qs_status na_fail(qs_status s, const char *msg) {
    qs::set_last_error(msg);   // reported by qs_last_error()
    return s;
}

}  // namespace

extern "C" qs_status qs_expect_noalloc(const void *dev_state, int n, int batch, const qs_pauli *terms,
                                       size_t n_terms, double *out, void *cuda_stream) {
    if (!dev_state || !out || (n_terms && !terms)) return na_fail(QS_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > qs::kMaxQubits) return na_fail(QS_ERR_INVALID_ARG, "n must be in [1, 33]");
    if (batch < 1) return na_fail(QS_ERR_INVALID_ARG, "batch < 1");
    if (batch > kNaMaxBatch) return na_fail(QS_ERR_UNSUPPORTED, "batch exceeds the no-alloc maximum of 16");
    if (n_terms > (size_t)kNaMaxTerms)
        return na_fail(QS_ERR_UNSUPPORTED, "n_terms exceeds the no-alloc maximum of 256");
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // set-up, once per device and context, with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(QS_ERR_CUDA, "cudaGetDevice failed");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        CUcontext ctx = nullptr;
        if (!na_current_ctx(&ctx)) return na_fail(QS_ERR_CUDA, "cuCtxGetCurrent failed");
        for (int i = 0; i < g_na_count && ctx; ++i)
            if (g_na_addr[i].dev == dev && g_na_addr[i].ctx == ctx) base = g_na_addr[i].addr;
        if (!base) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return na_fail(QS_ERR_CUDA, "cudaGetSymbolAddress failed");
            base = static_cast<unsigned char *>(p);
            // the lookup binds the device's primary context when none was current
            if (!na_current_ctx(&ctx) || !ctx) return na_fail(QS_ERR_CUDA, "no current CUDA context");
            if (g_na_count < 64) g_na_addr[g_na_count++] = NaAddr{dev, ctx, base};
        }
    }
    double *d_partial = reinterpret_cast<double *>(base);
    double *d_out = d_partial + kNaPartialDoubles;
    qs::PauliDev *d_terms = reinterpret_cast<qs::PauliDev *>(d_out + kNaOutDoubles);

    // terms in index-bit space (qubit q = bit n-1-q), grouped by x mask
    qs::PauliDev ht[kNaMaxTerms];
    int ny[kNaMaxTerms];
    const uint64_t lim = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    for (size_t k = 0; k < n_terms; ++k) {
        if ((terms[k].x_mask & ~lim) || (terms[k].z_mask & ~lim))
            return na_fail(QS_ERR_INVALID_ARG, "Pauli mask outside the register");
        if (!std::isfinite(terms[k].coeff)) return na_fail(QS_ERR_INVALID_ARG, "non-finite Pauli coefficient");
    }
    int cnt = 0;
    bool used[kNaMaxTerms] = {false};
    int chunk_first[kNaMaxTerms], chunk_len[kNaMaxTerms], n_chunks = 0;
    uint64_t chunk_x[kNaMaxTerms];
    for (size_t k = 0; k < n_terms; ++k) {
        if (used[k]) continue;
        const uint64_t xq = terms[k].x_mask;
        for (size_t j = k; j < n_terms; ++j) {
            if (used[j] || terms[j].x_mask != xq) continue;
            if (n_chunks == 0 || chunk_x[n_chunks - 1] != xq || chunk_len[n_chunks - 1] == kNaGroupTerms ||
                chunk_first[n_chunks - 1] + chunk_len[n_chunks - 1] != cnt) {
                chunk_first[n_chunks] = cnt;
                chunk_len[n_chunks] = 0;
                chunk_x[n_chunks] = 0;
                n_chunks++;
            }
            qs::PauliDev t;
            t.coeff = terms[j].coeff;
            t.x = t.z = 0;
            for (int q = 0; q < n; ++q) {
                if ((terms[j].x_mask >> q) & 1) t.x |= 1ull << (n - 1 - q);
                if ((terms[j].z_mask >> q) & 1) t.z |= 1ull << (n - 1 - q);
            }
            chunk_x[n_chunks - 1] = xq;
            ht[cnt] = t;
            ny[cnt] = __builtin_popcountll(t.x & t.z) & 3;
            chunk_len[n_chunks - 1]++;
            cnt++;
            used[j] = true;
        }
    }
    for (int b = 0; b < batch; ++b) out[b] = 0.0;
    if (cnt == 0) return QS_OK;

    if (cudaMemcpyAsync(d_terms, ht, sizeof(qs::PauliDev) * cnt, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return na_fail(QS_ERR_CUDA, "copy of the Pauli terms failed");
    const long long elems = 1ll << n;
    for (int c = 0; c < n_chunks; ++c) {
        qs::ExpectArgs A;
        std::memset(&A, 0, sizeof A);
        A.psi = static_cast<const float2 *>(dev_state);
        A.lam = nullptr;
        A.state_elems = elems;
        A.batch = batch;
        A.xmask = ht[chunk_first[c]].x;
        A.n_terms = chunk_len[c];
        A.terms = d_terms + chunk_first[c];
        A.partial = d_partial;
        A.grid = kNaGrid;
        if (qs::launch_expect_group(A, st) != cudaSuccess) return na_fail(QS_ERR_CUDA, "reduction launch failed");
        // this chunk's sums: [b][j][re, im] at out slot offset batch * first * 2
        if (qs::launch_expect_finish(d_partial, d_out + (size_t)batch * chunk_first[c] * 2, batch, kNaGrid,
                                     chunk_len[c], st) != cudaSuccess)
            return na_fail(QS_ERR_CUDA, "finish launch failed");
    }
    static thread_local double hsum[kNaMaxBatch * kNaMaxTerms * 2];
    if (cudaMemcpyAsync(hsum, d_out, sizeof(double) * (size_t)batch * cnt * 2, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return na_fail(QS_ERR_CUDA, "copy of the results failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return na_fail(QS_ERR_CUDA, "stream synchronisation failed");
    for (int c = 0; c < n_chunks; ++c)
        for (int b = 0; b < batch; ++b)
            for (int j = 0; j < chunk_len[c]; ++j) {
                const int k = chunk_first[c] + j;
                double re = hsum[(size_t)batch * chunk_first[c] * 2 + ((size_t)b * chunk_len[c] + j) * 2];
                double im = hsum[(size_t)batch * chunk_first[c] * 2 + ((size_t)b * chunk_len[c] + j) * 2 + 1];
                double r = re;
                switch (ny[k]) {   // multiply by i^ny, keep the real part
                    case 1: r = -im; break;
                    case 2: r = -re; break;
                    case 3: r = im; break;
                    default: break;
                }
                out[b] += ht[k].coeff * r;
            }
    return QS_OK;
}
