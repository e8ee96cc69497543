// C ABI (include/qs.h): state handles, plan cache, executor, expectation and
// adjoint gradients.  All arithmetic on amplitudes runs in the CUDA kernels;
// this file validates, plans, routes buffers and launches.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>
#include <thread>
#include <atomic>

#include "qs.h"
#include "qs_internal.h"
#include "qs_kernels.h"
#include "qs_plan.h"
#include "qs_qasm.h"

using namespace qs;

namespace {
thread_local std::string g_last_error;

qs_status fail(qs_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

#define QS_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

struct DevicePlan {          // a plan uploaded to the device
    Plan host;
    std::vector<TilePass *> d_tile;
    std::vector<float2 *> d_consts;
    std::vector<GatherPass *> d_gather;
    PgOp *d_pg = nullptr;
    size_t bytes = 0;
    std::list<uint64_t>::iterator lru;
};

struct ProfRec {
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
};
struct PendingEv {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
};

float2 *g_roots[16] = {nullptr};   // per device
int g_num_sms[16] = {0};
std::mutex g_mu;

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

qs_status ensure_device_tables(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_roots[dev]) return QS_OK;
    std::vector<float2> r(kRootsEntries);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 256; ++c) {
            // exp(i pi c 2^(8k) / 2^32)
            double ang = pi * std::ldexp((double)c, 8 * k - 32);
            r[k * 256 + c] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
    float2 *d = nullptr;
    QS_CUDA(cudaMalloc(&d, kRootsEntries * sizeof(float2)));
    QS_CUDA(cudaMemcpy(d, r.data(), kRootsEntries * sizeof(float2), cudaMemcpyHostToDevice));
    cudaDeviceProp prop;
    QS_CUDA(cudaGetDeviceProperties(&prop, dev));
    g_num_sms[dev] = prop.multiProcessorCount;
    g_roots[dev] = d;
    return QS_OK;
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t plan_key(int n, int batch, const std::vector<RGate> &g, const qs_opts &o) {
    uint64_t h = fnv1a(&n, sizeof n);
    h = fnv1a(&batch, sizeof batch, h);
    h = fnv1a(&o, sizeof o, h);
    for (const RGate &r : g) {
        h = fnv1a(&r.kind, sizeof r.kind, h);
        h = fnv1a(r.q, sizeof r.q, h);
        h = fnv1a(r.p, sizeof r.p, h);
        if (r.kind == QS_U) h = fnv1a(r.dense, sizeof r.dense, h);
    }
    return h;
}

qs_opts default_opts(const qs_opts *o) {
    qs_opts d;
    std::memset(&d, 0, sizeof d);
    if (o) d = *o;
    return d;
}
}  // namespace

struct qs_state {
    int n = 0, batch = 1, dev = 0;
    long long elems = 0;
    float2 *home = nullptr;      // where results live between calls
    bool owned = false;
    float2 *scratch = nullptr;
    size_t scratch_bytes = 0;
    bool scratch_owned = false;
    cudaStream_t stream = nullptr;
    int *d_err = nullptr;
    double *d_partial = nullptr;
    size_t partial_cap = 0;      // doubles
    double *d_out = nullptr;
    size_t out_cap = 0;
    PauliDev *d_terms = nullptr;
    size_t terms_cap = 0;
    std::unordered_map<uint64_t, std::unique_ptr<DevicePlan>> cache;
    std::list<uint64_t> lru;
    size_t cache_bytes = 0;
    bool prof = false;
    std::map<std::string, ProfRec> prof_recs;
    std::vector<PendingEv> prof_pending;
    // page-locked staging for host -> device uploads (plans, term tables): a
    // copy from pageable memory waits for the stream's earlier work, one from
    // page-locked memory does not.  A chunk is reused once the event recorded
    // after its last copy has completed.
    struct Pinned {
        char *p = nullptr;
        size_t cap = 0, used = 0;
        cudaEvent_t ev = nullptr;
    };
    std::vector<Pinned> pinned;
    size_t pin_cur = 0;
    // qs_grad's (psi, lam) pair workspace, kept between calls: mapping and
    // unmapping 2 x batch x 2^n amplitudes every call cost more than the sweep
    float2 *grad_ws = nullptr;
    size_t grad_ws_bytes = 0;
};

namespace {

// Copy `bytes` from host memory to device memory on the state's stream
// without waiting for the stream: the data goes through a page-locked chunk.
qs_status h2d_async(qs_state *st, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return QS_OK;
    constexpr size_t kChunk = 4u << 20;
    constexpr size_t kMaxChunks = 16;
    const size_t need = (bytes + 255) & ~(size_t)255;
    qs_state::Pinned *c = nullptr;
    if (st->pin_cur < st->pinned.size() && st->pinned[st->pin_cur].used + need <= st->pinned[st->pin_cur].cap)
        c = &st->pinned[st->pin_cur];
    for (size_t i = 0; !c && i < st->pinned.size(); ++i) {   // a chunk whose copies have completed
        qs_state::Pinned &q = st->pinned[i];
        if (q.cap >= need && cudaEventQuery(q.ev) == cudaSuccess) {
            q.used = 0;
            st->pin_cur = i;
            c = &q;
        }
    }
    cudaGetLastError();   // cudaEventQuery's cudaErrorNotReady
    if (!c && st->pinned.size() < kMaxChunks) {
        qs_state::Pinned q;
        q.cap = std::max(kChunk, need);
        if (cudaMallocHost((void **)&q.p, q.cap) != cudaSuccess) {
            cudaGetLastError();
            return fail(QS_ERR_OOM, "page-locked staging allocation failed");
        }
        QS_CUDA(cudaEventCreateWithFlags(&q.ev, cudaEventDisableTiming));
        st->pinned.push_back(q);
        st->pin_cur = st->pinned.size() - 1;
        c = &st->pinned.back();
    }
    if (!c) {   // all chunks in flight: wait for the one with room
        for (size_t i = 0; i < st->pinned.size() && !c; ++i)
            if (st->pinned[i].cap >= need) {
                QS_CUDA(cudaEventSynchronize(st->pinned[i].ev));
                st->pinned[i].used = 0;
                st->pin_cur = i;
                c = &st->pinned[i];
            }
        if (!c) {   // larger than every chunk: plain copy
            QS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st->stream));
            return QS_OK;
        }
    }
    char *stage = c->p + c->used;
    c->used += need;
    std::memcpy(stage, src, bytes);
    QS_CUDA(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyHostToDevice, st->stream));
    QS_CUDA(cudaEventRecord(c->ev, st->stream));
    return QS_OK;
}

void free_pinned(qs_state *st) {
    for (auto &q : st->pinned) {
        if (q.ev) cudaEventDestroy(q.ev);
        if (q.p) cudaFreeHost(q.p);
    }
    st->pinned.clear();
}

void free_plan(qs_state *st, DevicePlan *dp) {
    for (auto p : dp->d_tile) cudaFreeAsync(p, st->stream);
    for (auto p : dp->d_consts)
        if (p) cudaFreeAsync(p, st->stream);
    for (auto p : dp->d_gather)
        if (p) cudaFreeAsync(p, st->stream);
    if (dp->d_pg) cudaFreeAsync(dp->d_pg, st->stream);
}

qs_status upload_plan(qs_state *st, DevicePlan &dp) {
    const Plan &p = dp.host;
    if (p.mode == QS_MODE_PERGATE) {
        if (!p.pg.empty()) {
            size_t b = p.pg.size() * sizeof(PgOp);
            QS_CUDA(cudaMallocAsync((void **)&dp.d_pg, b, st->stream));
            qs_status r = h2d_async(st, dp.d_pg, p.pg.data(), b);
            if (r != QS_OK) return r;
            dp.bytes += b;
        }
        return QS_OK;
    }
    dp.d_tile.assign(p.passes.size(), nullptr);
    dp.d_consts.assign(p.passes.size(), nullptr);
    dp.d_gather.assign(p.passes.size(), nullptr);
    for (size_t i = 0; i < p.passes.size(); ++i) {
        const HostPass &hp = p.passes[i];
        if (hp.type == HostPass::TILE) {
            QS_CUDA(cudaMallocAsync((void **)&dp.d_tile[i], sizeof(TilePass), st->stream));
            qs_status r = h2d_async(st, dp.d_tile[i], &hp.tile, sizeof(TilePass));
            if (r != QS_OK) return r;
            dp.bytes += sizeof(TilePass);
            if (!hp.consts.empty()) {
                size_t b = hp.consts.size() * sizeof(float2);
                QS_CUDA(cudaMallocAsync((void **)&dp.d_consts[i], b, st->stream));
                r = h2d_async(st, dp.d_consts[i], hp.consts.data(), b);
                if (r != QS_OK) return r;
                dp.bytes += b;
            }
        } else if (hp.type == HostPass::GATHER) {
            QS_CUDA(cudaMallocAsync((void **)&dp.d_gather[i], sizeof(GatherPass), st->stream));
            qs_status r = h2d_async(st, dp.d_gather[i], &hp.gather, sizeof(GatherPass));
            if (r != QS_OK) return r;
            dp.bytes += sizeof(GatherPass);
        }
    }
    return QS_OK;
}

DevicePlan *cache_lookup(qs_state *st, uint64_t key) {
    auto it = st->cache.find(key);
    if (it == st->cache.end()) return nullptr;
    st->lru.erase(it->second->lru);
    st->lru.push_front(key);
    it->second->lru = st->lru.begin();
    return it->second.get();
}

qs_status cache_insert(qs_state *st, uint64_t key, Plan &&plan, DevicePlan **out);

qs_status get_plan(qs_state *st, const std::vector<RGate> &gates, const qs_opts &o, int batch, DevicePlan **out) {
    uint64_t key = plan_key(st->n, batch, gates, o);
    if ((*out = cache_lookup(st, key)) != nullptr) return QS_OK;
    Plan plan;
    std::string err;
    qs_status s = (o.mode == QS_MODE_PERGATE) ? build_pergate_plan(st->n, gates, plan, err)
                                              : build_fused_plan(st->n, batch, gates, o, plan, err);
    if (s != QS_OK) return fail(s, err);
    return cache_insert(st, key, std::move(plan), out);
}

// upload a host plan and add it to the state's plan cache (bounded LRU)
qs_status cache_insert(qs_state *st, uint64_t key, Plan &&plan, DevicePlan **out) {
    std::unique_ptr<DevicePlan> dp(new DevicePlan());
    dp->host = std::move(plan);
    qs_status s = upload_plan(st, *dp);
    if (s != QS_OK) {
        free_plan(st, dp.get());
        return s;
    }
    st->lru.push_front(key);
    dp->lru = st->lru.begin();
    st->cache_bytes += dp->bytes;
    *out = dp.get();
    st->cache[key] = std::move(dp);
    // bound the cache (entries and bytes)
    while (st->cache.size() > 64 || st->cache_bytes > (256ull << 20)) {
        uint64_t victim = st->lru.back();
        if (victim == key) break;
        st->lru.pop_back();
        auto v = st->cache.find(victim);
        st->cache_bytes -= v->second->bytes;
        free_plan(st, v->second.get());
        st->cache.erase(v);
    }
    return QS_OK;
}

qs_status ensure_scratch(qs_state *st) {
    size_t need = (size_t)st->elems * st->batch * sizeof(float2);
    if (st->scratch && st->scratch_bytes >= need) return QS_OK;
    if (st->scratch && st->scratch_owned) cudaFree(st->scratch);
    st->scratch = nullptr;
    QS_CUDA(cudaMalloc(&st->scratch, need));
    st->scratch_bytes = need;
    st->scratch_owned = true;
    return QS_OK;
}

void prof_begin(qs_state *st, cudaEvent_t *a) {
    if (!st->prof) return;
    cudaEventCreate(a);
    cudaEventRecord(*a, st->stream);
}
void prof_end(qs_state *st, cudaEvent_t a, const char *name, double bytes) {
    if (!st->prof) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, st->stream);
    st->prof_pending.push_back({name, a, b, bytes});
}

qs_status check_err_word(qs_state *st) {
    int h = 0;
    QS_CUDA(cudaMemcpyAsync(&h, st->d_err, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    if (h != 0) {
        cudaMemsetAsync(st->d_err, 0, sizeof(int), st->stream);
        return fail(h, h == QS_ERR_TIMEOUT ? "a bounded device wait expired" : "device-side check failed");
    }
    return QS_OK;
}

// -------- executor --------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

qs_status get_encoder() {
    if (g_encode) return QS_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(QS_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return QS_OK;
}

qs_status encode_map(const TmaPlan &g, const void *base, bool swizzle, CUtensorMap *out) {
    qs_status s = get_encoder();
    if (s != QS_OK) return s;
    cuuint64_t gdim[5], gstr[4];
    cuuint32_t box[5], es[5];
    for (int d = 0; d < 5; ++d) {
        gdim[d] = g.gdim[d];
        box[d] = g.box[d];
        es[d] = 1;
        if (d >= 1) gstr[d - 1] = g.gstride[d];
    }
    CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void *>(base), gdim, gstr, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(QS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return QS_OK;
}

qs_status run_tile(qs_state *st, const DevicePlan &dp, size_t i, const float2 *src, float2 *dst, int batch) {
    const HostPass &hp = dp.host.passes[i];
    const TilePass &tp = hp.tile;
    TileArgs A;
    std::memset(&A, 0, sizeof A);
    A.pass = dp.d_tile[i];
    A.consts = dp.d_consts[i];
    if (dp.host.items > 1) {   // per-item constants, item after item
        if (batch % dp.host.items) return fail(QS_ERR_INTERNAL, "batch is not a multiple of the plan's items");
        A.const_stride = tp.n_const;
        A.const_group = batch / dp.host.items;
    }
    A.roots = g_roots[st->dev];
    A.src = src;
    A.dst = dst;
    A.state_elems = st->elems;
    A.n_tiles = 1ll << (st->n - tp.T);
    A.batch = batch;
    uint64_t tilebits = (1ull << tp.L) - 1;
    for (int k = 0; k < tp.H; ++k) tilebits |= 1ull << tp.hb[k];
    A.n_outer = 0;
    for (int b = 0; b < st->n; ++b)
        if (!((tilebits >> b) & 1)) A.outer_pos[A.n_outer++] = b;
    A.err = st->d_err;
    for (int k = 0; k < tp.n_sweeps; ++k) {
        if (tp.sweeps[k].dense) A.dense = 1;
        if (tp.sweeps[k].dense == DS_TF32X3) A.tmem = 1;
    }
    A.kset = 1;
    for (int k = 0; k < tp.n_micro; ++k) {
        const MicroOp &mo = tp.micro[k];
        if (mo.kind == MK_DIAG || mo.kind == MK_DIAGQ || mo.kind == MK_DIAGC || mo.kind == MK_QFT ||
            mo.kind == MK_QFTL || (mo.cmask && mo.kind != MK_DIAGC))
            A.needs_gidx = 1;
        if (!(mo.kind == MK_LAYER || mo.kind == MK_RXC || mo.kind == MK_U1R || mo.kind == MK_ROT || mo.kind == MK_H ||
              mo.kind == MK_U1 || mo.kind == MK_ZYZ ||
              mo.kind == MK_DIAG || mo.kind == MK_DIAGQ || mo.kind == MK_DIAGC))
            A.kset = 0;
    }
    // shared memory (after aligning the base to 1024 bytes in the kernel):
    // [mbarriers, flags, hb, contrib | descriptor | constants | roots | tile buffers]
    auto al = [](int v, int a) { return (v + a - 1) / a * a; };
    const int buf_bytes = 8 << tp.T;
    auto layout = [&](int const_copies) {
        int off = 256;
        A.off_desc = off;
        off += tp.n_sweeps * (int)sizeof(Sweep) + tp.n_micro * (int)sizeof(MicroOp) +
               kMaxDiag * (int)sizeof(DiagDesc);
        off += tp.n_sweeps * kItemTab * (8 + 4);   // item-address tables
        // dense tensor-core operands in the constants need 1024-byte alignment
        off = al(off, A.dense ? 1024 : 128);
        A.off_consts = off;
        // one item's constants (per copy, 16-entry aligned as the kernel indexes them)
        off = al(off + const_copies * al(tp.n_const, 16) * 8, 128);
        A.off_roots = 0;
        if (hp.uses_roots) {
            A.off_roots = off;
            off += kRootsEntries * 8;
        }
        off = al(off, 1024);
        A.off_buf0 = off;
        return off;
    };
    // Warp-specialised kernel (one CTA per SM, a producer warpgroup and two
    // consumer groups over three or more tile buffers) for 13-bit tiles with
    // 4- or 5-bit groups on the tensor-copy path, when three buffers fit.
    static int ws_env = -2;
    if (ws_env == -2) {
        const char *e = getenv("QS_TILE_WS");
        ws_env = e ? atoi(e) : -1;
    }
    const int ws_limit = 227 * 1024 - 1024;
    const int ws_copies = dp.host.items > 1 ? 2 : 1;
    if (ws_env != 0 && hp.tma.ok && tp.T == 13 && (tp.R == 4 || tp.R == 5) && !A.dense &&
        layout(ws_copies) + 3 * buf_bytes <= ws_limit) {
        A.ws = 1;
        A.ctas_per_sm = 1;
        A.n_buf = std::min(kMaxTileBuffers, std::min(4, (ws_limit - A.off_buf0) / buf_bytes));
        A.prefetch = 0;
    }
    int off = A.ws ? A.off_buf0 : layout(1);
    // Two co-resident CTAs per SM for 4-bit groups on 12- and 13-bit tiles,
    // and for 5-bit groups of layer/diagonal passes on 13-bit tiles (128
    // threads each, whose 255 registers just fill the register file twice):
    // while one CTA's warps run their sweeps, the other's copies are in flight
    // and its warps sit at a different phase of their own sweeps, so the SM's
    // shared-memory, FP32 and TMA work overlap instead of lining up behind
    // each barrier.  12-bit tiles keep three buffers per CTA; a 13-bit tile
    // (64 KB) leaves room for one buffer per CTA, loaded after the previous
    // tile's store has left it (no prefetch inside the CTA).  One CTA with
    // up to 6 buffers when two do not fit.
    int limit = 227 * 1024 - 1024;
    if (!A.ws) {
        int cps = ((tp.R == 4 && (tp.T == 12 || tp.T == 13)) || (tp.R == 5 && tp.T == 13 && A.kset && !A.dense)) ? 2 : 1;
        limit = (cps == 2 ? 113 * 1024 : 227 * 1024) - 1024;   // 1 KB for the base alignment
        int nb = std::min(cps == 2 ? 3 : 6, (limit - off) / buf_bytes);
        if (cps == 2 && nb < 1) {
            cps = 1;
            limit = 227 * 1024 - 1024;
            nb = std::min(6, (limit - off) / buf_bytes);
        }
        A.ctas_per_sm = cps;
        A.n_buf = std::min(nb, kMaxTileBuffers);
        if (A.n_buf < (cps == 2 ? 1 : 2)) return fail(QS_ERR_INTERNAL, "tile pass needs too much shared memory");
        A.prefetch = A.n_buf == 1 ? 0 : std::max(1, A.n_buf - 2);
    }
    off += A.n_buf * buf_bytes;
    if (off > limit) return fail(QS_ERR_INTERNAL, "tile pass needs too much shared memory");
    off += 1024;
    static int configured[16] = {0};
    if (configured[st->dev] < 227 * 1024) {
        tile_kernel_smem_config(227 * 1024);
        configured[st->dev] = 227 * 1024;
    }
    CUtensorMap tms, tmd;
    std::memset(&tms, 0, sizeof tms);
    std::memset(&tmd, 0, sizeof tmd);
    A.use_tma = hp.tma.ok ? 1 : 0;
    if (A.use_tma) {
        A.geo.ndims = hp.tma.ndims;
        A.geo.batch_dim = hp.tma.batch_dim;
        for (int d = 0; d < 5; ++d) {
            A.geo.kind[d] = hp.tma.kind[d];
            A.geo.off[d] = hp.tma.off[d];
            A.geo.w[d] = hp.tma.w[d];
        }
        qs_status s = encode_map(hp.tma, src, tp.swizzle != 0, &tms);
        if (s != QS_OK) return s;
        s = encode_map(hp.tma, dst, tp.swizzle != 0, &tmd);
        if (s != QS_OK) return s;
    }
    A.threads = (tp.R == 4 && tp.T >= 13 && A.ctas_per_sm == 1) ? 512 : (tp.R == 5 && A.ctas_per_sm == 2) ? 128 : 256;
    if (A.ws) A.threads = tile_ws_threads(tp.R);
    if (A.dense && (tp.R != 5 || A.ctas_per_sm != 1)) return fail(QS_ERR_INTERNAL, "dense pass without 5-bit groups");
    if (A.dense) A.threads = 256;
    {
        static int pf_env = -2, d_env = -2;
        if (pf_env == -2) {
            const char *e = getenv("QS_TILE_L2PF");
            pf_env = e ? atoi(e) : -1;
            e = getenv("QS_TILE_PREFETCH");
            d_env = e ? atoi(e) : -1;
        }
        // L2 warm-up of later tiles helps the multi-buffer CTAs; with one buffer
        // per CTA the prefetched lines were partly evicted before their load
        // (40% extra DRAM reads on 28q TFIM passes) and bought no time
        A.l2_prefetch = pf_env >= 0 ? pf_env : (A.n_buf == 1 ? 0 : 2);
        if (d_env > 0 && d_env < A.n_buf) A.prefetch = d_env;
    }
    long long total = A.n_tiles * batch;
    int grid = (int)std::min<long long>(total, (long long)A.ctas_per_sm * (g_num_sms[st->dev] > 0 ? g_num_sms[st->dev] : 148));
    cudaEvent_t ev;
    prof_begin(st, &ev);
    {
        cudaError_t e = launch_tile_pass(tp.R, A, &tms, &tmd, grid, off, st->stream);
        if (e != cudaSuccess)
            return fail(QS_ERR_CUDA, std::string("tile pass launch: ") + cudaGetErrorString(e) + " (smem=" +
                                         std::to_string(off) + " " + tile_kernel_attrs(tp.R, A) + ")");
    }
    prof_end(st, ev, "tile_pass", 16.0 * (double)st->elems * batch);
    return QS_OK;
}

qs_status run_perm(qs_state *st, const PermPass &pp, const float2 *src, float2 *dst, int batch) {
    const int n = st->n;
    PermArgs A;
    std::memset(&A, 0, sizeof A);
    A.src = src;
    A.dst = dst;
    A.state_elems = st->elems;
    A.batch = batch;
    const int L = std::min(pp.L, n);
    // input tile bits: low L, then input bits landing on output low bits, then
    // more low-positioned bits up to 12 tile bits
    std::vector<int> in_bits;
    uint64_t in_mask = 0;
    for (int b = 0; b < L; ++b) {
        in_bits.push_back(b);
        in_mask |= 1ull << b;
    }
    for (int b = L; b < n; ++b)
        if (pp.out_pos[b] < L) {
            in_bits.push_back(b);
            in_mask |= 1ull << b;
        }
    for (int b = L; b < n && (int)in_bits.size() < 12; ++b)
        if (!((in_mask >> b) & 1)) {
            in_bits.push_back(b);
            in_mask |= 1ull << b;
        }
    A.TB = (int)in_bits.size();
    for (int k = 0; k < A.TB; ++k) A.in_pos[k] = in_bits[k];
    std::vector<int> outs;
    uint64_t qmask = 0;
    for (int k = 0; k < A.TB; ++k) {
        outs.push_back(pp.out_pos[in_bits[k]]);
        qmask |= 1ull << pp.out_pos[in_bits[k]];
    }
    std::sort(outs.begin(), outs.end());
    for (int k = 0; k < A.TB; ++k) {
        A.out_pos_loc[k] = outs[k];
        for (int m = 0; m < A.TB; ++m)
            if (pp.out_pos[in_bits[m]] == outs[k]) A.out_to_in[k] = m;
        if ((pp.xor_mask >> outs[k]) & 1) A.xor_loc |= 1u << k;
    }
    A.n_outer = 0;
    for (int b = 0; b < n; ++b)
        if (!((in_mask >> b) & 1)) {
            A.outer_in[A.n_outer] = b;
            A.outer_out[A.n_outer] = pp.out_pos[b];
            A.n_outer++;
        }
    A.xor_outer = pp.xor_mask & ~qmask;
    cudaEvent_t ev;
    prof_begin(st, &ev);
    QS_CUDA(launch_perm(A, st->stream));
    prof_end(st, ev, "perm", 16.0 * (double)st->elems * batch);
    return QS_OK;
}

qs_status run_gather(qs_state *st, const GatherPass *dg, const float2 *src, float2 *dst, int batch) {
    GatherArgs A;
    A.g = dg;
    A.src = src;
    A.dst = dst;
    A.state_elems = st->elems;
    A.batch = batch;
    cudaEvent_t ev;
    prof_begin(st, &ev);
    QS_CUDA(launch_gather(A, st->stream));
    prof_end(st, ev, "gather", 16.0 * (double)st->elems * batch);
    return QS_OK;
}

void pg_fixed(const PgOp &op, int n, PgArgs &A) {
    uint64_t fixed = op.cmask;
    if (op.kind == PG_U1) fixed |= 1ull << op.t0;
    if (op.kind == PG_U2 || op.kind == PG_SWAP) fixed |= (1ull << op.t0) | (1ull << op.t1);
    A.n_fixed = 0;
    for (int b = 0; b < n; ++b)
        if ((fixed >> b) & 1) A.fixed_pos[A.n_fixed++] = b;
    A.n_work = 1ll << (n - A.n_fixed);
    A.vec2 = !(fixed & 1ull) && A.n_work >= 2;
}

double pg_bytes(const PgOp &op, int n) {
    // bytes the op reads + writes
    int fixed = __builtin_popcountll(op.cmask);
    double touched;
    switch (op.kind) {
        case PG_U1: touched = std::ldexp(1.0, n - fixed); break;
        case PG_SWAP: touched = std::ldexp(1.0, n - fixed - 1); break;
        case PG_U2: touched = std::ldexp(1.0, n); break;
        default: touched = std::ldexp(1.0, n - fixed); break;
    }
    return 16.0 * touched;
}

qs_status run_pergate(qs_state *st, const DevicePlan &dp, float2 *psi, int batch) {
    const Plan &p = dp.host;
    for (size_t i = 0; i < p.pg.size(); ++i) {
        PgArgs A;
        std::memset(&A, 0, sizeof A);
        A.ops = dp.d_pg + i;
        A.op_stride = 0;
        A.psi[0] = psi;
        A.n_arrays = 1;
        A.state_elems = st->elems;
        A.batch = batch;
        A.n = st->n;
        pg_fixed(p.pg[i], st->n, A);
        cudaEvent_t ev;
        prof_begin(st, &ev);
        QS_CUDA(launch_pergate(A, st->stream));
        prof_end(st, ev, "pergate", pg_bytes(p.pg[i], st->n) * batch);
    }
    return QS_OK;
}

// Execute a fused plan on `batch` states starting at `home` (results land
// back in `home`); out-of-place passes ping-pong with `other`.
qs_status run_fused(qs_state *st, const DevicePlan &dp, float2 *home, float2 *other, int batch) {
    const Plan &p = dp.host;
    int n_oop = 0, first_tile = -1;
    for (size_t i = 0; i < p.passes.size(); ++i) {
        if (p.passes[i].type != HostPass::TILE) n_oop++;
        else if (first_tile < 0) first_tile = (int)i;
    }
    // parity: results must end in `home`
    bool flip_tile = (n_oop % 2 == 1) && first_tile >= 0;
    bool final_copy = (n_oop % 2 == 1) && first_tile < 0;
    float2 *cur = home, *oth = other;
    for (size_t i = 0; i < p.passes.size(); ++i) {
        const HostPass &hp = p.passes[i];
        qs_status s = QS_OK;
        if (hp.type == HostPass::TILE) {
            if (flip_tile && (int)i == first_tile) {
                s = run_tile(st, dp, i, cur, oth, batch);
                std::swap(cur, oth);
            } else {
                s = run_tile(st, dp, i, cur, cur, batch);
            }
        } else if (hp.type == HostPass::PERM) {
            s = run_perm(st, hp.perm, cur, oth, batch);
            std::swap(cur, oth);
        } else {
            s = run_gather(st, dp.d_gather[i], cur, oth, batch);
            std::swap(cur, oth);
        }
        if (s != QS_OK) return s;
    }
    if (final_copy) {
        QS_CUDA(cudaMemcpyAsync(home, cur, (size_t)st->elems * batch * sizeof(float2), cudaMemcpyDeviceToDevice,
                                st->stream));
    }
    return QS_OK;
}

bool plan_needs_scratch(const Plan &p) {
    if (p.mode == QS_MODE_PERGATE) return false;
    for (auto &hp : p.passes)
        if (hp.type != HostPass::TILE) return true;
    return false;
}

qs_status apply_resolved(qs_state *st, const std::vector<RGate> &gates, const qs_opts &o, float2 *home, int batch) {
    DevicePlan *dp = nullptr;
    qs_status s = get_plan(st, gates, o, batch, &dp);
    if (s != QS_OK) return s;
    if (dp->host.mode == QS_MODE_PERGATE) return run_pergate(st, *dp, home, batch);
    if (plan_needs_scratch(dp->host)) {
        s = ensure_scratch(st);
        if (s != QS_OK) return s;
    }
    float2 *other = st->scratch ? st->scratch + (home - st->home) : nullptr;
    return run_fused(st, *dp, home, other, batch);
}

bool has_param_gates(const qs_gate *g, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (g[i].param_idx >= 0) return true;
    return false;
}

qs_status ensure_partial(qs_state *st, size_t doubles) {
    if (st->partial_cap >= doubles) return QS_OK;
    if (st->d_partial) cudaFree(st->d_partial);
    st->d_partial = nullptr;
    QS_CUDA(cudaMalloc(&st->d_partial, doubles * sizeof(double)));
    st->partial_cap = doubles;
    return QS_OK;
}
qs_status ensure_out(qs_state *st, size_t doubles) {
    if (st->out_cap >= doubles) return QS_OK;
    if (st->d_out) cudaFree(st->d_out);
    st->d_out = nullptr;
    QS_CUDA(cudaMalloc(&st->d_out, doubles * sizeof(double)));
    st->out_cap = doubles;
    return QS_OK;
}
qs_status ensure_terms(qs_state *st, size_t n) {
    if (st->terms_cap >= n) return QS_OK;
    if (st->d_terms) cudaFree(st->d_terms);
    st->d_terms = nullptr;
    QS_CUDA(cudaMalloc(&st->d_terms, n * sizeof(PauliDev)));
    st->terms_cap = n;
    return QS_OK;
}

// <psi_b| sum_k coeff_k Z^{z_k} |psi_b> for every batch item b (terms with
// x = 0, 1..256 of them) into d_dst[2 b] (real part; d_dst[2 b + 1] = 0),
// enqueued on the state's stream without waiting for the result.
qs_status diag_expect_async(qs_state *st, const std::vector<PauliDev> &hz, double *d_dst) {
    const int B = st->batch;
    const int grid = std::max(1, std::min<int>((int)((st->elems / 2 + 255) / 256), g_num_sms[st->dev] * 4));
    qs_status s = ensure_partial(st, (size_t)B * grid * 2);
    if (s == QS_OK) s = ensure_terms(st, hz.size());
    if (s != QS_OK) return s;
    s = h2d_async(st, st->d_terms, hz.data(), hz.size() * sizeof(PauliDev));
    if (s != QS_OK) return s;
    DiagExpectArgs A;
    std::memset(&A, 0, sizeof A);
    A.psi = st->home;
    A.elems = st->elems;
    A.bstride = st->elems;
    A.batch = B;
    A.n_terms = (int)hz.size();
    A.terms = st->d_terms;
    A.partial = st->d_partial;
    A.grid = grid;
    cudaEvent_t ev;
    prof_begin(st, &ev);
    QS_CUDA(launch_diag_expect(A, st->stream));
    prof_end(st, ev, "diag_expect", 8.0 * (double)st->elems * B);
    QS_CUDA(launch_expect_finish(st->d_partial, d_dst, B, grid, 1, st->stream));
    return QS_OK;
}

// Pauli terms in index-bit space
struct TermIdx {
    double coeff;
    uint64_t x, z;
    int ny;
};

qs_status convert_terms(int n, const qs_pauli *terms, size_t n_terms, std::vector<TermIdx> &out) {
    out.clear();
    const uint64_t lim = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    for (size_t k = 0; k < n_terms; ++k) {
        if ((terms[k].x_mask & ~lim) || (terms[k].z_mask & ~lim))
            return fail(QS_ERR_INVALID_ARG, "Pauli mask outside the register");
        if (!std::isfinite(terms[k].coeff)) return fail(QS_ERR_INVALID_ARG, "non-finite Pauli coefficient");
        TermIdx t;
        t.coeff = terms[k].coeff;
        t.x = t.z = 0;
        for (int q = 0; q < n; ++q) {
            if ((terms[k].x_mask >> q) & 1) t.x |= 1ull << (n - 1 - q);
            if ((terms[k].z_mask >> q) & 1) t.z |= 1ull << (n - 1 - q);
        }
        t.ny = __builtin_popcountll(t.x & t.z) & 3;
        out.push_back(t);
    }
    return QS_OK;
}

// S[b][k] (complex) = sum_x conj(phi[x ^ x_k]) (-1)^popcount(x & z_k) psi[x]
// for every term; results to host `S` (batch x n_terms x 2).
qs_status overlaps(qs_state *st, const float2 *psi, const float2 *phi, int batch, const std::vector<TermIdx> &t,
                   std::vector<double> &S, long long bstride = 0) {
    const int nt = (int)t.size();
    S.assign((size_t)batch * nt * 2, 0.0);
    if (nt == 0) return QS_OK;
    // group by x mask, chunks of <= 16 terms
    std::map<uint64_t, std::vector<int>> groups;
    for (int k = 0; k < nt; ++k) groups[t[k].x].push_back(k);
    const int grid = std::max(1, std::min<int>((int)((st->elems + 255) / 256), g_num_sms[st->dev] * 4));
    qs_status s = ensure_partial(st, (size_t)batch * grid * 16 * 2);
    if (s != QS_OK) return s;
    s = ensure_out(st, (size_t)batch * nt * 2);
    if (s != QS_OK) return s;
    s = ensure_terms(st, (size_t)nt);
    if (s != QS_OK) return s;
    std::vector<PauliDev> hterms;
    std::vector<std::pair<int, int>> chunks;   // (first index in hterms, count)
    std::vector<uint64_t> chunk_x;
    std::vector<int> order;
    for (auto &g : groups) {
        for (size_t i = 0; i < g.second.size(); i += 16) {
            int c = (int)std::min<size_t>(16, g.second.size() - i);
            chunks.push_back({(int)hterms.size(), c});
            chunk_x.push_back(g.first);
            for (int j = 0; j < c; ++j) {
                int k = g.second[i + j];
                hterms.push_back({t[k].coeff, t[k].x, t[k].z});
                order.push_back(k);
            }
        }
    }
    s = h2d_async(st, st->d_terms, hterms.data(), hterms.size() * sizeof(PauliDev));
    if (s != QS_OK) return s;
    for (size_t c = 0; c < chunks.size(); ++c) {
        ExpectArgs A;
        std::memset(&A, 0, sizeof A);
        A.psi = psi;
        A.lam = phi;
        A.state_elems = st->elems;
        A.bstride = bstride;
        A.batch = batch;
        A.xmask = chunk_x[c];
        A.n_terms = chunks[c].second;
        A.terms = st->d_terms + chunks[c].first;
        A.partial = st->d_partial;
        A.grid = grid;
        cudaEvent_t ev;
        prof_begin(st, &ev);
        QS_CUDA(launch_expect_group(A, st->stream));
        prof_end(st, ev, "expect", 8.0 * (double)st->elems * batch * (phi && phi != psi ? 2 : 1));
        // partial -> out slots [chunk offset .. ) in hterms order
        QS_CUDA(launch_expect_finish(st->d_partial, st->d_out + 0, batch, grid, A.n_terms, st->stream));
        std::vector<double> h((size_t)batch * A.n_terms * 2);
        QS_CUDA(cudaMemcpyAsync(h.data(), st->d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
        QS_CUDA(cudaStreamSynchronize(st->stream));
        for (int b = 0; b < batch; ++b)
            for (int j = 0; j < A.n_terms; ++j) {
                int k = order[chunks[c].first + j];
                S[((size_t)b * nt + k) * 2] = h[((size_t)b * A.n_terms + j) * 2];
                S[((size_t)b * nt + k) * 2 + 1] = h[((size_t)b * A.n_terms + j) * 2 + 1];
            }
    }
    return check_err_word(st);
}

// multiply (re, im) by i^ny
inline void times_i_pow(double &re, double &im, int ny) {
    double r = re, i = im;
    switch (ny & 3) {
        case 0: break;
        case 1: re = -i; im = r; break;
        case 2: re = -r; im = -i; break;
        default: re = i; im = -r; break;
    }
}

}  // namespace

namespace qs {
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace qs

// ===========================================================================
// exported C ABI
// ===========================================================================
extern "C" {

const char *qs_last_error(void) { return g_last_error.c_str(); }

const char *qs_version(void) { return "qs 0.1 (sm_103a)"; }

static qs_status make_state(int n, int batch, qs_state **out) {
    if (!out) return fail(QS_ERR_INVALID_ARG, "out == NULL");
    *out = nullptr;
    if (batch < 1) return fail(QS_ERR_INVALID_ARG, "batch < 1");
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_UNSUPPORTED, "n must be in [1, 33]");
    std::unique_ptr<qs_state> st(new qs_state());
    st->n = n;
    st->batch = batch;
    st->elems = 1ll << n;
    st->dev = current_device();
    qs_status s = ensure_device_tables(st->dev);
    if (s != QS_OK) return s;
    QS_CUDA(cudaMalloc(&st->d_err, sizeof(int)));
    QS_CUDA(cudaMemset(st->d_err, 0, sizeof(int)));
    *out = st.release();
    return QS_OK;
}

qs_status qs_alloc(int n, int batch, qs_state **out) {
    qs_state *st = nullptr;
    qs_status s = make_state(n, batch, &st);
    if (s != QS_OK) return s;
    size_t bytes = (size_t)st->elems * batch * sizeof(float2);
    cudaError_t e = cudaMalloc(&st->home, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(st->d_err);
        delete st;
        return fail(QS_ERR_OOM, "cudaMalloc of the state failed");
    }
    st->owned = true;
    e = (cudaError_t)launch_init_zero(st->home, st->elems, batch, st->stream);
    if (e != cudaSuccess) {
        qs_free(st);
        return fail(QS_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = st;
    return QS_OK;
}

qs_status qs_wrap(void *dev_ptr, int n, int batch, void *cuda_stream, qs_state **out) {
    if (!dev_ptr) return fail(QS_ERR_INVALID_ARG, "dev_ptr == NULL");
    if (((uintptr_t)dev_ptr) & 15) return fail(QS_ERR_INVALID_ARG, "dev_ptr must be 16-byte aligned");
    qs_state *st = nullptr;
    qs_status s = make_state(n, batch, &st);
    if (s != QS_OK) return s;
    st->home = (float2 *)dev_ptr;
    st->owned = false;
    st->stream = (cudaStream_t)cuda_stream;
    *out = st;
    return QS_OK;
}

qs_status qs_free(qs_state *st) {
    if (!st) return QS_OK;
    cudaStreamSynchronize(st->stream);
    for (auto &kv : st->cache) free_plan(st, kv.second.get());
    cudaStreamSynchronize(st->stream);
    for (auto &pe : st->prof_pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    if (st->owned && st->home) cudaFree(st->home);
    if (st->scratch_owned && st->scratch) cudaFree(st->scratch);
    if (st->d_err) cudaFree(st->d_err);
    if (st->d_partial) cudaFree(st->d_partial);
    if (st->d_out) cudaFree(st->d_out);
    if (st->d_terms) cudaFree(st->d_terms);
    if (st->grad_ws) cudaFree(st->grad_ws);
    free_pinned(st);
    delete st;
    return QS_OK;
}

qs_status qs_set_stream(qs_state *st, void *cuda_stream) {
    if (!st) return fail(QS_ERR_INVALID_ARG, "st == NULL");
    st->stream = (cudaStream_t)cuda_stream;
    return QS_OK;
}

qs_status qs_set_scratch(qs_state *st, void *dev_ptr, size_t bytes) {
    if (!st) return fail(QS_ERR_INVALID_ARG, "st == NULL");
    if (dev_ptr && (((uintptr_t)dev_ptr) & 15)) return fail(QS_ERR_INVALID_ARG, "scratch must be 16-byte aligned");
    if (dev_ptr && bytes < (size_t)st->elems * st->batch * sizeof(float2))
        return fail(QS_ERR_INVALID_ARG, "scratch smaller than the state");
    if (st->scratch_owned && st->scratch) cudaFree(st->scratch);
    st->scratch = (float2 *)dev_ptr;
    st->scratch_bytes = dev_ptr ? bytes : 0;
    st->scratch_owned = false;
    return QS_OK;
}

qs_status qs_device_ptr(const qs_state *st, void **out) {
    if (!st || !out) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    *out = st->home;
    return QS_OK;
}

qs_status qs_init_zero(qs_state *st) {
    if (!st) return fail(QS_ERR_INVALID_ARG, "st == NULL");
    QS_CUDA(launch_init_zero(st->home, st->elems, st->batch, st->stream));
    return QS_OK;
}

qs_status qs_set_amplitudes(qs_state *st, const void *src, int is_device) {
    if (!st || !src) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    size_t bytes = (size_t)st->elems * st->batch * sizeof(float2);
    QS_CUDA(cudaMemcpyAsync(st->home, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    return QS_OK;
}

qs_status qs_get_amplitudes(const qs_state *st, void *dst, int is_device) {
    if (!st || !dst) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    size_t bytes = (size_t)st->elems * st->batch * sizeof(float2);
    QS_CUDA(cudaMemcpyAsync(dst, st->home, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    return QS_OK;
}

namespace {
// Upload and run a plan built outside the cache (per-item plans of the
// adjoint sweep are used once); the device copies are freed in stream order.
qs_status run_host_plan(qs_state *st, Plan &&plan, float2 *home, int batch) {
    DevicePlan dp;
    dp.host = std::move(plan);
    qs_status s = upload_plan(st, dp);
    if (s == QS_OK) {
        if (dp.host.mode == QS_MODE_PERGATE) {
            s = run_pergate(st, dp, home, batch);
        } else {
            if (plan_needs_scratch(dp.host)) s = ensure_scratch(st);
            if (s == QS_OK) s = run_fused(st, dp, home, st->scratch ? st->scratch + (home - st->home) : nullptr, batch);
        }
    }
    free_plan(st, &dp);
    return s;
}

// Fused plans for many gate lists at once, on up to 16 host threads (the
// planner keeps no shared state between calls).
// item_plans: the lists are the items of one batch, whose plans are to be
// merged (see build_fused_plan).
qs_status build_plans_parallel(int n, int batch, const std::vector<std::vector<RGate>> &lists, const qs_opts &o,
                               std::vector<Plan> &out, std::string &err, bool item_plans) {
    out.assign(lists.size(), Plan());
    std::vector<qs_status> st(lists.size(), QS_OK);
    std::vector<std::string> errs(lists.size());
    std::atomic<size_t> next(0);
    auto work = [&]() {
        for (size_t i; (i = next.fetch_add(1)) < lists.size();)
            st[i] = build_fused_plan(n, batch, lists[i], o, out[i], errs[i], item_plans);
    };
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const size_t nt = std::min<size_t>(hw, lists.size());
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    for (size_t i = 0; i < lists.size(); ++i)
        if (st[i] != QS_OK) {
            err = errs[i];
            return st[i];
        }
    return QS_OK;
}
}  // namespace

qs_status qs_apply_circuit(qs_state *st, const qs_gate *gates, size_t n_gates, const double *params, int n_params,
                           const qs_opts *opts) {
    if (!st) return fail(QS_ERR_INVALID_ARG, "st == NULL");
    if (n_params < 0) return fail(QS_ERR_INVALID_ARG, "n_params < 0");
    qs_opts o = default_opts(opts);
    if (o.mode != QS_MODE_FUSED && o.mode != QS_MODE_PERGATE) return fail(QS_ERR_INVALID_ARG, "unknown mode");
    const bool per_item = params && has_param_gates(gates, n_gates) && st->batch > 1;
    // validate every batch item before launching anything
    std::vector<std::vector<RGate>> resolved(per_item ? st->batch : 1);
    for (size_t bi = 0; bi < resolved.size(); ++bi) {
        std::string err;
        qs_status s = resolve_gates(st->n, gates, n_gates, params, n_params, (int)bi, resolved[bi], err);
        if (s != QS_OK) return fail(s, err);
    }
    if (n_gates == 0) return QS_OK;
    if (!per_item) return apply_resolved(st, resolved[0], o, st->home, st->batch);
    if (o.mode == QS_MODE_FUSED) {
        // per-item parameters: plans for every item (built on host threads) are
        // merged into one batched plan with per-item constants when they agree
        // in structure; otherwise each item runs its own plan
        std::vector<uint64_t> keys(st->batch);
        uint64_t ck = 1469598103934665603ull;
        for (int bi = 0; bi < st->batch; ++bi) {
            keys[bi] = plan_key(st->n, 1, resolved[bi], o);
            ck = fnv1a(&keys[bi], sizeof keys[bi], ck);
        }
        DevicePlan *dp = cache_lookup(st, ck);
        qs_status s = QS_OK;
        std::vector<Plan> built;
        if (!dp) {
            bool all_cached = true;
            for (int bi = 0; bi < st->batch && all_cached; ++bi) all_cached = st->cache.count(keys[bi]) != 0;
            if (!all_cached) {
                std::string err;
                s = build_plans_parallel(st->n, 1, resolved, o, built, err, true);
                if (s != QS_OK) return fail(s, err);
                Plan merged;
                if (merge_item_plans(built, merged, st->batch)) {
                    s = cache_insert(st, ck, std::move(merged), &dp);
                    if (s != QS_OK) return s;
                }
            }
        }
        if (dp) {   // one launch per pass for the whole batch
            if (plan_needs_scratch(dp->host)) {
                s = ensure_scratch(st);
                if (s != QS_OK) return s;
            }
            return run_fused(st, *dp, st->home, st->scratch, st->batch);
        }
        for (int bi = 0; bi < st->batch; ++bi) {   // each item with its own plan, run as soon as it is found
            DevicePlan *d = cache_lookup(st, keys[bi]);
            if (!d) {
                if ((size_t)bi >= built.size()) return fail(QS_ERR_INTERNAL, "per-item plan missing");
                s = cache_insert(st, keys[bi], std::move(built[bi]), &d);
                if (s != QS_OK) return s;
            }
            float2 *home = st->home + (size_t)bi * st->elems;
            if (plan_needs_scratch(d->host)) {
                s = ensure_scratch(st);
                if (s != QS_OK) return s;
            }
            s = run_fused(st, *d, home, st->scratch ? st->scratch + (home - st->home) : nullptr, 1);
            if (s != QS_OK) return s;
        }
        return QS_OK;
    }
    for (int bi = 0; bi < st->batch; ++bi) {
        qs_status s = apply_resolved(st, resolved[bi], o, st->home + (size_t)bi * st->elems, 1);
        if (s != QS_OK) return s;
    }
    return QS_OK;
}

qs_status qs_expect(qs_state *st, const qs_pauli *terms, size_t n_terms, double *out) {
    if (!st || !out || (n_terms && !terms)) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    std::vector<TermIdx> all;
    qs_status s = convert_terms(st->n, terms, n_terms, all);
    if (s != QS_OK) return s;
    // Z-only terms (two or more) take one diagonal-weight pass; the rest go
    // through the Pauli-group reductions
    std::vector<TermIdx> t, dz;
    for (auto &x : all) (x.x == 0 && st->elems >= 2 ? dz : t).push_back(x);
    if (dz.size() < 2 || dz.size() > 256) {
        t.insert(t.end(), dz.begin(), dz.end());
        dz.clear();
    }
    std::vector<double> S;
    s = overlaps(st, st->home, nullptr, st->batch, t, S);
    if (s != QS_OK) return s;
    for (int b = 0; b < st->batch; ++b) {
        double e = 0.0;
        for (size_t k = 0; k < t.size(); ++k) {
            double re = S[((size_t)b * t.size() + k) * 2], im = S[((size_t)b * t.size() + k) * 2 + 1];
            times_i_pow(re, im, t[k].ny);
            e += t[k].coeff * re;
        }
        out[b] = e;
    }
    if (!dz.empty()) {
        const int B = st->batch;
        std::vector<PauliDev> hz;
        for (auto &x : dz) hz.push_back({x.coeff, 0, x.z});
        s = ensure_out(st, (size_t)B * 2);
        if (s == QS_OK) s = diag_expect_async(st, hz, st->d_out);
        if (s != QS_OK) return s;
        std::vector<double> r((size_t)B * 2);
        QS_CUDA(cudaMemcpyAsync(r.data(), st->d_out, r.size() * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
        QS_CUDA(cudaStreamSynchronize(st->stream));
        for (int b = 0; b < B; ++b) out[b] += r[(size_t)b * 2];
    }
    return QS_OK;
}

namespace {
// The inverse of a resolved gate as gates of the library, in application
// order: 1q gates as their conjugate-transposed 2x2 (QS_U), angle gates with
// the angle negated, ISWAP^dagger = ISWAP (Z (x) Z), the rest self-inverse.
void invert_gate(const RGate &g, std::vector<RGate> &out) {
    if (g.nw == 1) {
        cd M[4];
        gate_matrix(g, M);
        RGate u = g;
        u.kind = QS_U;
        u.dense[0] = std::conj(M[0]);
        u.dense[1] = std::conj(M[2]);
        u.dense[2] = std::conj(M[1]);
        u.dense[3] = std::conj(M[3]);
        out.push_back(u);
        return;
    }
    switch (g.kind) {
        case QS_CRX: case QS_CRY: case QS_CRZ: case QS_CP: case QS_RZZ: case QS_RXX: case QS_RYY: {
            RGate r = g;
            r.p[0] = -g.p[0];
            out.push_back(r);
            return;
        }
        case QS_ISWAP: {
            for (int w = 0; w < 2; ++w) {
                RGate z;
                z.kind = QS_Z;
                z.nw = 1;
                z.q[0] = g.q[w];
                z.b[0] = g.b[w];
                out.push_back(z);
            }
            out.push_back(g);
            return;
        }
        default:   // CX, CY, CZ, CH, SWAP, CCX, CSWAP
            out.push_back(g);
            return;
    }
}
}  // namespace


namespace {
// Tile bit sets for lam = H psi on shared-memory tiles: every term's x mask
// must lie in the 4 low index bits plus the H high bits of one pass.  Terms
// are regrouped pass by pass (diagonal terms in the first pass); returns false
// when a mask does not fit or more than 6 passes would be needed.
struct PsumPass {
    std::vector<int> hb;      // ascending high bits
    size_t first, count;      // range in the regrouped term array
};
bool plan_psum_passes(int n, const std::vector<PauliDev> &terms, std::vector<PauliDev> &out,
                      std::vector<PsumPass> &passes) {
    if (n < 8 || terms.empty()) return false;
    const int H = std::min(7, n - 4);
    std::vector<uint64_t> sets;                 // high-bit set of each pass
    std::vector<std::vector<PauliDev>> groups;
    std::vector<PauliDev> diag;
    for (const PauliDev &t : terms) {
        const uint64_t hx = t.x & ~15ull;
        if (hx == 0) {
            diag.push_back(t);
            continue;
        }
        if (__builtin_popcountll(hx) > H) return false;
        size_t g = 0;
        for (; g < sets.size(); ++g)
            if (__builtin_popcountll(sets[g] | hx) <= H) break;
        if (g == sets.size()) {
            sets.push_back(0);
            groups.emplace_back();
        }
        sets[g] |= hx;
        groups[g].push_back(t);
    }
    if (sets.empty()) {
        sets.push_back(0);
        groups.emplace_back();
    }
    groups[0].insert(groups[0].begin(), diag.begin(), diag.end());
    out.clear();
    passes.clear();
    for (size_t g = 0; g < sets.size(); ++g) {
        uint64_t S = sets[g];
        for (int b = 4; b < n && __builtin_popcountll(S) < H; ++b) S |= 1ull << b;   // fill the tile
        std::vector<int> hb;
        for (int b = 4; b < n; ++b)
            if ((S >> b) & 1) hb.push_back(b);
        for (size_t i = 0; i < groups[g].size(); i += kPsumMaxTerms) {
            PsumPass ps;
            ps.hb = hb;
            ps.first = out.size();
            ps.count = std::min<size_t>(kPsumMaxTerms, groups[g].size() - i);
            out.insert(out.end(), groups[g].begin() + i, groups[g].begin() + i + ps.count);
            passes.push_back(ps);
        }
    }
    return passes.size() <= 6;
}
}  // namespace

qs_status qs_grad(qs_state *st, const qs_gate *gates, size_t n_gates, const double *params, int n_params,
                  const qs_pauli *terms, size_t n_terms, double *energy, double *grad) {
    if (!st || !energy || !grad || (n_terms && !terms) || (n_gates && !gates))
        return fail(QS_ERR_INVALID_ARG, "NULL argument");
    if (n_params < 0 || (n_params > 0 && !params)) return fail(QS_ERR_INVALID_ARG, "bad params");
    for (size_t i = 0; i < n_gates; ++i)
        if (gates[i].param_idx >= 0) {
            int k = gates[i].kind;
            if (k != QS_RX && k != QS_RY && k != QS_RZ && k != QS_RZZ && k != QS_CP)
                return fail(QS_ERR_UNSUPPORTED, "qs_grad: parameterised gates must be RX, RY, RZ, RZZ or CP");
        }
    const int B = st->batch;
    std::vector<std::vector<RGate>> rg(B);
    for (int b = 0; b < B; ++b) {
        std::string err;
        qs_status s = resolve_gates(st->n, gates, n_gates, params, n_params, b, rg[b], err);
        if (s != QS_OK) return fail(s, err);
    }
    std::vector<TermIdx> t;
    qs_status s = convert_terms(st->n, terms, n_terms, t);
    if (s != QS_OK) return s;
    // the forward and un-apply plans: 13-bit tiles with 5-bit register groups
    // (the warp-specialised kernel) from 20 qubits on, where every item has
    // 128 tiles or more (VQE config, n = 24, batch 32: 94 -> 104 gradient
    // vectors/s against the planner's 12-bit choice for these per-item layer
    // passes)
    qs_opts fo = default_opts(nullptr);
    if (st->n >= 20) {
        fo.tile_qubits = 13;
        fo.group_qubits = 5;
    }
    // Un-apply segments: the gates between two gradient points, latest first.
    // Their plans (per item when the segment carries parameters, else one for
    // all pairs) are built up front on host threads.
    struct Segment {
        std::vector<size_t> gates;
        bool per_item = false;
        size_t first_plan = 0;
    };
    std::vector<Segment> segs;
    std::vector<size_t> pending;   // gates to un-apply, latest first
    auto close_segment = [&]() {
        if (pending.empty()) return;
        Segment sg;
        sg.gates.swap(pending);
        for (size_t gi : sg.gates)
            if (gates[gi].param_idx >= 0) sg.per_item = true;
        segs.push_back(std::move(sg));
    };
    size_t next_seg = 0;
    std::vector<Plan> seg_plans;
    // dry run of the sweep: the segments in execution order, and the gradient
    // points (the last gate index of each point's layer or 2q gate), latest first
    std::vector<size_t> gpts;
    for (size_t gi = n_gates; gi-- > 0;) {
        if (rg[0][gi].nw == 1) {
            size_t lo = gi;
            while (lo > 0 && rg[0][lo - 1].nw == 1) --lo;
            bool has_param = false;
            for (size_t k = lo; k <= gi; ++k)
                if (gates[k].param_idx >= 0) has_param = true;
            if (has_param) {
                close_segment();
                gpts.push_back(gi);
            }
            for (size_t k = gi + 1; k-- > lo;) pending.push_back(k);
            gi = lo;
            continue;
        }
        if (gates[gi].param_idx >= 0) {
            close_segment();
            gpts.push_back(gi);
        }
        pending.push_back(gi);
    }
    pending.clear();   // the gates before the first gradient point are never un-applied
    // Checkpoint mode, when the device has room for one copy of the states per
    // gradient point: the forward pass stores psi at every gradient point and
    // the reverse sweep un-applies only lambda (half the work of un-applying
    // the (psi, lambda) pairs).  Otherwise the pairs are un-applied.
    const long long E = st->elems;
    const size_t K = gpts.size();
    const size_t ck_bytes = (K + 1) * (size_t)B * E * sizeof(float2);
    bool ckpt = false;
    {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            const size_t held = st->grad_ws_bytes;
            ckpt = K > 0 && fr + held > ck_bytes + ((size_t)2 << 30);
        }
        cudaGetLastError();
    }
    // workspace: checkpoint mode = K checkpoints then lambda (B states each);
    // pair mode = (psi_b, lam_b) pairs next to each other, so that an item's
    // pair is a batch of two states for the fused executor.  Allocated before
    // the un-apply plans are built (their batch depends on the mode); when the
    // checkpoints cannot be allocated after all, pair mode is used.
    auto ensure_ws = [&](size_t bytes) {
        if (st->grad_ws_bytes >= bytes) return true;
        if (st->grad_ws) {
            cudaStreamSynchronize(st->stream);
            cudaFree(st->grad_ws);
            st->grad_ws = nullptr;
            st->grad_ws_bytes = 0;
        }
        if (cudaMalloc((void **)&st->grad_ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            st->grad_ws = nullptr;
            return false;
        }
        st->grad_ws_bytes = bytes;
        return true;
    };
    if (ckpt && !ensure_ws(ck_bytes)) ckpt = false;
    if (!ckpt && !ensure_ws((size_t)E * 2 * B * sizeof(float2)))
        return fail(QS_ERR_OOM, "qs_grad: no memory for the adjoint states");
    const int un_b = ckpt ? 1 : 2;   // states per item in an un-apply launch
    // the un-apply plans are built on host threads while the GPU runs the
    // forward circuit and the Hamiltonian
    qs_status seg_status = QS_OK;
    std::string seg_err;
    std::thread seg_thread([&]() {
        {
            std::vector<std::vector<RGate>> lists;
            for (Segment &sg : segs) {
                sg.first_plan = lists.size();
                for (int b = 0; b < (sg.per_item ? B : 1); ++b) {
                    std::vector<RGate> inv;
                    for (size_t gi : sg.gates) invert_gate(rg[b][gi], inv);
                    lists.push_back(std::move(inv));
                }
            }
            // per-item segments run on a pair (batch 2), shared ones on all pairs
            std::vector<std::vector<RGate>> l2, lB;
            std::vector<size_t> i2, iB;
            for (const Segment &sg : segs)
                for (int b = 0; b < (sg.per_item ? B : 1); ++b) {
                    const size_t i = sg.first_plan + b;
                    if (sg.per_item) {
                        i2.push_back(i);
                        l2.push_back(lists[i]);
                    } else {
                        iB.push_back(i);
                        lB.push_back(lists[i]);
                    }
                }
            std::vector<Plan> p2, pB;
            std::string err;
            qs_status r = build_plans_parallel(st->n, un_b, l2, fo, p2, err, true);
            if (r == QS_OK) r = build_plans_parallel(st->n, un_b * B, lB, fo, pB, err, false);
            if (r != QS_OK) {
                seg_status = r;
                seg_err = err;
                return;
            }
            seg_plans.resize(lists.size());
            for (size_t j = 0; j < i2.size(); ++j) seg_plans[i2[j]] = std::move(p2[j]);
            for (size_t j = 0; j < iB.size(); ++j) seg_plans[iB[j]] = std::move(pB[j]);
        }
    });
    struct Joiner {
        std::thread &t;
        ~Joiner() {
            if (t.joinable()) t.join();
        }
    } joiner{seg_thread};
    float2 *W = st->grad_ws;
    float2 *Lam = ckpt ? W + K * (size_t)B * E : W + E;   // lambda of item 0
    const long long ls = ckpt ? E : 2 * E;                // item stride of psi / lambda buffers
    auto ckpt_at = [&](size_t c) { return W + c * (size_t)B * E; };   // c = 0: earliest point
    // 1. forward: psi = U(theta)|0>; per item plans built in parallel and merged
    QS_CUDA(launch_init_zero(st->home, st->elems, B, st->stream));
    qs_opts o = fo;
    auto run_forward = [&](size_t g_begin, size_t g_end) -> qs_status {   // gates [g_begin, g_end)
        if (g_end <= g_begin) return QS_OK;
        bool pi = false;
        for (size_t i = g_begin; i < g_end; ++i)
            if (gates[i].param_idx >= 0) pi = true;
        std::vector<std::vector<RGate>> lists(pi ? B : 1);
        for (size_t b = 0; b < lists.size(); ++b)
            lists[b].assign(rg[b].begin() + g_begin, rg[b].begin() + g_end);
        std::vector<Plan> fwd;
        std::string err;
        qs_status r = build_plans_parallel(st->n, pi ? 1 : B, lists, o, fwd, err, pi);
        if (r != QS_OK) return fail(r, err);
        if (!pi) return run_host_plan(st, std::move(fwd[0]), st->home, B);
        Plan merged;
        if (B > 1 && merge_item_plans(fwd, merged, B)) return run_host_plan(st, std::move(merged), st->home, B);
        for (int b = 0; b < B; ++b) {
            r = run_host_plan(st, std::move(fwd[b]), st->home + (size_t)b * E, 1);
            if (r != QS_OK) return r;
        }
        return QS_OK;
    };
    if (ckpt) {   // chunks ending at the gradient points, psi stored after each
        size_t g0 = 0;
        for (size_t c = 0; c < K; ++c) {
            const size_t e = gpts[K - 1 - c] + 1;
            s = run_forward(g0, e);
            if (s != QS_OK) return s;
            QS_CUDA(cudaMemcpyAsync(ckpt_at(c), st->home, (size_t)B * E * sizeof(float2), cudaMemcpyDeviceToDevice,
                                    st->stream));
            g0 = e;
        }
        s = run_forward(g0, n_gates);
    } else {
        s = run_forward(0, n_gates);
    }
    if (s != QS_OK) return s;
    // 2. the energy comes with lam = H psi below: E = Re <psi|lam>
    qs_state *aux = nullptr;
    struct Guard {
        qs_state **aux;
        ~Guard() {
            if (*aux) qs_free(*aux);
        }
    } guard{&aux};
    const float2 *Psi0 = ckpt ? st->home : W;   // psi(theta) next to lambda for the energy
    if (!ckpt)
        QS_CUDA(cudaMemcpy2DAsync(W, 2 * E * sizeof(float2), st->home, E * sizeof(float2), E * sizeof(float2), B,
                                  cudaMemcpyDeviceToDevice, st->stream));
    // lam = H psi; the term array (H's terms, then the identity used for the
    // energy) stays alive until the call ends, so nothing waits here
    std::vector<PauliDev> hp;
    for (auto &x : t) hp.push_back({x.coeff, x.x, x.z});
    std::stable_sort(hp.begin(), hp.end(), [](const PauliDev &a, const PauliDev &b) { return a.x < b.x; });
    // shared-memory tiles when the x masks fit a few tile bit sets
    std::vector<PauliDev> regrouped;
    std::vector<PsumPass> ppass;
    const bool tiled_sum = plan_psum_passes(st->n, hp, regrouped, ppass);
    if (tiled_sum) hp = regrouped;
    const int n_h = (int)hp.size();
    hp.push_back({1.0, 0, 0});
    s = ensure_terms(st, hp.size());
    if (s != QS_OK) return s;
    s = h2d_async(st, st->d_terms, hp.data(), hp.size() * sizeof(PauliDev));
    if (s != QS_OK) return s;
    if (n_h && tiled_sum) {
        for (size_t k = 0; k < ppass.size(); ++k) {
            PsumTileArgs A;
            std::memset(&A, 0, sizeof A);
            A.psi = Psi0;
            A.lam = Lam;
            A.elems = E;
            A.bstride = ls;
            A.batch = B;
            A.H = (int)ppass[k].hb.size();
            uint64_t tb = 15;
            for (int j = 0; j < A.H; ++j) {
                A.hb[j] = ppass[k].hb[j];
                tb |= 1ull << A.hb[j];
            }
            for (int b = 0; b < st->n; ++b)
                if (!((tb >> b) & 1)) A.outer[A.n_outer++] = b;
            A.terms = st->d_terms + ppass[k].first;
            A.n_terms = (int)ppass[k].count;
            A.accumulate = k > 0;
            const long long n_tiles = E >> (4 + A.H);
            A.grid = (int)std::max(1ll, std::min<long long>(n_tiles, (8ll * g_num_sms[st->dev] + B - 1) / B));
            cudaEvent_t ev;
            prof_begin(st, &ev);
            QS_CUDA(launch_pauli_sum_tile(A, st->stream));
            prof_end(st, ev, "pauli_sum", (k ? 24.0 : 16.0) * (double)E * B);
        }
    } else if (n_h) {
        cudaEvent_t ev;
        prof_begin(st, &ev);
        QS_CUDA(launch_apply_pauli_sum(Psi0, Lam, E, B, st->d_terms, n_h, st->stream, ls));
        prof_end(st, ev, "pauli_sum", 16.0 * (double)E * B);
    } else {
        QS_CUDA(cudaMemset2DAsync(Lam, ls * sizeof(float2), 0, E * sizeof(float2), B, st->stream));
    }
    // E_b = Re sum_x conj(lam_x) psi_x into a device array, read with the gradients
    double *d_en = nullptr;
    QS_CUDA(cudaMallocAsync((void **)&d_en, (size_t)B * 2 * sizeof(double), st->stream));
    struct Guard2 {
        qs_state *st;
        double *p;
        ~Guard2() {
            if (p) cudaFreeAsync(p, st->stream);
        }
    } guard2{st, d_en};
    {
        const int grid = std::max(1, std::min<int>((int)((E + 255) / 256), g_num_sms[st->dev] * 4));
        s = ensure_partial(st, (size_t)B * grid * 2);
        if (s != QS_OK) return s;
        ExpectArgs A;
        std::memset(&A, 0, sizeof A);
        A.psi = Psi0;
        A.lam = Lam;
        A.state_elems = E;
        A.bstride = ls;
        A.batch = B;
        A.xmask = 0;
        A.n_terms = 1;
        A.terms = st->d_terms + n_h;
        A.partial = st->d_partial;
        A.grid = grid;
        cudaEvent_t ev;
        prof_begin(st, &ev);
        QS_CUDA(launch_expect_group(A, st->stream));
        prof_end(st, ev, "expect", 16.0 * (double)E * B);
        QS_CUDA(launch_expect_finish(st->d_partial, d_en, B, grid, 1, st->stream));
    }
    s = ckpt ? qs_wrap(Lam, st->n, B, st->stream, &aux) : qs_wrap(W, st->n, 2 * B, st->stream, &aux);
    if (s != QS_OK) return s;
    for (size_t i = 0; i < (size_t)B * n_params; ++i) grad[i] = 0.0;

    // 4. reverse sweep (Jones & Gacon 2020), a layer at a time.  A maximal run
    //    of 1q gates is one layer: every parameterised gate in it has
    //    dE/dtheta = Im<lam|V G V^dagger|psi> at the post-layer states, V the
    //    later gates of the run on its wire (those on other wires commute
    //    with G); V G V^dagger = c_x X + c_y Y + c_z Z (FP64, per item), so one
    //    X / Y / Z overlap pass per 4 wires serves the whole layer.  The gates
    //    between gradient points are un-applied with the fused executor:
    //    per item (batch = the pair) when they carry parameters, otherwise
    //    once for all pairs.  Parameterised 2q gates (RZZ, CP) take their own
    //    overlap of generator terms.
    seg_thread.join();
    if (seg_status != QS_OK) return fail(seg_status, seg_err);
    auto flush = [&]() -> qs_status {
        if (pending.empty()) return QS_OK;
        pending.clear();
        const Segment &sg = segs[next_seg++];
        // checkpoint mode: lambda only (B states); pair mode: all pairs (2B)
        float2 *base = ckpt ? Lam : W;
        const int nb = un_b * B;
        if (!sg.per_item) return run_host_plan(aux, std::move(seg_plans[sg.first_plan]), base, nb);
        if (B > 1) {   // the items' plans merged: one launch per pass over all items
            std::vector<Plan> items(std::make_move_iterator(seg_plans.begin() + sg.first_plan),
                                    std::make_move_iterator(seg_plans.begin() + sg.first_plan + B));
            Plan merged;
            if (merge_item_plans(items, merged, nb)) return run_host_plan(aux, std::move(merged), base, nb);
            for (int b = 0; b < B; ++b) seg_plans[sg.first_plan + b] = std::move(items[b]);
        }
        for (int b = 0; b < B; ++b) {
            qs_status r = run_host_plan(aux, std::move(seg_plans[sg.first_plan + b]), base + (size_t)b * ls, un_b);
            if (r != QS_OK) return r;
        }
        return QS_OK;
    };
    // overlap launches: shared-memory tiles of the 4 low bits + <= 8 wires
    // (n >= 6), else register groups of <= 4 wires
    const bool tiled = st->n >= 6;
    struct XyzLaunch {
        int k;                   // group bits (register kernel) or H (tile kernel)
        int gbit[8];             // the group bits / the tile's high bits
        uint32_t xymask;         // tile kernel: tile bits whose X / Y are taken
        uint64_t zmask;
    };
    struct LayerRec {
        std::vector<size_t> gates;          // the run, in circuit order
        std::vector<XyzLaunch> launches;    // results at d_res[first + i]
        size_t first;
    };
    std::vector<LayerRec> layers;
    size_t n_launch = 0;
    // first pass: plan the layers and their overlap launches
    for (size_t gi = n_gates; gi-- > 0;) {
        if (rg[0][gi].nw != 1) continue;
        size_t lo = gi;
        while (lo > 0 && rg[0][lo - 1].nw == 1) --lo;
        LayerRec L;
        uint64_t wires = 0;
        for (size_t k = lo; k <= gi; ++k) {
            L.gates.push_back(k);
            if (gates[k].param_idx >= 0) wires |= 1ull << rg[0][k].b[0];
        }
        if (wires && tiled) {
            std::vector<int> hi, others;
            for (int q = 4; q < st->n; ++q) ((wires >> q) & 1 ? hi : others).push_back(q);
            // 11-bit tiles (three CTAs per SM with double buffers) for large
            // states; up to 21 qubits 12-bit tiles, whose fewer launches win
            // (n = 20: 54 -> 38 ms per 32-item batch; n = 24: 504 vs 595 ms)
            const int hmax = std::min(st->n <= 21 ? 8 : 7, st->n - 4);
            size_t c = 0;
            do {
                XyzLaunch x;
                std::memset(&x, 0, sizeof x);
                std::vector<int> hb(hi.begin() + c, hi.begin() + std::min(hi.size(), c + (size_t)hmax));
                const int used = (int)hb.size();
                // larger tiles amortise the per-tile work: pad with bits that are not wires
                for (size_t o = 0; (int)hb.size() < hmax && o < others.size(); ++o) hb.push_back(others[o]);
                std::sort(hb.begin(), hb.end());
                x.k = (int)hb.size();
                uint64_t tb = 15;
                for (int k = 0; k < x.k; ++k) {
                    x.gbit[k] = hb[k];
                    tb |= 1ull << hb[k];
                    if ((wires >> hb[k]) & 1) x.xymask |= 1u << (4 + k);
                }
                if (c == 0) {
                    x.xymask |= (uint32_t)(wires & 15);
                    x.zmask = wires & ~tb;
                }
                L.launches.push_back(x);
                c += used;
            } while (c < hi.size());
        } else if (wires) {
            std::vector<int> bits;
            for (int q = 0; q < st->n; ++q)
                if ((wires >> q) & 1) bits.push_back(q);
            for (size_t c = 0; c < bits.size(); c += kXyzGroup) {
                XyzLaunch x;
                std::memset(&x, 0, sizeof x);
                x.k = (int)std::min<size_t>(kXyzGroup, bits.size() - c);
                uint64_t gm = 0;
                for (int j = 0; j < x.k; ++j) {
                    x.gbit[j] = bits[c + j];
                    gm |= 1ull << bits[c + j];
                }
                x.zmask = c == 0 ? (wires & ~gm) : 0;
                L.launches.push_back(x);
            }
        }
        if (wires) {
            L.first = n_launch;
            n_launch += L.launches.size();
            layers.push_back(L);
        }
        gi = lo;
    }
    const int slots = tiled ? kXyzTSlots : kXyzSlots;
    const int xgrid = tiled ? (int)std::max(1ll, std::min<long long>(E >> 11, (6ll * g_num_sms[st->dev] + B - 1) / B))
                            : xyz_grid(E, 1);
    double *d_res = nullptr;
    if (n_launch) {
        s = ensure_partial(st, (size_t)B * xgrid * slots);
        if (s != QS_OK) return s;
        QS_CUDA(cudaMallocAsync((void **)&d_res, n_launch * B * slots * sizeof(double), st->stream));
    }
    struct Guard3 {
        qs_state *st;
        double *p;
        ~Guard3() {
            if (p) cudaFreeAsync(p, st->stream);
        }
    } guard3{st, d_res};
    size_t li = 0, gp = 0;   // layers done, gradient points done
    // psi at the current gradient point: its checkpoint, or the pairs' psi
    auto psi_now = [&]() -> const float2 * { return ckpt ? ckpt_at(K - 1 - gp) : W; };
    for (size_t gi = n_gates; gi-- > 0;) {
        const RGate &r0 = rg[0][gi];
        if (r0.nw == 1) {
            size_t lo = gi;
            while (lo > 0 && rg[0][lo - 1].nw == 1) --lo;
            bool has_param = false;
            for (size_t k = lo; k <= gi; ++k)
                if (gates[k].param_idx >= 0) has_param = true;
            if (has_param) {
                s = flush();
                if (s != QS_OK) return s;
                if (li >= layers.size() || (ckpt && gp >= K)) return fail(QS_ERR_INTERNAL, "qs_grad: layer bookkeeping");
                const LayerRec &L = layers[li++];
                for (size_t c = 0; c < L.launches.size(); ++c) {
                    const XyzLaunch &x = L.launches[c];
                    cudaEvent_t ev;
                    prof_begin(st, &ev);
                    if (tiled) {
                        XyzTileArgs A;
                        std::memset(&A, 0, sizeof A);
                        A.psi = psi_now();
                        A.lam = Lam;
                        A.elems = E;
                        A.bstride = ls;
                        A.batch = B;
                        A.n = st->n;
                        A.H = x.k;
                        for (int j = 0; j < x.k; ++j) A.hb[j] = x.gbit[j];
                        A.xymask = x.xymask;
                        A.zmask = x.zmask;
                        A.partial = st->d_partial;
                        A.grid = xgrid;
                        QS_CUDA(launch_xyz_tile(A, st->stream));
                    } else {
                        XyzArgs A;
                        std::memset(&A, 0, sizeof A);
                        A.psi = psi_now();
                        A.lam = Lam;
                        A.elems = E;
                        A.bstride = ls;
                        A.batch = B;
                        A.k = x.k;
                        for (int j = 0; j < A.k; ++j) A.gbit[j] = x.gbit[j];
                        A.zmask = x.zmask;
                        A.partial = st->d_partial;
                        A.grid = xgrid;
                        QS_CUDA(launch_xyz_overlaps(A, st->stream));
                    }
                    prof_end(st, ev, "xyz_overlap", 16.0 * (double)E * B);
                    QS_CUDA(launch_expect_finish(st->d_partial, d_res + (L.first + c) * B * slots, B, xgrid, slots / 2,
                                                 st->stream));
                }
                ++gp;
            }
            for (size_t k = gi + 1; k-- > lo;) pending.push_back(k);
            gi = lo;
            continue;
        }
        if (gates[gi].param_idx >= 0) {   // RZZ / CP: generator overlap at the post-gate states
            s = flush();
            if (s != QS_OK) return s;
            if (ckpt && gp >= K) return fail(QS_ERR_INTERNAL, "qs_grad: gradient point bookkeeping");
            std::vector<TermIdx> gt;
            auto term = [&](double c, uint64_t x, uint64_t z) {
                TermIdx q;
                q.coeff = c;
                q.x = x;
                q.z = z;
                q.ny = __builtin_popcountll(x & z) & 3;
                gt.push_back(q);
            };
            const uint64_t ba = 1ull << r0.b[0], bb = 1ull << r0.b[1];
            if (gates[gi].kind == QS_RZZ) {
                term(1.0, 0, ba | bb);
            } else {   // CP(t) = exp(i t P11), P11 = (1 - Za - Zb + ZaZb) / 4
                term(0.25, 0, 0);
                term(-0.25, 0, ba);
                term(-0.25, 0, bb);
                term(0.25, 0, ba | bb);
            }
            std::vector<double> S;
            s = overlaps(st, psi_now(), Lam, B, gt, S, ls);
            if (s != QS_OK) return s;
            for (int b = 0; b < B; ++b) {
                double im_tot = 0.0;
                for (size_t k = 0; k < gt.size(); ++k) {
                    double re = S[((size_t)b * gt.size() + k) * 2], im = S[((size_t)b * gt.size() + k) * 2 + 1];
                    times_i_pow(re, im, gt[k].ny);
                    im_tot += gt[k].coeff * im;
                }
                // R(t) = exp(-i t G/2): dE/dt = Im<lam|G|psi>;  CP(t) = exp(i t P11): dE/dt = -2 Im<lam|P11|psi>
                grad[(size_t)b * n_params + gates[gi].param_idx] += gates[gi].kind == QS_CP ? -2.0 * im_tot : im_tot;
            }
            ++gp;
        }
        pending.push_back(gi);
    }
    // 5. the energies, and the gradients of the 1q layers from their X / Y / Z overlaps
    {
        std::vector<double> en((size_t)B * 2);
        QS_CUDA(cudaMemcpyAsync(en.data(), d_en, en.size() * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
        QS_CUDA(cudaStreamSynchronize(st->stream));
        for (int b = 0; b < B; ++b) energy[b] = en[(size_t)b * 2];
    }
    if (n_launch) {
        std::vector<double> res(n_launch * B * slots);
        QS_CUDA(cudaMemcpyAsync(res.data(), d_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
        QS_CUDA(cudaStreamSynchronize(st->stream));
        for (const LayerRec &L : layers) {
            for (int b = 0; b < B; ++b) {
                // Im<X_q>, Im<Y_q>, Im<Z_q> of the layer's wires for item b
                std::map<int, std::array<double, 3>> ov;
                double total = 0.0;
                std::map<int, double> sq;
                for (size_t c = 0; c < L.launches.size(); ++c) {
                    const double *r = &res[((L.first + c) * B + b) * slots];
                    const XyzLaunch &x = L.launches[c];
                    if (tiled) {
                        // tile bit t: low bit t (t < 4) or high bit gbit[t - 4]
                        for (int t = 0; t < 4 + x.k; ++t) {
                            if (!((x.xymask >> t) & 1)) continue;
                            const int q = t < 4 ? t : x.gbit[t - 4];
                            ov[q][0] = r[t];
                            ov[q][1] = r[kXyzTileBits + t];
                        }
                        if (c == 0) {
                            total = r[2 * kXyzTileBits + kXyzZBits];
                            for (int q = 0; q < kXyzZBits && q < st->n; ++q) sq[q] = r[2 * kXyzTileBits + q];
                        }
                        continue;
                    }
                    if (c == 0) total = r[3 * kXyzGroup + kXyzZBits];
                    for (int j = 0; j < x.k; ++j) {
                        ov[x.gbit[j]][0] = r[j];
                        ov[x.gbit[j]][1] = r[kXyzGroup + j];
                        sq[x.gbit[j]] = r[2 * kXyzGroup + j];
                    }
                    for (int q = 0; q < kXyzZBits; ++q)
                        if ((x.zmask >> q) & 1) sq[q] = r[3 * kXyzGroup + q];
                }
                for (auto &kv : sq) ov[kv.first][2] = total - 2.0 * kv.second;
                for (size_t a = 0; a < L.gates.size(); ++a) {
                    const size_t gi = L.gates[a];
                    if (gates[gi].param_idx < 0) continue;
                    const RGate &g = rg[b][gi];
                    // V = product of the later gates of the run on this wire
                    cd V[4] = {1, 0, 0, 1};
                    for (size_t c2 = a + 1; c2 < L.gates.size(); ++c2) {
                        const RGate &h = rg[b][L.gates[c2]];
                        if (h.b[0] != g.b[0]) continue;
                        cd M[4], T[4];
                        gate_matrix(h, M);
                        T[0] = M[0] * V[0] + M[1] * V[2];
                        T[1] = M[0] * V[1] + M[1] * V[3];
                        T[2] = M[2] * V[0] + M[3] * V[2];
                        T[3] = M[2] * V[1] + M[3] * V[3];
                        for (int e2 = 0; e2 < 4; ++e2) V[e2] = T[e2];
                    }
                    cd Gm[4];
                    switch (g.kind) {
                        case QS_RX: Gm[0] = 0; Gm[1] = 1; Gm[2] = 1; Gm[3] = 0; break;
                        case QS_RY: Gm[0] = 0; Gm[1] = cd(0, -1); Gm[2] = cd(0, 1); Gm[3] = 0; break;
                        default: Gm[0] = 1; Gm[1] = 0; Gm[2] = 0; Gm[3] = -1; break;
                    }
                    // Ge = V G V^dagger
                    cd VG[4], Ge[4];
                    VG[0] = V[0] * Gm[0] + V[1] * Gm[2];
                    VG[1] = V[0] * Gm[1] + V[1] * Gm[3];
                    VG[2] = V[2] * Gm[0] + V[3] * Gm[2];
                    VG[3] = V[2] * Gm[1] + V[3] * Gm[3];
                    Ge[0] = VG[0] * std::conj(V[0]) + VG[1] * std::conj(V[1]);
                    Ge[2] = VG[2] * std::conj(V[0]) + VG[3] * std::conj(V[1]);
                    const double cx = Ge[2].real(), cy = Ge[2].imag(), cz = Ge[0].real();
                    const auto &o3 = ov[g.b[0]];
                    grad[(size_t)b * n_params + gates[gi].param_idx] += cx * o3[0] + cy * o3[1] + cz * o3[2];
                }
            }
        }
    }
    s = check_err_word(aux);
    if (s != QS_OK) return s;
    return check_err_word(st);
}

qs_status qs_qaoa_maxcut(const qs_graph *graphs, size_t n_graphs, int n_sets, int p, const double *gammas,
                         const double *betas, double *out, void *cuda_stream) {
    if (!graphs || !gammas || !betas || !out) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    if (n_sets < 1) return fail(QS_ERR_INVALID_ARG, "n_sets < 1");
    if (p < 1 || p > kQaoaMaxP) return fail(QS_ERR_UNSUPPORTED, "p must be in [1, 16]");
    for (size_t g = 0; g < n_graphs; ++g) {
        const qs_graph &G = graphs[g];
        if (G.n < 1 || G.n > 30) return fail(QS_ERR_UNSUPPORTED, "graph size must be in [1, 30]");
        if (G.n_edges < 0 || G.n_edges > kQaoaMaxEdges) return fail(QS_ERR_UNSUPPORTED, "at most 64 edges per graph");
        if (G.n_edges && !G.edges) return fail(QS_ERR_INVALID_ARG, "edges == NULL");
        for (int e = 0; e < G.n_edges; ++e) {
            const int u = G.edges[2 * e], v = G.edges[2 * e + 1];
            if (u < 0 || v < 0 || u >= G.n || v >= G.n || u == v) return fail(QS_ERR_INVALID_ARG, "bad edge");
        }
    }
    for (size_t i = 0; i < n_graphs * (size_t)n_sets * p; ++i)
        if (!std::isfinite(gammas[i]) || !std::isfinite(betas[i])) return fail(QS_ERR_INVALID_ARG, "non-finite angle");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int dev = current_device();
    qs_status s = ensure_device_tables(dev);
    if (s != QS_OK) return s;
    const size_t n_out = n_graphs * (size_t)n_sets;

    // ---- every instance with n <= 24: one persistent launch, largest first ----
    std::vector<QaoaItem> items;
    std::vector<uint32_t> masks;
    std::vector<float2> luts, mix;
    std::vector<size_t> order(n_graphs);
    for (size_t g = 0; g < n_graphs; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return graphs[a].n > graphs[b].n; });
    int n_slot = 0;   // largest n kept in a device-memory slot
    for (size_t g : order) {
        const qs_graph &G = graphs[g];
        if (G.n > kQaoaMaxPersistentN) continue;
        if (G.n > kQaoaMaxSmallN) n_slot = std::max(n_slot, G.n);
        const int eo = (int)masks.size();
        for (int e = 0; e < G.n_edges; ++e)
            masks.push_back((1u << (G.n - 1 - G.edges[2 * e])) | (1u << (G.n - 1 - G.edges[2 * e + 1])));
        for (int a = 0; a < n_sets; ++a) {
            QaoaItem it;
            it.n = G.n;
            it.n_edges = G.n_edges;
            it.edge_off = eo;
            it.lut_off = (int)luts.size();
            it.mix_off = (int)mix.size();
            it.out_idx = (int)(g * n_sets + a);
            const double *gm = gammas + (g * n_sets + a) * p, *bt = betas + (g * n_sets + a) * p;
            for (int l = 0; l < p; ++l) {
                for (int k = 0; k <= G.n_edges; ++k) {
                    const double ph = std::remainder(-gm[l] * k, 2.0 * 3.14159265358979323846);
                    luts.push_back(make_float2((float)std::cos(ph), (float)std::sin(ph)));
                }
                mix.push_back(make_float2((float)std::cos(bt[l]), (float)-std::sin(bt[l])));
            }
            items.push_back(it);
        }
    }
    std::vector<double> hout(n_out, 0.0);
    if (!items.empty()) {
        QaoaItem *d_items = nullptr;
        uint32_t *d_masks = nullptr;
        float2 *d_luts = nullptr, *d_mix = nullptr, *d_slots = nullptr;
        double *d_out = nullptr;
        int *d_counter = nullptr;
        auto cleanup = [&]() {
            cudaFree(d_items);
            cudaFree(d_masks);
            cudaFree(d_luts);
            cudaFree(d_mix);
            cudaFree(d_out);
            cudaFree(d_counter);
            cudaFree(d_slots);
        };
        const int grid = (int)std::min<size_t>(items.size(), (size_t)g_num_sms[dev]);
        const long long slot_elems = n_slot ? (1ll << n_slot) : 0;
        bool okm = cudaMalloc(&d_items, items.size() * sizeof(QaoaItem)) == cudaSuccess &&
                   cudaMalloc(&d_masks, std::max<size_t>(1, masks.size()) * sizeof(uint32_t)) == cudaSuccess &&
                   cudaMalloc(&d_luts, luts.size() * sizeof(float2)) == cudaSuccess &&
                   cudaMalloc(&d_mix, mix.size() * sizeof(float2)) == cudaSuccess &&
                   cudaMalloc(&d_out, n_out * sizeof(double)) == cudaSuccess &&
                   cudaMalloc(&d_counter, sizeof(int)) == cudaSuccess &&
                   (!slot_elems ||
                    cudaMalloc(&d_slots, (size_t)grid * (size_t)slot_elems * sizeof(float2)) == cudaSuccess);
        if (!okm) {
            cudaGetLastError();
            cleanup();
            return fail(QS_ERR_OOM, "qs_qaoa_maxcut: device allocation failed");
        }
        cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(QaoaItem), cudaMemcpyHostToDevice, st);
        if (!masks.empty())
            cudaMemcpyAsync(d_masks, masks.data(), masks.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_luts, luts.data(), luts.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_mix, mix.data(), mix.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(d_counter, 0, sizeof(int), st);
        QaoaArgs A;
        A.items = d_items;
        A.n_items = (int)items.size();
        A.p = p;
        A.edge_masks = d_masks;
        A.luts = d_luts;
        A.mix = d_mix;
        A.out = d_out;
        A.counter = d_counter;
        A.slots = d_slots;
        A.slot_elems = slot_elems;
        cudaError_t e = launch_qaoa(A, grid, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hout.data(), d_out, n_out * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cleanup();
        if (e != cudaSuccess) return fail(QS_ERR_CUDA, std::string("qaoa kernel: ") + cudaGetErrorString(e));
        for (const QaoaItem &it : items) out[it.out_idx] = hout[it.out_idx];
    }

    // ---- states above 24 qubits: fused tile passes, all angle sets of a graph as one batch ----
    // Everything is enqueued on one stream and the results stay on the device
    // until the end, so the host plans graph g + 1 while the GPU runs graph g.
    std::map<int, qs_state *> states;
    qs_status rs = QS_OK;
    size_t n_large = 0;
    for (size_t g = 0; g < n_graphs; ++g)
        if (graphs[g].n > kQaoaMaxPersistentN) ++n_large;
    double *d_res = nullptr;   // (re, im) per (graph, angle set)
    if (n_large && cudaMalloc(&d_res, n_out * 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ERR_OOM, "qs_qaoa_maxcut: device allocation failed");
    }
    for (size_t g = 0; g < n_graphs && rs == QS_OK; ++g) {
        const qs_graph &G = graphs[g];
        if (G.n <= kQaoaMaxPersistentN) continue;
        qs_state *S = states[G.n];
        if (!S) {
            rs = qs_alloc(G.n, n_sets, &S);
            if (rs != QS_OK) break;
            qs_set_stream(S, cuda_stream);
            states[G.n] = S;
        }
        // H on all, then per layer RZZ(-gamma_l) per edge and RX(2 beta_l) per qubit;
        // parameter 2l = -gamma_l, 2l+1 = 2 beta_l
        std::vector<qs_gate> gl;
        auto gate = [&](int kind, int nw, int w0, int w1, int pidx) {
            qs_gate q;
            std::memset(&q, 0, sizeof q);
            q.kind = (uint16_t)kind;
            q.nw = (uint8_t)nw;
            q.w[0] = w0;
            q.w[1] = w1;
            q.param_idx = pidx;
            gl.push_back(q);
        };
        for (int q = 0; q < G.n; ++q) gate(QS_H, 1, q, 0, -1);
        for (int l = 0; l < p; ++l) {
            for (int e = 0; e < G.n_edges; ++e) gate(QS_RZZ, 2, G.edges[2 * e], G.edges[2 * e + 1], 2 * l);
            for (int q = 0; q < G.n; ++q) gate(QS_RX, 1, q, 0, 2 * l + 1);
        }
        std::vector<double> prm((size_t)n_sets * 2 * p);
        for (int a = 0; a < n_sets; ++a)
            for (int l = 0; l < p; ++l) {
                prm[(size_t)a * 2 * p + 2 * l] = -gammas[(g * n_sets + a) * p + l];
                prm[(size_t)a * 2 * p + 2 * l + 1] = 2.0 * betas[(g * n_sets + a) * p + l];
            }
        // <H_C> = |E| / 2 - 1/2 sum_edges <Z_u Z_v>: Z-only terms (index bit of qubit q is n - 1 - q)
        std::vector<PauliDev> hz;
        hz.push_back({0.5 * G.n_edges, 0, 0});
        for (int e = 0; e < G.n_edges; ++e)
            hz.push_back({-0.5, 0, (1ull << (G.n - 1 - G.edges[2 * e])) | (1ull << (G.n - 1 - G.edges[2 * e + 1]))});
        rs = qs_init_zero(S);
        if (rs == QS_OK) rs = qs_apply_circuit(S, gl.data(), gl.size(), prm.data(), 2 * p, nullptr);
        if (rs == QS_OK) rs = diag_expect_async(S, hz, d_res + g * n_sets * 2);
    }
    if (rs == QS_OK && n_large) {
        std::vector<double> r(n_out * 2);
        cudaError_t e = cudaMemcpyAsync(r.data(), d_res, r.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rs = fail(QS_ERR_CUDA, std::string("qaoa results: ") + cudaGetErrorString(e));
        for (auto &kv : states)
            if (rs == QS_OK) rs = check_err_word(kv.second);
        if (rs == QS_OK)
            for (size_t g = 0; g < n_graphs; ++g)
                if (graphs[g].n > kQaoaMaxPersistentN)
                    for (int a = 0; a < n_sets; ++a) out[g * n_sets + a] = r[(g * n_sets + a) * 2];
    }
    if (d_res) {
        cudaStreamSynchronize(st);
        cudaFree(d_res);
    }
    for (auto &kv : states) qs_free(kv.second);
    return rs;
}

qs_status qs_qasm_parse(const char *src, qs_gate **gates, size_t *n_gates, int *n_qubits) {
    if (gates) *gates = nullptr;
    if (n_gates) *n_gates = 0;
    if (n_qubits) *n_qubits = 0;
    if (!src || !gates || !n_gates || !n_qubits) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    std::vector<qs_gate> out;
    int nq = 0;
    std::string err;
    const qs_status s = parse_qasm(src, out, nq, err);
    if (s != QS_OK) return fail(s, err);
    if (!out.empty()) {
        qs_gate *a = static_cast<qs_gate *>(std::malloc(out.size() * sizeof(qs_gate)));
        if (!a) return fail(QS_ERR_OOM, "gate array allocation failed");
        std::memcpy(a, out.data(), out.size() * sizeof(qs_gate));
        *gates = a;
    }
    *n_gates = out.size();
    *n_qubits = nq;
    return QS_OK;
}

void qs_qasm_free(qs_gate *gates) { std::free(gates); }

qs_status qs_plan_describe(int n, const qs_gate *gates, size_t n_gates, const qs_opts *opts, char *buf, size_t len,
                           int *passes) {
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_UNSUPPORTED, "n must be in [1, 33]");
    qs_opts o = default_opts(opts);
    std::vector<RGate> rg;
    std::string err;
    qs_status s = resolve_gates(n, gates, n_gates, nullptr, 0, 0, rg, err);
    if (s != QS_OK) return fail(s, err);
    Plan p;
    s = (o.mode == QS_MODE_PERGATE) ? build_pergate_plan(n, rg, p, err) : build_fused_plan(n, 1, rg, o, p, err);
    if (s != QS_OK) return fail(s, err);
    std::string d = p.describe();
    if (buf && len) {
        size_t c = std::min(len - 1, d.size());
        std::memcpy(buf, d.data(), c);
        buf[c] = 0;
    }
    if (passes) *passes = p.hbm_passes();
    return QS_OK;
}

qs_status qs_profile_enable(qs_state *st, int enable) {
    if (!st) return fail(QS_ERR_INVALID_ARG, "st == NULL");
    cudaStreamSynchronize(st->stream);
    for (auto &pe : st->prof_pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    st->prof_pending.clear();
    st->prof_recs.clear();
    st->prof = enable != 0;
    return QS_OK;
}

qs_status qs_profile_read(qs_state *st, qs_profile_record *out, int cap, int *count) {
    if (!st || !count || (cap > 0 && !out)) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    QS_CUDA(cudaStreamSynchronize(st->stream));
    for (auto &pe : st->prof_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pe.a, pe.b);
        ProfRec &r = st->prof_recs[pe.name];
        r.launches++;
        r.ms += ms;
        r.bytes += pe.bytes;
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    st->prof_pending.clear();
    int i = 0;
    for (auto &kv : st->prof_recs) {
        if (i >= cap) break;
        std::memset(&out[i], 0, sizeof(qs_profile_record));
        std::strncpy(out[i].name, kv.first.c_str(), 31);
        out[i].launches = kv.second.launches;
        out[i].total_ms = kv.second.ms;
        out[i].bytes = kv.second.bytes;
        ++i;
    }
    *count = i;
    return QS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {
struct TuneChoice {
    int T = 0, L = 0, R = 0;
    double ms = 0.0;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;   // key -> choice
std::map<std::string, bool> g_tune_files;   // cache files already read

std::string gpu_name(int dev) {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s(pr.name);
    for (char &ch : s)
        if (ch == ' ' || ch == '\t') ch = '_';
    return s;
}

// structure of a circuit: kinds, wires and parameter slots (not angle values)
uint64_t gate_structure_key(const qs_gate *g, size_t n_gates) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n_gates; ++i) {
        const int32_t rec[6] = {g[i].kind, g[i].nw, g[i].w[0], g[i].nw > 1 ? g[i].w[1] : -1,
                                g[i].nw > 2 ? g[i].w[2] : -1, g[i].param_idx >= 0 ? g[i].param_idx : -1};
        h = fnv1a(rec, sizeof rec, h);
    }
    return h;
}

void read_tune_file(const std::string &path) {
    if (g_tune_files.count(path)) return;
    g_tune_files[path] = true;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char tag[32], key[400];
        TuneChoice c;
        // "qs-autotune <key with '|' separators> T L R ms"
        if (std::sscanf(line, "%31s %399s %d %d %d %lf", tag, key, &c.T, &c.L, &c.R, &c.ms) == 6 &&
            std::strcmp(tag, "qs-autotune") == 0)
            g_tune[key] = c;
    }
    std::fclose(f);
}
}  // namespace

extern "C" qs_status qs_autotune(qs_state *st, const qs_gate *gates, size_t n_gates, const double *params,
                                 int n_params, const qs_opts *base, int reps, const char *cache_path, qs_opts *best,
                                 double *best_ms) {
    if (!st || !best) return fail(QS_ERR_INVALID_ARG, "NULL argument");
    if (reps < 1 || reps > 100) return fail(QS_ERR_INVALID_ARG, "reps must be in [1, 100]");
    if (n_gates && !gates) return fail(QS_ERR_INVALID_ARG, "gates == NULL");
    const qs_opts b = default_opts(base);
    if (b.mode != QS_MODE_FUSED) return fail(QS_ERR_INVALID_ARG, "the autotuner tunes the fused executor");
    {   // validate before allocating anything
        std::vector<RGate> rg;
        std::string err;
        const int items = params && has_param_gates(gates, n_gates) ? st->batch : 1;
        for (int bi = 0; bi < items; ++bi) {
            qs_status s = resolve_gates(st->n, gates, n_gates, params, n_params, bi, rg, err);
            if (s != QS_OK) return fail(s, err);
        }
    }
    char kbuf[400];
    std::snprintf(kbuf, sizeof kbuf, "%s|n%d|b%d|g%016llx|d%d|k%d", gpu_name(st->dev).c_str(), st->n, st->batch,
                  (unsigned long long)gate_structure_key(gates, n_gates), b.dense_prec, b.block_qubits);
    const std::string key(kbuf);
    auto fill = [&](const TuneChoice &c) {
        *best = b;
        best->tile_qubits = c.T;
        best->low_qubits = c.L;
        best->group_qubits = c.R;
        if (best_ms) *best_ms = c.ms;
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (cache_path) read_tune_file(cache_path);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            fill(it->second);
            return QS_OK;
        }
    }
    // candidates: the planner's choice first, then the explicit shapes
    std::vector<std::array<int, 3>> cand;
    cand.push_back({0, 0, 0});
    const int Rs[2] = {4, 5};
    for (int T : {12, 13})
        for (int L : {4, 5})
            for (int R : Rs) {
                if (b.dense_prec != QS_DENSE_OFF && R != 5) continue;
                const int t = std::min(T, st->n), l = std::min(L, t), r = std::min(R, t);
                std::array<int, 3> c = {t, l, r};
                if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
            }
    // a private copy of the state, on the same stream
    QS_CUDA(cudaStreamSynchronize(st->stream));
    qs_state *tr = nullptr;
    qs_status s = qs_alloc(st->n, st->batch, &tr);
    if (s != QS_OK) return s;
    cudaStreamSynchronize(nullptr);
    tr->stream = st->stream;
    const size_t bytes = (size_t)st->elems * st->batch * sizeof(float2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TuneChoice win;
    bool have = false;
    cudaError_t ce = cudaMemcpyAsync(tr->home, st->home, bytes, cudaMemcpyDeviceToDevice, st->stream);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) s = fail(QS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    for (size_t i = 0; i < cand.size() && s == QS_OK; ++i) {
        qs_opts o = b;
        o.tile_qubits = cand[i][0];
        o.low_qubits = cand[i][1];
        o.group_qubits = cand[i][2];
        qs_status r = qs_apply_circuit(tr, gates, n_gates, params, n_params, &o);
        // a shape this circuit cannot use (the gates themselves were validated above)
        if (r == QS_ERR_INTERNAL || r == QS_ERR_UNSUPPORTED || (r == QS_ERR_INVALID_ARG && i > 0)) continue;
        if (r != QS_OK) {
            s = r;
            break;
        }
        cudaEventRecord(e0, tr->stream);
        for (int k = 0; k < reps && r == QS_OK; ++k) r = qs_apply_circuit(tr, gates, n_gates, params, n_params, &o);
        cudaEventRecord(e1, tr->stream);
        ce = cudaEventSynchronize(e1);
        if (r != QS_OK) {
            s = r;
            break;
        }
        if (ce != cudaSuccess) {
            s = fail(QS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = (double)ms / reps;
        if (!have || per < win.ms) {
            win.T = cand[i][0];
            win.L = cand[i][1];
            win.R = cand[i][2];
            win.ms = per;
            have = true;
        }
    }
    if (s == QS_OK) s = check_err_word(tr);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st->stream);
    tr->stream = nullptr;
    qs_free(tr);
    if (s != QS_OK) return s;
    if (!have) return fail(QS_ERR_INTERNAL, "autotune: no candidate configuration could run");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = win;
        if (cache_path) {
            FILE *f = std::fopen(cache_path, "a");
            if (f) {
                std::fprintf(f, "qs-autotune %s %d %d %d %.6f\n", key.c_str(), win.T, win.L, win.R, win.ms);
                std::fclose(f);
            }
        }
    }
    fill(win);
    return QS_OK;
}
