// Host interpreter of fused plans: applies every pass of a plan the planner
// built (tile passes with their sweeps, micro-ops, diagonal descriptors,
// constant tables and dense blocks; permutation and gather passes) to a
// complex128 state, following the contracts the pass descriptors document,
// and checks the descriptors' structural invariants on the way:
//   * tile bits, sweep bits (group + item bits cover the tile once), table
//     limits (item bits, group table, micro-ops, sweeps, constants);
//   * shared-memory offsets: XOR-linear and one-to-one over the tile, equal to
//     the 128-byte swizzle of the dense tile-local order when the pass uses
//     it, pairs adjacent for 16-byte accesses;
//   * the TMA box: at the coordinates of every tile, the box enumerates exactly
//     that tile's amplitudes in tile-local order, inside the tensor, with an
//     aligned innermost coordinate, legal box extents and 16-byte strides;
//   * every constant read inside the pass's table; 16-byte constant loads at
//     even offsets; control masks off the target bits.
// Batches of parameter vectors: one plan per item, merged into one batched
// plan with per-item constants (as the executor does when the items' plans
// agree in structure); each item's state runs with its own constants and the
// TMA boxes are checked at the batch coordinate of every item.
// Input: a case file, one case per block:
//   case <n> <T> <L> <R> <dense_prec> <block> <mode> <count> <B> <P> <psi0.bin> <out.bin>
//   (mode: QS_MODE_FUSED or QS_MODE_PERGATE, whose one-op-per-launch plans
//   are applied by their own contract: each op over the subspace
//   (x & cmask) == cval)
//   then <count> gate lines: kind nw w0 w1 w2 p0 p1 p2 param_idx has_dense [8 doubles]
//   then B x P parameter values (item after item)
// psi0 / out: B x 2^n complex128, or "-" for both: structure only (every
// invariant, the boxes of 8 sampled tiles per pass; no state).  Prints one "CASE <i> ..." line per case
// with the pass and micro-op counts, or "FAIL <i> <reason>" and exits 1.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qs_internal.h"
#include "qs_plan.h"

using namespace qs;
using C = std::complex<double>;

namespace {

int popc(uint64_t x) {
    int c = 0;
    while (x) {
        x &= x - 1;
        ++c;
    }
    return c;
}

struct Counts {
    long micro[13] = {0};
    long dense[4] = {0};
    long tile = 0, perm = 0, gather = 0, tma = 0, rows = 0, swz = 0, sweeps = 0, pergate = 0;
};

struct Fail {
    std::string why;
};

// exp(i pi u / 2^p)
C twiddle(uint64_t u, int p) {
    if (p == 0 || u == 0) return 1.0;
    return std::polar(1.0, M_PI * (double)u / std::ldexp(1.0, p));
}

// float -> BF16 -> float, round to nearest even
double bf16(double x) {
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    std::memcpy(&f, &u, 4);
    return f;
}

double bf16_half(uint32_t w, int half) {
    uint32_t u = ((w >> (16 * half)) & 0xffffu) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

class TileRun {
  public:
    // item: which item's constants; batch: states in the tensor the boxes address
    TileRun(int n, const HostPass &hp, Counts &cnt, int item, int items, int batch)
        : n_(n), hp_(hp), P_(hp.tile), cnt_(cnt), item_(item), items_(items), batch_(batch) {}

    // psi: the item's state, at position `bi` of the batch
    void run(C *psi, int bi) {
        bi_ = bi;
        structure();
        const int T = P_.T;
        std::vector<uint64_t> outer;
        for (int b = 0; b < n_; ++b)
            if (!((tilebits_ >> b) & 1)) outer.push_back(b);
        std::vector<C> tile((size_t)1 << T);
        for (uint64_t ti = 0; ti < (1ull << outer.size()); ++ti) {
            uint64_t base = 0;
            for (size_t i = 0; i < outer.size(); ++i)
                if ((ti >> i) & 1) base |= 1ull << outer[i];
            if (hp_.tma.ok) check_box(ti, base);
            for (uint64_t t = 0; t < tile.size(); ++t) tile[t] = psi[base | glob(t)];
            for (int s = 0; s < P_.n_sweeps; ++s) sweep(P_.sweeps[s], tile, base);
            for (uint64_t t = 0; t < tile.size(); ++t) psi[base | glob(t)] = tile[t];
        }
    }

    // structure only (states too large for the host): every invariant of the
    // pass, the tensor-copy box of 8 sampled tiles (the first, the last, six
    // pseudo-random ones), and the sweeps run on a zero tile of each (constant
    // bounds, micro-op and diagonal invariants)
    void check_only(int bi, uint64_t seed) {
        bi_ = bi;
        structure();
        std::vector<uint64_t> outer;
        for (int b = 0; b < n_; ++b)
            if (!((tilebits_ >> b) & 1)) outer.push_back(b);
        std::vector<C> tile((size_t)1 << P_.T);
        const uint64_t n_tiles = 1ull << outer.size();
        uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
        for (int k = 0; k < 8; ++k) {
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            const uint64_t ti = k == 0 ? 0 : k == 1 ? n_tiles - 1 : x % n_tiles;
            uint64_t base = 0;
            for (size_t i = 0; i < outer.size(); ++i)
                if ((ti >> i) & 1) base |= 1ull << outer[i];
            if (hp_.tma.ok) check_box(ti, base);
            std::fill(tile.begin(), tile.end(), C(0.0));
            for (int s = 0; s < P_.n_sweeps; ++s) sweep(P_.sweeps[s], tile, base);
        }
    }

  private:
    int n_;
    const HostPass &hp_;
    const TilePass &P_;
    Counts &cnt_;
    int item_, items_, batch_, bi_ = 0;
    uint64_t tilebits_ = 0;
    int gbit_[kMaxTileBits];   // global bit of tile-local bit k

    [[noreturn]] void fail(const std::string &w) { throw Fail{w}; }
    void need(bool c, const std::string &w) {
        if (!c) fail(w);
    }
    uint64_t glob(uint64_t t) const {
        uint64_t g = 0;
        for (int k = 0; k < P_.T; ++k)
            if ((t >> k) & 1) g |= 1ull << gbit_[k];
        return g;
    }
    C K(long i) {
        const float2 &v = Kraw(i);
        return C(v.x, v.y);
    }
    const float2 &Kraw(long i) {
        need(i >= 0 && i < P_.n_const, "constant index " + std::to_string(i) + " outside the table");
        return hp_.consts[(size_t)item_ * P_.n_const + i];
    }

    void structure() {
        const int T = P_.T, L = P_.L, H = P_.H;
        need(T == L + H && T >= 1 && T <= kMaxTileBits && T <= n_ && L >= 1, "tile shape");
        need(P_.n == n_, "pass n");
        for (int k = 0; k < L; ++k) gbit_[k] = k;
        for (int k = 0; k < H; ++k) {
            need(P_.hb[k] >= L && P_.hb[k] < n_ && (k == 0 || P_.hb[k] > P_.hb[k - 1]), "high bits ascending");
            gbit_[L + k] = P_.hb[k];
        }
        for (int k = 0; k < T; ++k) tilebits_ |= 1ull << gbit_[k];
        need(P_.n_sweeps >= 1 && P_.n_sweeps <= kMaxSweeps, "sweep count");
        need(P_.n_micro >= 0 && P_.n_micro <= kMaxMicro, "micro-op count");
        bool dense = false;
        for (int s = 0; s < P_.n_sweeps; ++s) dense |= P_.sweeps[s].dense != DS_NONE;
        need(P_.n_const >= 0 && P_.n_const <= (dense ? kMaxConstDense : kMaxConst), "constant count");
        need((long)hp_.consts.size() == (long)items_ * P_.n_const, "constant vector size");
        // shared-memory offsets: XOR-linear, one-to-one over [0, 2^T)
        std::vector<uint32_t> basis;
        for (int k = 0; k < T; ++k) {
            const uint32_t c = (uint32_t)P_.smem_contrib[k];
            need(c < (1u << T), "offset outside the tile buffer");
            if (P_.swizzle) {
                const uint32_t d = 1u << k;   // 128-byte swizzle: 16-byte chunk ^= 128-byte row mod 8
                need(c == (d ^ (((d >> 4) & 7u) << 1)), "swizzled offset of tile bit " + std::to_string(k));
            } else {
                need(c == (1u << k), "dense offset of tile bit " + std::to_string(k));
            }
            uint32_t v = c;
            for (uint32_t b : basis)
                if ((v ^ b) < v) v ^= b;
            need(v != 0, "offsets not one-to-one");
            basis.push_back(v);
            for (size_t i = basis.size() - 1; i > 0 && basis[i] > basis[i - 1]; --i) std::swap(basis[i], basis[i - 1]);
        }
        need(!P_.swizzle || hp_.tma.ok, "swizzle without the tensor copy");
        if (hp_.tma.ok) {
            const TmaPlan &g = hp_.tma;
            need(g.ndims >= 1 && g.ndims <= 5, "tensor rank");
            need(g.box[0] * 8 % 16 == 0, "inner box extent not a multiple of 16 bytes");
            if (P_.swizzle) need(g.box[0] * 8 <= 128, "inner box wider than the swizzle span");
            uint64_t vol = 1;
            need(batch_ == 1 || g.batch_dim >= 0, "batched tensor copy without a batch dim");
            for (int d = 0; d < 5; ++d) {
                need(g.box[d] >= 1 && g.box[d] <= 256 && g.box[d] <= g.gdim[d], "box extent");
                if (d >= 1) need(g.gstride[d] % 16 == 0, "stride not a multiple of 16 bytes");
                if (d >= g.ndims) need(g.gdim[d] == 1 && g.box[d] == 1, "unused tensor dim");
                vol *= g.box[d];
            }
            need(vol == (1ull << T), "box volume");
            cnt_.tma++;
        } else {
            cnt_.rows++;
        }
        if (P_.swizzle) cnt_.swz++;
        cnt_.tile++;
    }

    // the tensor copy of tile `ti` covers exactly the tile, in tile-local order
    void check_box(uint64_t ti, uint64_t base) {
        const TmaPlan &g = hp_.tma;
        long long c[5];
        for (int d = 0; d < 5; ++d) {
            long long v = 0;
            if (d < g.ndims && g.kind[d] == 1) v = (long long)((ti >> g.off[d]) & ((1ull << g.w[d]) - 1));
            if (d < g.ndims && d == g.batch_dim) v += (long long)bi_ << g.w[d];
            c[d] = v;
            need(v + g.box[d] <= (long long)g.gdim[d], "box outside the tensor");
        }
        need((c[0] * 8) % 16 == 0, "innermost coordinate not 16-byte aligned");
        uint64_t t = 0;
        for (uint32_t e4 = 0; e4 < g.box[4]; ++e4)
            for (uint32_t e3 = 0; e3 < g.box[3]; ++e3)
                for (uint32_t e2 = 0; e2 < g.box[2]; ++e2)
                    for (uint32_t e1 = 0; e1 < g.box[1]; ++e1)
                        for (uint32_t e0 = 0; e0 < g.box[0]; ++e0, ++t) {
                            const uint64_t e[5] = {e0, e1, e2, e3, e4};
                            uint64_t byte = (c[0] + e0) * 8;
                            for (int d = 1; d < 5; ++d) byte += (c[d] + e[d]) * g.gstride[d];
                            const uint64_t want = ((uint64_t)bi_ << n_) + (base | glob(t));
                            need(byte % 8 == 0 && byte / 8 == want, "box element of tile " + std::to_string(ti) +
                                                                         " of item " + std::to_string(bi_));
                        }
    }

    void sweep(const Sweep &S, std::vector<C> &tile, uint64_t tbase) {
        const int T = P_.T, r = S.r;
        cnt_.sweeps++;
        need(r >= 1 && r <= kMaxGroup && r <= kGroupTab && r <= T, "group size");
        const int nb = T - r;
        need(nb <= 14, "more item bits than the item tables hold");
        uint64_t seen = 0;
        for (int m = 0; m < r; ++m) seen |= 1ull << S.gbit[m];
        for (int i = 0; i < nb; ++i) seen |= 1ull << S.tbit[i];
        need(seen == (T >= 64 ? ~0ull : (1ull << T) - 1) && popc(seen) == T, "sweep bits do not cover the tile");
        if (S.vec) {
            need(P_.smem_contrib[S.gbit[0]] == 1, "paired access without adjacent pairs");
            for (int k = 0; k < T; ++k)
                if (k != S.gbit[0]) need(P_.smem_contrib[k] % 2 == 0, "paired access not 16-byte aligned");
        }
        if (S.dense) {
            dense(S, tile);
            return;
        }
        need(S.op_begin >= 0 && S.op_begin <= S.op_end && S.op_end <= P_.n_micro, "micro-op range");
        uint64_t gg[kMaxGroup];
        for (int m = 0; m < r; ++m) gg[m] = 1ull << gbit_[S.gbit[m]];
        std::vector<C> a((size_t)1 << r);
        for (uint64_t item = 0; item < (1ull << nb); ++item) {
            uint64_t tl = 0;
            for (int i = 0; i < nb; ++i)
                if ((item >> i) & 1) tl |= 1ull << S.tbit[i];
            const uint64_t gbase = tbase | glob(tl);
            auto elem = [&](int j) {
                uint64_t t = tl;
                for (int m = 0; m < r; ++m)
                    if ((j >> m) & 1) t |= 1ull << S.gbit[m];
                return t;
            };
            auto gidx = [&](int j) {
                uint64_t x = gbase;
                for (int m = 0; m < r; ++m)
                    if ((j >> m) & 1) x |= gg[m];
                return x;
            };
            for (int j = 0; j < (1 << r); ++j) a[j] = tile[elem(j)];
            for (int oi = S.op_begin; oi < S.op_end; ++oi) op(P_.micro[oi], r, gg, gbase, a, gidx, item == 0);
            for (int j = 0; j < (1 << r); ++j) tile[elem(j)] = a[j] * (double)S.scale;
        }
    }

    template <class GI>
    void u1(int m, int r, std::vector<C> &a, C m00, C m01, C m10, C m11, uint64_t cmask, uint64_t cval, GI &gidx) {
        need(m >= 0 && m < r, "target bit outside the group");
        for (int j = 0; j < (1 << r); ++j) {
            if ((j >> m) & 1) continue;
            if (cmask && (gidx(j) & cmask) != cval) continue;
            const int k = j | (1 << m);
            const C a0 = a[j], a1 = a[k];
            a[j] = m00 * a0 + m01 * a1;
            a[k] = m10 * a0 + m11 * a1;
        }
    }
    void qft(int m, int r, std::vector<C> &a, long gtab, C w) {
        need(m >= 0 && m < r, "QFT bit outside the group");
        for (int j = 0; j < (1 << r); ++j) {
            if ((j >> m) & 1) continue;
            const int k = j | (1 << m);
            const C a0 = a[j], a1 = a[k];
            a[j] = a0 + a1;
            a[k] = (a0 - a1) * w * K(gtab + k);
        }
    }
    void layer_bit(int kind, int m, int r, std::vector<C> &a, long k0) {
        auto no = [](int) { return 0ull; };
        switch (kind) {
            case MK_RXC: {
                const C cs = K(k0 + m);
                const double c = cs.real(), s = cs.imag();
                u1(m, r, a, c, C(0, s), C(0, s), c, 0, 0, no);
                break;
            }
            case MK_U1R: {
                const long o = k0 + 4 * m;
                need(o % 2 == 0, "packed real 2x2 constants at an odd offset");
                const float2 q0 = Kraw(o), q1 = Kraw(o + 1), q2 = Kraw(o + 2), q3 = Kraw(o + 3);
                need(q0.x == q0.y && q1.x == q1.y && q2.x == q2.y && q3.x == q3.y, "real 2x2 not packed as pairs");
                u1(m, r, a, q0.x, q1.x, q2.x, q3.x, 0, 0, no);
                break;
            }
            case MK_U1:
                u1(m, r, a, K(k0 + 4 * m), K(k0 + 4 * m + 1), K(k0 + 4 * m + 2), K(k0 + 4 * m + 3), 0, 0, no);
                break;
            case MK_ROT: {
                // [[1, t], [-t, 1]]; the factor c is in the sweep scale
                const float2 q0 = Kraw(k0 + 2 * m), q1 = Kraw(k0 + 2 * m + 1);
                need(q0.x == q0.y && q1.x == q1.y && q1.x == -q0.x, "rotation not packed as (t, t), (-t, -t)");
                need(std::abs(q0.x) <= 1.f, "rotation tangent above 1");
                u1(m, r, a, 1.0, q0.x, q1.x, 1.0, 0, 0, no);
                break;
            }
            case MK_H:
                u1(m, r, a, 1.0, 1.0, 1.0, -1.0, 0, 0, no);
                break;
            default:
                fail("layer of kind " + std::to_string(kind));
        }
    }

    C diag_part(const DiagDesc &d, uint64_t x, uint32_t smask, uint32_t gmask, C ph) {
        for (int s = 0; s < d.n_slices; ++s)
            if ((smask >> s) & 1) ph *= K(d.slice_off[s] + (long)((x >> d.slice_lo[s]) & ((1ull << d.slice_w[s]) - 1)));
        for (int g = 0; g < d.n_groups; ++g)
            if ((gmask >> g) & 1) {
                const uint64_t f = d.grp_type[g] ? (x & (x >> d.grp_d[g])) : (x ^ (x >> d.grp_d[g]));
                ph *= K(d.grp_off[g] + popc(f & d.grp_mask[g]));
            }
        return ph;
    }

    template <class GI>
    void op(const MicroOp &o, int r, const uint64_t *gg, uint64_t gbase, std::vector<C> &a, GI &gidx, bool first) {
        need(o.kind >= 0 && o.kind <= MK_ZYZ, "micro-op kind");
        if (first) {
            cnt_.micro[o.kind]++;
            // a layer also exercises its op kind (lone rotations become one-bit layers)
            if (o.kind == MK_LAYER && o.a >= 0 && o.a <= MK_ROT) cnt_.micro[o.a]++;
        }
        uint64_t gmask = 0;
        for (int m = 0; m < r; ++m) gmask |= gg[m];
        switch (o.kind) {
            case MK_U1:
                need(o.a >= 0 && o.a < r && !(o.cmask & gg[o.a]), "control on the target bit");
                u1(o.a, r, a, K(o.cst), K(o.cst + 1), K(o.cst + 2), K(o.cst + 3), o.cmask, o.cval, gidx);
                break;
            case MK_H:
            case MK_RXC:
            case MK_U1R:
            case MK_ROT:
                layer_bit(o.kind, o.a, r, a,
                          o.cst - (o.kind == MK_RXC ? o.a : o.kind == MK_U1R ? 4 * o.a : o.kind == MK_ROT ? 2 * o.a : 0));
                break;
            case MK_U2: {
                need(o.a >= 0 && o.a < r && o.b >= 0 && o.b < r && o.a != o.b, "4x4 bits");
                need(!(o.cmask & (gg[o.a] | gg[o.b])), "control on a target bit");
                C M[16];
                for (int e = 0; e < 16; ++e) M[e] = K(o.cst + e);
                for (int j = 0; j < (1 << r); ++j) {
                    if (((j >> o.a) & 1) || ((j >> o.b) & 1)) continue;
                    if (o.cmask && (gidx(j) & o.cmask) != o.cval) continue;
                    const int id[4] = {j, j | (1 << o.b), j | (1 << o.a), j | (1 << o.a) | (1 << o.b)};
                    C v[4], w[4];
                    for (int i = 0; i < 4; ++i) v[i] = a[id[i]];
                    for (int q = 0; q < 4; ++q) w[q] = M[4 * q] * v[0] + M[4 * q + 1] * v[1] + M[4 * q + 2] * v[2] +
                                                       M[4 * q + 3] * v[3];
                    for (int i = 0; i < 4; ++i) a[id[i]] = w[i];
                }
                break;
            }
            case MK_QFT: {
                need(o.p >= 0 && o.p <= 32 && o.lo >= 0 && o.lo <= o.p, "QFT stage bits");
                need(gg[o.a] == (1ull << o.p), "QFT stage bit is not the group bit");
                const uint64_t mk = (o.p > o.lo) ? (((1ull << o.p) - 1) & ~((1ull << o.lo) - 1)) : 0;
                qft(o.a, r, a, o.cst, twiddle(gbase & mk, o.p));
                break;
            }
            case MK_ZYZ: {
                // input phases, rotations in one-FMA form, output phases, then
                // element j of the result is the computed value j ^ F
                const int P = 1 << r;
                need(o.cst >= 0, "U(2) layer constants");
                auto no = [](int) { return 0ull; };
                for (int j = 0; j < P; ++j) a[j] *= K(o.cst + j);
                for (int m = 0; m < r; ++m) {
                    const float2 q0 = Kraw(o.cst + 2 * P + 2 * m), q1 = Kraw(o.cst + 2 * P + 2 * m + 1);
                    need(q0.x == q0.y && q1.x == q1.y && q1.x == -q0.x, "U(2) rotation not packed as (k, k), (-k, -k)");
                    need(std::abs(q0.x) <= 1.f, "U(2) rotation coefficient above 1");
                    u1(m, r, a, 1.0, q0.x, q1.x, 1.0, 0, 0, no);
                }
                for (int j = 0; j < P; ++j) a[j] *= K(o.cst + P + j);
                int F;
                const float2 fe = Kraw(o.cst + 2 * P + 2 * r);
                std::memcpy(&F, &fe.x, 4);
                need(F >= 0 && F < P, "U(2) exchange mask");
                std::vector<C> b(a);
                for (int j = 0; j < P; ++j) a[j ^ F] = b[j];
                break;
            }
            case MK_LAYER: {
                need(o.b > 0 && o.b < (1 << r), "layer mask");
                // a rotation program's layer: the bits outside its own (lo) are
                // identities, which the kernel may skip
                if (o.a == MK_ROT && o.lo) {
                    need((o.lo & ~o.b) == 0, "rotation layer's own bits outside its mask");
                    for (int m = 0; m < r; ++m)
                        if (((o.b >> m) & 1) && !((o.lo >> m) & 1))
                            need(Kraw(o.cst + 2 * m).x == 0.f && Kraw(o.cst + 2 * m + 1).x == 0.f,
                                 "padded rotation bit is not the identity");
                }
                if (o.a == MK_U1R) need(o.cst % 2 == 0, "packed real 2x2 layer at an odd offset");
                for (int m = 0; m < r; ++m)
                    if ((o.b >> m) & 1) layer_bit(o.a, m, r, a, o.cst);
                break;
            }
            case MK_QFTL: {
                need(o.b > 0 && o.b < (1 << r), "QFT ladder mask");
                for (int m = r - 1; m >= 0; --m)
                    if ((o.b >> m) & 1) {
                        const int p = (int)((o.cmask >> (6 * m)) & 63);
                        need(p <= 32 && gg[m] == (1ull << p), "QFT ladder bit");
                        qft(m, r, a, o.cst + (long)m * (1 << r), twiddle(gbase & ((1ull << p) - 1), p));
                    }
                break;
            }
            case MK_DIAG: {
                need(o.cst >= 0 && o.cst < kMaxDiag, "diagonal index");
                const DiagDesc &d = P_.diags[o.cst];
                need(d.n_tw == 0 && d.n_slices <= kMaxSlices && d.n_groups <= kMaxLutGroups, "diagonal descriptor");
                const uint32_t dyn_s = (uint32_t)o.a, dyn_g = (uint32_t)o.b;
                // the factors outside the dynamic masks must not see the group bits
                for (int s = 0; s < d.n_slices; ++s)
                    if (!((dyn_s >> s) & 1)) {
                        const uint64_t sm = ((1ull << d.slice_w[s]) - 1) << d.slice_lo[s];
                        need(!(sm & gmask), "static slice depends on the group bits");
                    }
                for (int g = 0; g < d.n_groups; ++g)
                    if (!((dyn_g >> g) & 1)) {
                        const uint64_t m1 = d.grp_mask[g], m2 = d.grp_mask[g] << d.grp_d[g];
                        need(!((m1 | m2) & gmask), "static LUT group depends on the group bits");
                    }
                C stat = d.pad0 ? K(d.gph_off) : C(1.0);
                stat = diag_part(d, gbase, ~dyn_s, ~dyn_g, stat);
                for (int j = 0; j < (1 << r); ++j) a[j] *= diag_part(d, gidx(j), dyn_s, dyn_g, stat);
                break;
            }
            case MK_DIAGQ: {
                need(o.cst >= 0 && o.cst < kMaxDiag, "diagonal index");
                const DiagDesc &d = P_.diags[o.cst];
                need(d.n_tw == 0, "diagonal descriptor");
                std::vector<C> z((size_t)1 << r);
                z[0] = d.pad0 ? K(d.gph_off) : C(1.0);
                z[0] = diag_part(d, gbase, ~0u, ~0u, z[0]);
                for (int m = 0; m < r; ++m) {
                    C e = 1.0;
                    const int cnt = (int)((o.cmask >> (6 * m)) & 63);
                    need(cnt <= kMaxCouple, "coupling count");
                    for (int k = 0; k < cnt; ++k) {
                        const float2 ent = Kraw(o.lo + 2 * m * kMaxCouple + 2 * k);
                        int b;
                        std::memcpy(&b, &ent.x, 4);
                        need(b >= 0 && b < n_ && !((1ull << b) & gmask), "coupling bit");
                        if ((gbase >> b) & 1) e *= K(o.lo + 2 * m * kMaxCouple + 2 * k + 1);
                    }
                    for (int j = 0; j < (1 << m); ++j) z[j | (1 << m)] = z[j] * e;
                }
                for (int j = 0; j < (1 << r); ++j) a[j] *= z[j] * K(o.p + j);
                break;
            }
            case MK_DIAGC: {
                need(o.a >= 0 && o.a <= kMaxCountClasses, "count-table classes");
                auto slot = [&](int i) {
                    const float2 &lo = Kraw(o.lo + i);
                    uint64_t v;
                    std::memcpy(&v, &lo, 8);
                    return v;
                };
                const bool cz = o.b != 0;
                const uint64_t degs = slot(r), mz = slot(r + 1), zinc = slot(r + 2);
                need(!(gbase & gmask), "item base has group bits set");
                int c0 = o.p * popc(gbase & mz);
                for (int k = 0; k < o.a; ++k) {
                    const uint64_t m = slot(r + 3 + 2 * k);
                    const int d = (int)slot(r + 4 + 2 * k);
                    need(d >= 1 && d < 64, "class distance");
                    const uint64_t f = cz ? (gbase & (gbase >> d)) : (gbase ^ (gbase >> d));
                    c0 += popc(f & m);
                }
                std::vector<int> cnt((size_t)1 << r);
                cnt[0] = c0;
                for (int m = 0; m < r; ++m) {
                    const uint64_t nm = slot(m);
                    need(!(nm & gmask), "neighbour mask holds group bits");
                    const int s = popc(gbase & nm);
                    const int dm = (cz ? s : (int)((degs >> (6 * m)) & 63) - 2 * s) + (int)((zinc >> (12 * m)) & 4095);
                    for (int j = 0; j < (1 << m); ++j) cnt[j | (1 << m)] = cnt[j] + dm;
                }
                for (int j = 0; j < (1 << r); ++j) {
                    const uint64_t qw = j < 16 ? o.cmask : o.cval;
                    const int q = (int)((qw >> (4 * (j & 15))) & 15);
                    need(cnt[j] + q >= 0, "negative count");
                    a[j] *= K(o.cst + cnt[j] + q);
                }
                break;
            }
            default:
                fail("micro-op kind " + std::to_string(o.kind));
        }
    }

    // dense block: out = U X on the 5 group bits (row), per column of item bits
    void dense(const Sweep &S, std::vector<C> &tile) {
        need(S.r == 5 && S.op_begin == S.op_end && S.scale == 1.f, "dense sweep shape");
        need(S.dense >= DS_FP32 && S.dense <= DS_BF16, "dense kind");
        need(S.dcst % 2 == 0, "dense constants at an odd offset");
        cnt_.dense[S.dense]++;
        const int T = P_.T, nb = T - 5;
        // real 64 x 64 form: row 2 i + (0 re, 1 im) of the input, column 2 o + (0 re, 1 im) of the output
        std::vector<double> B(64 * 64, 0.0);
        auto put_complex = [&](int o, int i, C u) {
            B[(2 * i) * 64 + 2 * o] = u.real();
            B[(2 * i + 1) * 64 + 2 * o] = -u.imag();
            B[(2 * i) * 64 + 2 * o + 1] = u.imag();
            B[(2 * i + 1) * 64 + 2 * o + 1] = u.real();
        };
        if (S.dense == DS_FP32) {
            for (int o = 0; o < 32; ++o)
                for (int i = 0; i < 32; ++i) put_complex(o, i, K(S.dcst + o * 32 + i));
        } else if (S.dense == DS_TF32X3) {
            // tensor-core B operands: Re U hi, Im U hi, Re U lo, Im U lo, each 32 x 32
            // floats K-major (row = output o), 128-byte swizzle, 1024-byte aligned
            need(S.dcst % 128 == 0, "tensor-core operands not on a 1024-byte boundary");
            auto f = [&](int mat, int o, int i) {
                const long e = 1024L * mat + o * 32 + (((i >> 2) ^ (o & 7)) << 2) + (i & 3);
                const float2 v = Kraw(S.dcst + e / 2);
                return (double)((e & 1) ? v.y : v.x);
            };
            for (int o = 0; o < 32; ++o)
                for (int i = 0; i < 32; ++i)
                    put_complex(o, i, C(f(0, o, i) + f(2, o, i), f(1, o, i) + f(3, o, i)));
        } else {
            // m16n8k16 B fragments (PTX ISA): register h of lane l holds k = 2 (l % 4) + 8 h + {0, 1},
            // n = l / 4; k-step s covers input rows 8 s .. 8 s + 7, n-tile t output rows 4 t .. 4 t + 3
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 8; ++t)
                    for (int l = 0; l < 32; ++l) {
                        const float2 v = Kraw(S.dcst + (s * 8 + t) * 32 + l);
                        uint32_t w[2];
                        std::memcpy(&w[0], &v.x, 4);
                        std::memcpy(&w[1], &v.y, 4);
                        for (int h = 0; h < 2; ++h)
                            for (int e = 0; e < 2; ++e) {
                                const int k = 16 * s + 2 * (l % 4) + 8 * h + e, nn = 8 * t + l / 4;
                                B[k * 64 + nn] = bf16_half(w[h], e);
                            }
                    }
        }
        for (uint64_t col = 0; col < (1ull << nb); ++col) {
            uint64_t tl = 0;
            for (int i = 0; i < nb; ++i)
                if ((col >> i) & 1) tl |= 1ull << S.tbit[i];
            double x[64], y[64];
            uint64_t idx[32];
            for (int row = 0; row < 32; ++row) {
                uint64_t t = tl;
                for (int q = 0; q < 5; ++q)
                    if ((row >> q) & 1) t |= 1ull << S.gbit[q];
                idx[row] = t;
                x[2 * row] = tile[t].real();
                x[2 * row + 1] = tile[t].imag();
                if (S.dense == DS_BF16) {
                    x[2 * row] = bf16(x[2 * row]);
                    x[2 * row + 1] = bf16(x[2 * row + 1]);
                }
            }
            for (int c = 0; c < 64; ++c) {
                double acc = 0;
                for (int k = 0; k < 64; ++k) acc += x[k] * B[k * 64 + c];
                y[c] = acc;
            }
            for (int row = 0; row < 32; ++row) tile[idx[row]] = C(y[2 * row], y[2 * row + 1]);
        }
    }
};

void run_perm(int n, const PermPass &pp, C *psi) {
    if (pp.n != n) throw Fail{"perm n"};
    uint64_t used = 0;
    for (int b = 0; b < n; ++b) {
        if (pp.out_pos[b] < 0 || pp.out_pos[b] >= n) throw Fail{"perm target"};
        used |= 1ull << pp.out_pos[b];
    }
    if (popc(used) != n) throw Fail{"perm is not a permutation"};
    const uint64_t N = 1ull << n;
    std::vector<C> out(N);
    for (uint64_t x = 0; x < N; ++x) {
        uint64_t y = 0;
        for (int b = 0; b < n; ++b)
            if ((x >> b) & 1) y |= 1ull << pp.out_pos[b];
        out[y ^ pp.xor_mask] = psi[x];
    }
    std::copy(out.begin(), out.end(), psi);
}

void run_gather(int n, const GatherPass &gp, C *psi) {
    if (gp.n != n || gp.n_slices < 1 || gp.n_slices > 5 || 8 * gp.n_slices < n) throw Fail{"gather slices"};
    const uint64_t N = 1ull << n;
    std::vector<C> out(N);
    std::vector<char> hit(N, 0);
    for (uint64_t y = 0; y < N; ++y) {
        uint64_t x = gp.c;
        for (int k = 0; k < gp.n_slices; ++k) x ^= gp.tab[k][(y >> (8 * k)) & 255];
        if (x >= N) throw Fail{"gather source outside the state"};
        if (hit[x]) throw Fail{"gather is not a bijection"};
        hit[x] = 1;
        out[y] = psi[x];
    }
    std::copy(out.begin(), out.end(), psi);
}

// one per-gate launch: U1 = 2x2 on bit t0, U2 = 4x4 on (t0 = matrix MSB, t1),
// PHASE = amp *= m[bit t0 | bit t1 << 1] (nbits_phase of them; 0: m[0]),
// SWAP = exchange of bits t0 and t1; every op only where (x & cmask) == cval
void run_pergate(int n, const PgOp &op, C *psi) {
    const uint64_t N = 1ull << n;
    auto M = [&](int e) { return C(op.m[e].x, op.m[e].y); };
    if ((op.cval & ~op.cmask) != 0) throw Fail{"per-gate control value outside its mask"};
    const uint64_t b0 = op.t0 >= 0 ? 1ull << op.t0 : 0, b1 = op.t1 >= 0 ? 1ull << op.t1 : 0;
    switch (op.kind) {
        case PG_U1:
            if (op.t0 < 0 || op.t0 >= n || (op.cmask & b0)) throw Fail{"per-gate U1 target"};
            for (uint64_t x = 0; x < N; ++x) {
                if ((x & b0) || (x & op.cmask) != op.cval) continue;
                const C a0 = psi[x], a1 = psi[x | b0];
                psi[x] = M(0) * a0 + M(1) * a1;
                psi[x | b0] = M(2) * a0 + M(3) * a1;
            }
            break;
        case PG_U2: {
            if (op.t0 < 0 || op.t1 < 0 || op.t0 >= n || op.t1 >= n || op.t0 == op.t1 || (op.cmask & (b0 | b1)))
                throw Fail{"per-gate U2 targets"};
            for (uint64_t x = 0; x < N; ++x) {
                if ((x & (b0 | b1)) || (x & op.cmask) != op.cval) continue;
                const uint64_t id[4] = {x, x | b1, x | b0, x | b0 | b1};
                C v[4], w[4];
                for (int i = 0; i < 4; ++i) v[i] = psi[id[i]];
                for (int r = 0; r < 4; ++r) w[r] = M(4 * r) * v[0] + M(4 * r + 1) * v[1] + M(4 * r + 2) * v[2] +
                                                   M(4 * r + 3) * v[3];
                for (int i = 0; i < 4; ++i) psi[id[i]] = w[i];
            }
            break;
        }
        case PG_PHASE:
            if (op.nbits_phase < 0 || op.nbits_phase > 2) throw Fail{"per-gate phase bits"};
            for (uint64_t x = 0; x < N; ++x) {
                if ((x & op.cmask) != op.cval) continue;
                int idx = 0;
                if (op.nbits_phase >= 1) idx |= (int)((x >> op.t0) & 1);
                if (op.nbits_phase >= 2) idx |= (int)((x >> op.t1) & 1) << 1;
                psi[x] *= M(idx);
            }
            break;
        case PG_SWAP:
            if (op.t0 < 0 || op.t1 < 0 || op.t0 == op.t1 || (op.cmask & (b0 | b1))) throw Fail{"per-gate swap bits"};
            for (uint64_t x = 0; x < N; ++x) {
                if ((x & (b0 | b1)) || (x & op.cmask) != op.cval) continue;
                std::swap(psi[x | b0], psi[x | b1]);
            }
            break;
        default:
            throw Fail{"per-gate op kind"};
    }
}

}  // namespace

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *fp = std::fopen(argv[1], "r");
    if (!fp) return 2;
    int n, T, L, R, dprec, block, mode, cnt, B, NP, ci = 0;
    char in_path[4096], out_path[4096];
    while (std::fscanf(fp, " case %d %d %d %d %d %d %d %d %d %d %4095s %4095s", &n, &T, &L, &R, &dprec, &block, &mode,
                       &cnt, &B, &NP, in_path, out_path) == 12) {
        std::vector<qs_gate> gl(cnt);
        std::vector<std::vector<double>> dense(cnt);
        for (int i = 0; i < cnt; ++i) {
            int kind, nw, w0, w1, w2, pidx, hd;
            double p0, p1, p2;
            if (std::fscanf(fp, "%d %d %d %d %d %lf %lf %lf %d %d", &kind, &nw, &w0, &w1, &w2, &p0, &p1, &p2, &pidx,
                            &hd) != 10)
                return 2;
            qs_gate &g = gl[i];
            std::memset(&g, 0, sizeof g);
            g.kind = (uint16_t)kind;
            g.nw = (uint8_t)nw;
            g.w[0] = w0;
            g.w[1] = w1;
            g.w[2] = w2;
            g.p[0] = p0;
            g.p[1] = p1;
            g.p[2] = p2;
            g.param_idx = pidx;
            if (hd) {
                dense[i].resize(8);
                for (int e = 0; e < 8; ++e)
                    if (std::fscanf(fp, "%lf", &dense[i][e]) != 1) return 2;
                g.dense = dense[i].data();
            }
        }
        std::vector<double> params((size_t)B * NP);
        for (auto &v : params)
            if (std::fscanf(fp, "%lf", &v) != 1) return 2;
        qs_opts o;
        std::memset(&o, 0, sizeof o);
        o.mode = QS_MODE_FUSED;
        o.tile_qubits = T;
        o.low_qubits = L;
        o.group_qubits = R;
        o.dense_prec = dprec;
        o.block_qubits = block;
        std::string err;
        std::vector<Plan> plans(B);
        for (int bi = 0; bi < B; ++bi) {
            std::vector<RGate> rg;
            if (resolve_gates(n, gl.data(), gl.size(), NP ? params.data() : nullptr, NP, bi, rg, err) != QS_OK) {
                std::printf("FAIL %d resolve: %s\n", ci, err.c_str());
                return 1;
            }
            const qs_status ps = mode == QS_MODE_PERGATE ? build_pergate_plan(n, rg, plans[bi], err)
                                                         : build_fused_plan(n, 1, rg, o, plans[bi], err, B > 1);
            if (ps != QS_OK) {
                std::printf("FAIL %d plan: %s\n", ci, err.c_str());
                return 1;
            }
        }
        // batched items run as one merged plan when the items' plans agree in structure
        std::vector<Plan> run_plans;
        bool merged = false;
        if (B > 1 && mode != QS_MODE_PERGATE) {
            Plan m;
            std::vector<Plan> copy = plans;
            if (merge_item_plans(copy, m, B)) {
                run_plans.push_back(std::move(m));
                merged = true;
            }
        }
        if (!merged) run_plans = plans;
        const size_t N = (size_t)1 << n;
        const bool structure_only = std::strcmp(in_path, "-") == 0;   // no state: invariants only
        std::vector<C> psi(structure_only ? 0 : N * B);
        if (!structure_only) {
            FILE *fi = std::fopen(in_path, "rb");
            if (!fi || std::fread(psi.data(), sizeof(C), psi.size(), fi) != psi.size()) return 2;
            std::fclose(fi);
        }
        Counts c;
        size_t pi = 0;
        size_t n_passes = mode == QS_MODE_PERGATE ? run_plans[0].pg.size() : run_plans[0].passes.size();
        try {
            for (int bi = 0; bi < B; ++bi) {
                const Plan &plan = merged ? run_plans[0] : run_plans[bi];
                if (plan.items != (merged ? B : 1)) throw Fail{"plan items"};
                if (structure_only) {
                    for (pi = 0; pi < plan.passes.size(); ++pi) {
                        const HostPass &hp = plan.passes[pi];
                        if (hp.type == HostPass::TILE) {
                            TileRun(n, hp, c, merged ? bi : 0, plan.items, merged ? B : 1)
                                .check_only(merged ? bi : 0, pi + 1);
                        } else if (hp.type == HostPass::PERM) {
                            uint64_t used = 0;
                            for (int b = 0; b < n; ++b) used |= 1ull << hp.perm.out_pos[b];
                            if (hp.perm.n != n || used != ((n >= 64) ? ~0ull : (1ull << n) - 1))
                                throw Fail{"perm is not a permutation"};
                            c.perm++;
                        } else {
                            const GatherPass &gp = hp.gather;
                            if (gp.n != n || gp.n_slices < 1 || gp.n_slices > 5 || 8 * gp.n_slices < n)
                                throw Fail{"gather slices"};
                            for (int k = 0; k < gp.n_slices; ++k)
                                for (int v = 0; v < 256; ++v)
                                    if (gp.tab[k][v] >> n) throw Fail{"gather table outside the state"};
                            c.gather++;
                        }
                    }
                    continue;
                }
                C *st = psi.data() + (size_t)bi * N;
                if (plan.mode == QS_MODE_PERGATE) {
                    for (pi = 0; pi < plan.pg.size(); ++pi) run_pergate(n, plan.pg[pi], st);
                    c.pergate += (long)plan.pg.size();
                    continue;
                }
                for (pi = 0; pi < plan.passes.size(); ++pi) {
                    const HostPass &hp = plan.passes[pi];
                    switch (hp.type) {
                        case HostPass::TILE:
                            TileRun(n, hp, c, merged ? bi : 0, plan.items, merged ? B : 1).run(st, merged ? bi : 0);
                            break;
                        case HostPass::PERM:
                            run_perm(n, hp.perm, st);
                            c.perm++;
                            break;
                        case HostPass::GATHER:
                            run_gather(n, hp.gather, st);
                            c.gather++;
                            break;
                    }
                }
            }
        } catch (const Fail &f) {
            std::printf("FAIL %d pass %zu: %s\n", ci, pi, f.why.c_str());
            return 1;
        }
        if (!structure_only) {
            FILE *fo = std::fopen(out_path, "wb");
            if (!fo || std::fwrite(psi.data(), sizeof(C), psi.size(), fo) != psi.size()) return 2;
            std::fclose(fo);
        }
        std::printf("CASE %d passes %zu tile %ld perm %ld gather %ld tma %ld rows %ld swz %ld sweeps %ld merged %d micro",
                    ci, n_passes, c.tile, c.perm, c.gather, c.tma, c.rows, c.swz, c.sweeps, merged ? 1 : 0);
        for (int k = 0; k <= MK_ZYZ; ++k) std::printf(" %ld", c.micro[k]);
        std::printf(" dense %ld %ld %ld pergate %ld\n", c.dense[1], c.dense[2], c.dense[3], c.pergate);
        ++ci;
    }
    return 0;
}
