// Host check of the count-table diagonal (MK_DIAGC) the planner emits.
//
// Circuit: an RY layer, then RZZ(theta) on every edge of a random graph and
// RZ(phi) on a subset of the qubits (one fused diagonal: all RZZ angles equal,
// one single-qubit angle), then another RY layer.  For every sweep holding the
// MK_DIAGC op, for random item bases and every register index, the table entry
// the op selects (counts from its distance classes, neighbour masks, degrees,
// single-bit increments and packed inner-edge counts) must equal
// exp(i phase(x)), with phase(x) evaluated from the gate definitions:
// RZZ(t) = exp(-i t/2 Z Z) and RZ(p) = exp(-i p/2 Z) on the index bit
// n - 1 - q of qubit q, times one positive factor per table (the planner
// folds the pass's normalisation factors into its first count table).
// Prints "OK <checked>" or the first mismatch.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "qs_plan.h"

using namespace qs;

static int run_case(int n, int degree_edges, bool cz, unsigned seed, long long &checked) {
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(-3.0, 3.0);
    // random edge set (distinct pairs)
    std::vector<std::pair<int, int>> edges;
    while ((int)edges.size() < degree_edges) {
        int u = (int)(rng() % n), v = (int)(rng() % n);
        if (u == v) continue;
        if (u > v) std::swap(u, v);
        bool dup = false;
        for (auto &e : edges) dup |= (e.first == u && e.second == v);
        if (!dup) edges.push_back({u, v});
    }
    const double theta = U(rng), phi = U(rng);
    std::vector<int> zq;
    for (int q = 0; q < n; ++q)
        if (rng() % 3 == 0) zq.push_back(q);
    std::vector<qs_gate> g;
    auto add = [&](int kind, int nw, int a, int b, double p) {
        qs_gate x;
        std::memset(&x, 0, sizeof x);
        x.kind = (uint16_t)kind;
        x.nw = (uint8_t)nw;
        x.w[0] = a;
        x.w[1] = b;
        x.p[0] = p;
        x.param_idx = -1;
        g.push_back(x);
    };
    for (int q = 0; q < n; ++q) add(QS_RY, 1, q, 0, U(rng));
    for (auto &e : edges) add(cz ? QS_CP : QS_RZZ, 2, e.first, e.second, theta);
    for (int q : zq) add(QS_RZ, 1, q, 0, phi);
    for (int q = 0; q < n; ++q) add(QS_RY, 1, q, 0, U(rng));
    std::vector<RGate> rg;
    std::string err;
    if (resolve_gates(n, g.data(), g.size(), nullptr, 0, 0, rg, err) != QS_OK) {
        std::printf("resolve: %s\n", err.c_str());
        return 1;
    }
    qs_opts o;
    std::memset(&o, 0, sizeof o);
    Plan P;
    if (build_fused_plan(n, 1, rg, o, P, err) != QS_OK) {
        std::printf("plan: %s\n", err.c_str());
        return 1;
    }
    auto phase = [&](uint64_t x) {   // from the gate definitions, index bit of qubit q = n - 1 - q
        double ph = 0.0;
        for (auto &e : edges) {
            const int bu = (int)((x >> (n - 1 - e.first)) & 1), bv = (int)((x >> (n - 1 - e.second)) & 1);
            if (cz) ph += (bu && bv) ? theta : 0.0;       // CP(t) = diag(1, 1, 1, e^{i t})
            else ph += (bu == bv) ? -theta / 2 : theta / 2;
        }
        for (int q : zq) ph += ((x >> (n - 1 - q)) & 1) ? phi / 2 : -phi / 2;
        return ph;
    };
    int found = 0;
    for (const HostPass &hp : P.passes) {
        if (hp.type != HostPass::TILE) continue;
        const TilePass &tp = hp.tile;
        const float2 *cs = hp.consts.data();
        for (int s = 0; s < tp.n_sweeps; ++s) {
            const Sweep &sw = tp.sweeps[s];
            for (int i = sw.op_begin; i < sw.op_end; ++i) {
                const MicroOp &op = tp.micro[i];
                if (op.kind != MK_DIAGC) continue;
                ++found;
                const int R = sw.r;
                uint64_t gbits[8], gm = 0;
                for (int m = 0; m < R; ++m) {
                    const int tb = sw.gbit[m];
                    gbits[m] = tb < tp.L ? (1ull << tb) : (1ull << tp.hb[tb - tp.L]);
                    gm |= gbits[m];
                }
                std::vector<uint64_t> dat(R + 3 + 2 * op.a);
                std::memcpy(dat.data(), cs + op.lo, dat.size() * 8);
                const uint64_t full = (n == 64) ? ~0ull : ((1ull << n) - 1);
                double scale = -1.0;   // the table's common factor, from its first entry
                for (int trial = 0; trial < 64; ++trial) {
                    const uint64_t x0 = rng() & full & ~gm;
                    int c0 = op.p * __builtin_popcountll(x0 & dat[R + 1]);
                    for (int k = 0; k < op.a; ++k) {
                        const uint64_t msk = dat[R + 3 + 2 * k];
                        const int d = (int)dat[R + 4 + 2 * k];
                        const uint64_t f = op.b ? (x0 & (x0 >> d)) : (x0 ^ (x0 >> d));
                        c0 += __builtin_popcountll(f & msk);
                    }
                    for (int j = 0; j < (1 << R); ++j) {
                        int c = c0;
                        uint64_t x = x0;
                        for (int m = 0; m < R; ++m) {
                            if (!((j >> m) & 1)) continue;
                            x |= gbits[m];
                            const int sm = __builtin_popcountll(x0 & dat[m]);
                            const int dm = op.b ? sm : (int)((dat[R] >> (6 * m)) & 63) - 2 * sm;
                            c += dm + (int)((dat[R + 2] >> (12 * m)) & 4095);
                        }
                        const uint64_t qw = j < 16 ? op.cmask : op.cval;
                        c += (int)((qw >> (4 * (j & 15))) & 15);
                        const float2 t = cs[op.cst + c];
                        if (scale < 0) scale = std::abs(std::complex<double>(t.x, t.y));
                        const std::complex<double> want = std::polar(scale, phase(x));
                        const double err2 = std::abs(std::complex<double>(t.x, t.y) - want);
                        if (!(scale > 0x1p-40 && scale < 0x1p40)) {
                            std::printf("TABLE FACTOR %g out of range\n", scale);
                            return 1;
                        }
                        if (!(err2 < 1e-6)) {
                            std::printf("MISMATCH n=%d cz=%d x=%llx idx=%d got=(%g,%g) want=(%g,%g)\n", n, (int)cz,
                                        (unsigned long long)x, c, t.x, t.y, want.real(), want.imag());
                            return 1;
                        }
                        ++checked;
                    }
                }
            }
        }
    }
    if (!found) {
        std::printf("no count-table diagonal in the plan (n=%d cz=%d)\n", n, (int)cz);
        return 1;
    }
    return 0;
}

int main() {
    long long checked = 0;
    const int ns[] = {6, 9, 13, 16, 20, 24};
    unsigned seed = 1;
    for (int n : ns)
        for (int cz = 0; cz < 2; ++cz)
            for (int rep = 0; rep < 3; ++rep)
                if (run_case(n, std::min(3 * n / 2, n * (n - 1) / 2), cz != 0, seed++, checked)) return 1;
    std::printf("OK %lld\n", checked);
    return 0;
}
