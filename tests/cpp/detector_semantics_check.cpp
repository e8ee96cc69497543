// Host check of the fusion detector's semantics.
//
// Reads gate lists (one circuit per block: "n <n> <count>", then one gate per
// line: kind nw w0 w1 w2 p0 p1 p2 has_dense [8 doubles]), resolves them with
// the planner's own validation, and compares two complex128 evolutions of a
// seeded random state:
//   reference: every gate applied in order as its full 2^nw x 2^nw matrix
//              (wire 0 = the most significant bit of the matrix index);
//   fused:     the detector's ops (1q / 2q unitaries with controls, diagonal
//              quadratic forms, QFT stages, GF(2) affine maps), and the same
//              ops regrouped into dense blocks of 3, 4 and 5 qubits,
//              each op applied by its definition.
// Prints "OK <circuits> kinds <count of each op kind>" or the first mismatch.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "qs_plan.h"

using namespace qs;
using C = std::complex<double>;

static void apply_matrix(std::vector<C> &psi, int n, const std::vector<int> &bits, const C *M) {
    const int k = (int)bits.size(), d = 1 << k;
    uint64_t mask = 0;
    for (int b : bits) mask |= 1ull << b;
    std::vector<C> v(d), w(d);
    for (uint64_t x = 0; x < (1ull << n); ++x) {
        if (x & mask) continue;
        for (int i = 0; i < d; ++i) {
            uint64_t y = x;
            for (int j = 0; j < k; ++j)
                if ((i >> (k - 1 - j)) & 1) y |= 1ull << bits[j];   // bits[0] = MSB of the matrix index
            v[i] = psi[y];
        }
        for (int r = 0; r < d; ++r) {
            C s = 0;
            for (int c = 0; c < d; ++c) s += M[r * d + c] * v[c];
            w[r] = s;
        }
        for (int i = 0; i < d; ++i) {
            uint64_t y = x;
            for (int j = 0; j < k; ++j)
                if ((i >> (k - 1 - j)) & 1) y |= 1ull << bits[j];
            psi[y] = w[i];
        }
    }
}

static void apply_fop(std::vector<C> &psi, int n, const FOp &f) {
    const uint64_t N = 1ull << n;
    switch (f.kind) {
        case F_U1: {
            const uint64_t b = 1ull << f.t0;
            for (uint64_t x = 0; x < N; ++x) {
                if ((x & b) || (x & f.cmask) != f.cval) continue;
                const C a0 = psi[x], a1 = psi[x | b];
                psi[x] = f.m[0] * a0 + f.m[1] * a1;
                psi[x | b] = f.m[2] * a0 + f.m[3] * a1;
            }
            break;
        }
        case F_U2: {
            const uint64_t ba = 1ull << f.t0, bb = 1ull << f.t1;
            for (uint64_t x = 0; x < N; ++x) {
                if ((x & (ba | bb)) || (x & f.cmask) != f.cval) continue;
                const uint64_t id[4] = {x, x | bb, x | ba, x | ba | bb};
                C v[4], w[4];
                for (int i = 0; i < 4; ++i) v[i] = psi[id[i]];
                for (int r = 0; r < 4; ++r) {
                    w[r] = 0;
                    for (int c = 0; c < 4; ++c) w[r] += f.m[r * 4 + c] * v[c];
                }
                for (int i = 0; i < 4; ++i) psi[id[i]] = w[i];
            }
            break;
        }
        case F_DIAG:
            for (uint64_t x = 0; x < N; ++x) {
                double ph = f.diag.g0;
                for (auto &kv : f.diag.a)
                    if ((x >> kv.first) & 1) ph += kv.second;
                for (auto &kv : f.diag.pairs)
                    if (((x >> kv.first.first) & 1) && ((x >> kv.first.second) & 1)) ph += kv.second;
                psi[x] *= std::polar(1.0, ph);
            }
            break;
        case F_QFT: {
            // H on bit p, then exp(i pi (x & bits[lo, p)) / 2^p) where bit p is set
            const uint64_t b = 1ull << f.p;
            const uint64_t mk = (f.p > f.lo) ? (((1ull << f.p) - 1) & ~((1ull << f.lo) - 1)) : 0;
            const double s = std::sqrt(0.5);
            for (uint64_t x = 0; x < N; ++x) {
                if (x & b) continue;
                const C a0 = psi[x], a1 = psi[x | b];
                psi[x] = s * (a0 + a1);
                psi[x | b] = s * (a0 - a1) * std::polar(1.0, M_PI * (double)(x & mk) / std::ldexp(1.0, f.p));
            }
            break;
        }
        case F_GF2: {
            std::vector<C> out(N);
            for (uint64_t x = 0; x < N; ++x) {
                uint64_t y = f.c;
                for (int i = 0; i < n; ++i)
                    if (__builtin_popcountll(f.rows[i] & x) & 1) y ^= 1ull << i;
                out[y] = psi[x];
            }
            psi.swap(out);
            break;
        }
        case F_DENSE: {
            // matrix index bit j = index bit dbits[j] (bit 0 = least significant)
            const int k = (int)f.dbits.size(), d = 1 << k;
            uint64_t mask = 0;
            for (int b : f.dbits) mask |= 1ull << b;
            std::vector<C> v(d), w(d);
            for (uint64_t x = 0; x < N; ++x) {
                if (x & mask) continue;
                for (int i = 0; i < d; ++i) {
                    uint64_t y = x;
                    for (int j = 0; j < k; ++j)
                        if ((i >> j) & 1) y |= 1ull << f.dbits[j];
                    v[i] = psi[y];
                }
                for (int r = 0; r < d; ++r) {
                    w[r] = 0;
                    for (int c = 0; c < d; ++c) w[r] += f.dm[(size_t)r * d + c] * v[c];
                }
                for (int i = 0; i < d; ++i) {
                    uint64_t y = x;
                    for (int j = 0; j < k; ++j)
                        if ((i >> j) & 1) y |= 1ull << f.dbits[j];
                    psi[y] = w[i];
                }
            }
            break;
        }
    }
}

static double maxdiff(const std::vector<C> &a, const std::vector<C> &b) {
    double m = 0;
    for (size_t i = 0; i < a.size(); ++i) m = std::max(m, std::abs(a[i] - b[i]));
    return m;
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *fp = std::fopen(argv[1], "r");
    if (!fp) return 2;
    int n, cnt, circuits = 0;
    long kinds[6] = {0, 0, 0, 0, 0, 0};
    std::mt19937_64 rng(5);
    std::normal_distribution<double> N01;
    while (std::fscanf(fp, " n %d %d", &n, &cnt) == 2) {
        std::vector<qs_gate> gl(cnt);
        std::vector<std::vector<double>> dense(cnt);
        for (int i = 0; i < cnt; ++i) {
            int kind, nw, w0, w1, w2, hd;
            double p0, p1, p2;
            if (std::fscanf(fp, "%d %d %d %d %d %lf %lf %lf %d", &kind, &nw, &w0, &w1, &w2, &p0, &p1, &p2, &hd) != 9)
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
            g.param_idx = -1;
            if (hd) {
                dense[i].resize(8);
                for (int e = 0; e < 8; ++e)
                    if (std::fscanf(fp, "%lf", &dense[i][e]) != 1) return 2;
                g.dense = dense[i].data();
            }
        }
        std::vector<RGate> rg;
        std::string err;
        if (resolve_gates(n, gl.data(), gl.size(), nullptr, 0, 0, rg, err) != QS_OK) {
            std::printf("resolve: %s\n", err.c_str());
            return 1;
        }
        std::vector<C> psi0((size_t)1 << n);
        for (auto &z : psi0) z = C(N01(rng), N01(rng));
        std::vector<C> ref = psi0;
        for (const RGate &g : rg) {
            C M[64];
            gate_matrix(g, M);
            std::vector<int> bits(g.b, g.b + g.nw);
            apply_matrix(ref, n, bits, M);
        }
        std::vector<FOp> ops;
        detect(n, rg, ops);
        std::vector<C> got = psi0;
        for (const FOp &f : ops) {
            apply_fop(got, n, f);
            kinds[f.kind]++;
        }
        double e = maxdiff(got, ref);
        if (!(e < 1e-9)) {
            std::printf("MISMATCH detector n=%d gates=%d ops=%zu maxdiff=%g (circuit %d)\n", n, cnt, ops.size(), e,
                        circuits);
            return 1;
        }
        for (int k = 3; k <= 5 && k <= n; ++k) {
            int cell_of[64];
            for (int b = 0; b < 64; ++b) cell_of[b] = 63;
            dense_cells(n, std::min(n, 13), std::min(4, n), k, cell_of);
            std::vector<FOp> blocks;
            fuse_dense(n, k, cell_of, ops, blocks);
            std::vector<C> gd = psi0;
            for (const FOp &f : blocks) {
                apply_fop(gd, n, f);
                kinds[f.kind]++;
            }
            e = maxdiff(gd, ref);
            if (!(e < 1e-9)) {
                std::printf("MISMATCH dense k=%d n=%d gates=%d maxdiff=%g (circuit %d)\n", k, n, cnt, e, circuits);
                return 1;
            }
        }
        ++circuits;
    }
    std::printf("OK %d kinds %ld %ld %ld %ld %ld %ld\n", circuits, kinds[0], kinds[1], kinds[2], kinds[3], kinds[4],
                kinds[5]);
    return 0;
}
