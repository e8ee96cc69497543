// Host-side planner: validation, FP64 gate matrices, the fusion detector and
// the HBM-pass scheduler (see qs_plan.h).
#include "qs_plan.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <set>
#include <sstream>

namespace qs {

static const double kPi = 3.14159265358979323846;
static const double kSqrtHalf = 0.70710678118654752440;

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

// ---------------------------------------------------------------------------
// gate library (Sec. 3.2.2; OpenQASM table of Sec. 3.3; Sec. 5.1 terms)
// ---------------------------------------------------------------------------
static int kind_arity(int k) {
    switch (k) {
        case QS_I: case QS_X: case QS_Y: case QS_Z: case QS_H: case QS_S: case QS_SDG:
        case QS_T: case QS_TDG: case QS_SX: case QS_RX: case QS_RY: case QS_RZ: case QS_P:
        case QS_U2: case QS_U3: case QS_U:
            return 1;
        case QS_CX: case QS_CY: case QS_CZ: case QS_CH: case QS_SWAP: case QS_ISWAP:
        case QS_CRX: case QS_CRY: case QS_CRZ: case QS_CP: case QS_RZZ: case QS_RXX: case QS_RYY:
            return 2;
        case QS_CCX: case QS_CSWAP:
            return 3;
        default:
            return -1;
    }
}

bool gate_is_diagonal(int k) {
    switch (k) {
        case QS_I: case QS_Z: case QS_S: case QS_SDG: case QS_T: case QS_TDG: case QS_RZ: case QS_P:
        case QS_CZ: case QS_CRZ: case QS_CP: case QS_RZZ: case K_DIAG2:
            return true;
        default:
            return false;
    }
}

static bool kind_takes_param(int k) {
    switch (k) {
        case QS_RX: case QS_RY: case QS_RZ: case QS_P: case QS_U2: case QS_U3: case QS_CRX:
        case QS_CRY: case QS_CRZ: case QS_CP: case QS_RZZ: case QS_RXX: case QS_RYY:
            return true;
        default:
            return false;
    }
}

qs_status resolve_gates(int n, const qs_gate *gates, size_t n_gates, const double *params,
                        int n_params, int bi, std::vector<RGate> &out, std::string &err) {
    out.clear();
    out.reserve(n_gates);
    if (n_gates && !gates) {
        err = "gates == NULL with n_gates > 0";
        return QS_ERR_INVALID_ARG;
    }
    for (size_t i = 0; i < n_gates; ++i) {
        const qs_gate &g = gates[i];
        int ar = kind_arity(g.kind);
        char buf[160];
        if (ar < 0) {
            snprintf(buf, sizeof buf, "gate %zu: unknown kind %d", i, (int)g.kind);
            err = buf;
            return QS_ERR_INVALID_ARG;
        }
        if ((int)g.nw != ar) {
            snprintf(buf, sizeof buf, "gate %zu: kind %d takes %d wires, got %d", i, (int)g.kind, ar, (int)g.nw);
            err = buf;
            return QS_ERR_INVALID_ARG;
        }
        RGate r;
        r.kind = g.kind;
        r.nw = ar;
        for (int m = 0; m < ar; ++m) {
            if (g.w[m] < 0 || g.w[m] >= n) {
                snprintf(buf, sizeof buf, "gate %zu: wire %d out of range [0,%d)", i, g.w[m], n);
                err = buf;
                return QS_ERR_INVALID_ARG;
            }
            for (int j = 0; j < m; ++j)
                if (g.w[j] == g.w[m]) {
                    snprintf(buf, sizeof buf, "gate %zu: duplicate wire %d", i, g.w[m]);
                    err = buf;
                    return QS_ERR_INVALID_ARG;
                }
            r.q[m] = g.w[m];
            r.b[m] = n - 1 - g.w[m];
        }
        for (int m = 0; m < 3; ++m) r.p[m] = g.p[m];
        if (g.param_idx >= 0) {
            if (!kind_takes_param(g.kind)) {
                snprintf(buf, sizeof buf, "gate %zu: kind %d has no angle to parameterise", i, (int)g.kind);
                err = buf;
                return QS_ERR_INVALID_ARG;
            }
            if (!params || g.param_idx >= n_params) {
                snprintf(buf, sizeof buf, "gate %zu: param_idx %d outside params[%d]", i, g.param_idx, n_params);
                err = buf;
                return QS_ERR_INVALID_ARG;
            }
            r.p[0] = params[(size_t)bi * n_params + g.param_idx];
        } else if (g.param_idx < -1) {
            snprintf(buf, sizeof buf, "gate %zu: param_idx %d < -1", i, g.param_idx);
            err = buf;
            return QS_ERR_INVALID_ARG;
        }
        if (g.kind == QS_U) {
            if (!g.dense) {
                snprintf(buf, sizeof buf, "gate %zu: QS_U needs a dense matrix", i);
                err = buf;
                return QS_ERR_INVALID_ARG;
            }
            for (int e = 0; e < 4; ++e) {
                if (!std::isfinite(g.dense[2 * e]) || !std::isfinite(g.dense[2 * e + 1])) {
                    snprintf(buf, sizeof buf, "gate %zu: non-finite matrix entry", i);
                    err = buf;
                    return QS_ERR_INVALID_ARG;
                }
                r.dense[e] = cd(g.dense[2 * e], g.dense[2 * e + 1]);
            }
        }
        for (int m = 0; m < 3; ++m)
            if (!std::isfinite(r.p[m])) {
                snprintf(buf, sizeof buf, "gate %zu: non-finite angle", i);
                err = buf;
                return QS_ERR_INVALID_ARG;
            }
        out.push_back(r);
    }
    return QS_OK;
}

// 2x2 unitary of a one-qubit kind.
static void mat1(int k, const double *p, const cd *dense, cd M[4]) {
    const cd I(0, 1);
    auto set = [&](cd a, cd b, cd c, cd d) { M[0] = a; M[1] = b; M[2] = c; M[3] = d; };
    double c, s;
    switch (k) {
        case QS_I: set(1, 0, 0, 1); break;
        case QS_X: set(0, 1, 1, 0); break;
        case QS_Y: set(0, -I, I, 0); break;
        case QS_Z: set(1, 0, 0, -1); break;
        case QS_H: set(kSqrtHalf, kSqrtHalf, kSqrtHalf, -kSqrtHalf); break;
        case QS_S: set(1, 0, 0, I); break;
        case QS_SDG: set(1, 0, 0, -I); break;
        case QS_T: set(1, 0, 0, std::polar(1.0, kPi / 4)); break;
        case QS_TDG: set(1, 0, 0, std::polar(1.0, -kPi / 4)); break;
        case QS_SX: set(cd(0.5, 0.5), cd(0.5, -0.5), cd(0.5, -0.5), cd(0.5, 0.5)); break;
        case QS_RX: c = cos(p[0] / 2); s = sin(p[0] / 2); set(c, -I * s, -I * s, c); break;
        case QS_RY: c = cos(p[0] / 2); s = sin(p[0] / 2); set(c, -s, s, c); break;
        case QS_RZ: set(std::polar(1.0, -p[0] / 2), 0, 0, std::polar(1.0, p[0] / 2)); break;
        case QS_P: set(1, 0, 0, std::polar(1.0, p[0])); break;
        case QS_U2: case QS_U3: {
            double th = (k == QS_U2) ? kPi / 2 : p[0];
            double ph = (k == QS_U2) ? p[0] : p[1];
            double la = (k == QS_U2) ? p[1] : p[2];
            c = cos(th / 2);
            s = sin(th / 2);
            set(c, -std::polar(1.0, la) * s, std::polar(1.0, ph) * s, std::polar(1.0, ph + la) * c);
            break;
        }
        case QS_U: for (int e = 0; e < 4; ++e) M[e] = dense[e]; break;
        default: set(1, 0, 0, 1);
    }
}

void gate_matrix(const RGate &g, cd *M) {
    if (g.nw == 1) {
        mat1(g.kind, g.p, g.dense, M);
        return;
    }
    const int K = 1 << g.nw;
    for (int i = 0; i < K * K; ++i) M[i] = 0;
    for (int i = 0; i < K; ++i) M[i * K + i] = 1;
    if (g.kind == K_DIAG2) {
        for (int i = 0; i < 4; ++i) M[i * 4 + i] = std::polar(1.0, g.dense[i].real());
        return;
    }
    const cd I(0, 1);
    auto ctrl1 = [&](int kind1, double ang) {   // controlled 2x2 in the lower-right block
        cd U[4];
        double pp[3] = {ang, 0, 0};
        mat1(kind1, pp, nullptr, U);
        M[2 * 4 + 2] = U[0]; M[2 * 4 + 3] = U[1]; M[3 * 4 + 2] = U[2]; M[3 * 4 + 3] = U[3];
    };
    double c, s;
    switch (g.kind) {
        case QS_CX: ctrl1(QS_X, 0); break;
        case QS_CY: ctrl1(QS_Y, 0); break;
        case QS_CZ: ctrl1(QS_Z, 0); break;
        case QS_CH: ctrl1(QS_H, 0); break;
        case QS_CRX: ctrl1(QS_RX, g.p[0]); break;
        case QS_CRY: ctrl1(QS_RY, g.p[0]); break;
        case QS_CRZ: ctrl1(QS_RZ, g.p[0]); break;
        case QS_CP: M[15] = std::polar(1.0, g.p[0]); break;
        case QS_SWAP: M[5] = 0; M[10] = 0; M[6] = 1; M[9] = 1; break;
        case QS_ISWAP: M[5] = 0; M[10] = 0; M[6] = I; M[9] = I; break;
        case QS_RZZ:
            M[0] = M[15] = std::polar(1.0, -g.p[0] / 2);
            M[5] = M[10] = std::polar(1.0, g.p[0] / 2);
            break;
        case QS_RXX: case QS_RYY: {
            c = cos(g.p[0] / 2);
            s = sin(g.p[0] / 2);
            // exp(-i t/2 P(x)P) = c I - i s P(x)P; XX flips both bits (+1),
            // YY = -XX on |00>,|11> and +XX on |01>,|10>
            double sg03 = (g.kind == QS_RXX) ? 1.0 : -1.0;
            for (int i = 0; i < 4; ++i) M[i * 4 + i] = c;
            M[0 * 4 + 3] = M[3 * 4 + 0] = -I * s * sg03;
            M[1 * 4 + 2] = M[2 * 4 + 1] = -I * s;
            break;
        }
        case QS_CCX:
            M[6 * 8 + 6] = 0; M[7 * 8 + 7] = 0; M[6 * 8 + 7] = 1; M[7 * 8 + 6] = 1;
            break;
        case QS_CSWAP:
            M[5 * 8 + 5] = 0; M[6 * 8 + 6] = 0; M[5 * 8 + 6] = 1; M[6 * 8 + 5] = 1;
            break;
        default: break;
    }
}

// phases of diagonal kinds (radians): 1q -> ph[0..1]; 2q -> ph[0..3], index x_w0*2 + x_w1
static void diag_phases(const RGate &g, double *ph) {
    const double t = g.p[0];
    switch (g.kind) {
        case QS_I: ph[0] = 0; ph[1] = 0; break;
        case QS_Z: ph[0] = 0; ph[1] = kPi; break;
        case QS_S: ph[0] = 0; ph[1] = kPi / 2; break;
        case QS_SDG: ph[0] = 0; ph[1] = -kPi / 2; break;
        case QS_T: ph[0] = 0; ph[1] = kPi / 4; break;
        case QS_TDG: ph[0] = 0; ph[1] = -kPi / 4; break;
        case QS_RZ: ph[0] = -t / 2; ph[1] = t / 2; break;
        case QS_P: ph[0] = 0; ph[1] = t; break;
        case QS_CZ: ph[0] = ph[1] = ph[2] = 0; ph[3] = kPi; break;
        case QS_CP: ph[0] = ph[1] = ph[2] = 0; ph[3] = t; break;
        case QS_CRZ: ph[0] = ph[1] = 0; ph[2] = -t / 2; ph[3] = t / 2; break;
        case QS_RZZ: ph[0] = ph[3] = -t / 2; ph[1] = ph[2] = t / 2; break;
        case K_DIAG2:
            for (int k = 0; k < 4; ++k) ph[k] = g.dense[k].real();
            break;
        default: ph[0] = ph[1] = ph[2] = ph[3] = 0;
    }
}

// ---------------------------------------------------------------------------
// Diag
// ---------------------------------------------------------------------------
uint64_t Diag::support() const {
    uint64_t s = 0;
    for (auto &kv : a) s |= 1ull << kv.first;
    for (auto &kv : pairs) s |= (1ull << kv.first.first) | (1ull << kv.first.second);
    return s;
}
void Diag::add1(int b, double ph0, double ph1) {
    g0 += ph0;
    if (ph1 - ph0 != 0.0) a[b] += ph1 - ph0;
}
void Diag::add2(int b0, int b1, const double ph[4]) {
    g0 += ph[0];
    if (ph[2] - ph[0] != 0.0) a[b0] += ph[2] - ph[0];
    if (ph[1] - ph[0] != 0.0) a[b1] += ph[1] - ph[0];
    double gam = ph[3] - ph[2] - ph[1] + ph[0];
    if (gam != 0.0) pairs[{std::min(b0, b1), std::max(b0, b1)}] += gam;
}
void Diag::merge(const Diag &o) {
    g0 += o.g0;
    for (auto &kv : o.a) a[kv.first] += kv.second;
    for (auto &kv : o.pairs) pairs[kv.first] += kv.second;
}

uint64_t FOp::N() const {
    switch (kind) {
        case F_U1: return 1ull << t0;
        case F_U2: return (1ull << t0) | (1ull << t1);
        case F_DIAG: return 0;
        case F_QFT: return 1ull << p;
        case F_GF2: return ~0ull;
        case F_DENSE: {
            uint64_t m = 0;
            for (int b : dbits) m |= 1ull << b;
            return m;
        }
    }
    return ~0ull;
}
uint64_t FOp::D() const {
    switch (kind) {
        case F_U1: case F_U2: return cmask;
        case F_DIAG: return diag.support();
        case F_QFT: return (p > lo) ? (((1ull << p) - 1) & ~((1ull << lo) - 1)) : 0;
        case F_GF2: return ~0ull;
        case F_DENSE: return 0;
    }
    return ~0ull;
}

static bool commute(const FOp &x, const FOp &y) {
    if (x.kind == F_GF2 || y.kind == F_GF2) return false;
    const uint64_t nx = x.cN, ny = y.cN;
    return (nx & (ny | y.cD)) == 0 && (ny & (nx | x.cD)) == 0;
}

// ---------------------------------------------------------------------------
// detector (Sec. 5.2): per-wire 1q window collapse with symbolic cancellation
// of involution pairs, commuting diagonal runs, QFT stages, GF(2) runs
// ---------------------------------------------------------------------------
namespace {
struct Window {
    std::vector<std::array<cd, 4>> mats;
    std::vector<int> kinds;
    int n_gates = 0;
};

bool is_involution_kind(int k) { return k == QS_H || k == QS_X || k == QS_Y || k == QS_Z; }

void mat2x2_mul(const cd A[4], const cd B[4], cd C[4]) {   // C = A B
    cd c0 = A[0] * B[0] + A[1] * B[2], c1 = A[0] * B[1] + A[1] * B[3];
    cd c2 = A[2] * B[0] + A[3] * B[2], c3 = A[2] * B[1] + A[3] * B[3];
    C[0] = c0; C[1] = c1; C[2] = c2; C[3] = c3;
}

struct Detector {
    int n;
    std::vector<FOp> &ops;
    Diag D;
    int D_gates = 0;
    std::vector<Window> pend;
    Detector(int n_, std::vector<FOp> &o) : n(n_), ops(o), pend(n_) {}

    void emit_diag() {
        if (!D.empty() || D_gates) {
            if (!D.empty()) {
                FOp f;
                f.kind = F_DIAG;
                f.diag = D;
                f.n_gates = D_gates;
                ops.push_back(f);
            }
            D = Diag();
            D_gates = 0;
        }
    }
    // Emit the open diagonal, then every pending window (non-diagonal
    // products as U1 ops; exactly diagonal products seed the next diagonal).
    void flush_all() {
        emit_diag();
        Diag nd;
        int nd_gates = 0;
        for (int q = 0; q < n; ++q) {
            Window &w = pend[q];
            if (w.mats.empty()) {
                w.n_gates = 0;
                continue;
            }
            cd P[4] = {1, 0, 0, 1};
            for (auto &m : w.mats) mat2x2_mul(m.data(), P, P);
            int b = n - 1 - q;
            bool ident = P[0] == cd(1, 0) && P[1] == cd(0, 0) && P[2] == cd(0, 0) && P[3] == cd(1, 0);
            bool diag = P[1] == cd(0, 0) && P[2] == cd(0, 0);
            if (ident) {
                // exact identity (rtol = 0): nothing to apply
            } else if (diag) {
                nd.g0 += std::arg(P[0]);
                nd.a[b] += std::arg(P[3]) - std::arg(P[0]);
                nd_gates += w.n_gates;
            } else {
                FOp f;
                f.kind = F_U1;
                f.t0 = b;
                for (int e = 0; e < 4; ++e) f.m[e] = P[e];
                f.n_gates = w.n_gates;
                ops.push_back(f);
            }
            w.mats.clear();
            w.kinds.clear();
            w.n_gates = 0;
        }
        D = nd;
        D_gates = nd_gates;
        if (D.empty() && nd_gates) {   // diagonal windows that multiplied out to phase 0
            D_gates = 0;
        }
    }
    bool any_pending(const RGate &g) const {
        for (int m = 0; m < g.nw; ++m)
            if (!pend[g.q[m]].mats.empty()) return true;
        return false;
    }
    void gate(const RGate &g) {
        if (g.nw == 1) {
            Window &w = pend[g.q[0]];
            if (gate_is_diagonal(g.kind) && w.mats.empty()) {
                double ph[2];
                diag_phases(g, ph);
                D.add1(g.b[0], ph[0], ph[1]);
                D_gates++;
                return;
            }
            if (g.kind == QS_I && w.mats.empty()) return;
            // symbolic cancellation of an involution pair (H H, X X, Y Y, Z Z)
            if (is_involution_kind(g.kind) && !w.kinds.empty() && w.kinds.back() == g.kind) {
                w.kinds.pop_back();
                w.mats.pop_back();
                w.n_gates++;
                return;
            }
            std::array<cd, 4> M;
            mat1(g.kind, g.p, g.dense, M.data());
            w.mats.push_back(M);
            w.kinds.push_back(g.kind);
            w.n_gates++;
            return;
        }
        if (gate_is_diagonal(g.kind)) {
            if (any_pending(g)) flush_all();
            double ph[4];
            diag_phases(g, ph);
            D.add2(g.b[0], g.b[1], ph);
            D_gates++;
            return;
        }
        flush_all();
        emit_diag();
        FOp f;
        f.n_gates = 1;
        cd M[64];
        gate_matrix(g, M);
        switch (g.kind) {
            case QS_CX: case QS_CY: case QS_CH: case QS_CRX: case QS_CRY:
                f.kind = F_U1;
                f.t0 = g.b[1];
                f.cmask = f.cval = 1ull << g.b[0];
                f.m[0] = M[10]; f.m[1] = M[11]; f.m[2] = M[14]; f.m[3] = M[15];
                break;
            case QS_CCX:
                f.kind = F_U1;
                f.t0 = g.b[2];
                f.cmask = f.cval = (1ull << g.b[0]) | (1ull << g.b[1]);
                f.m[0] = 0; f.m[1] = 1; f.m[2] = 1; f.m[3] = 0;
                break;
            case QS_CSWAP:
                f.kind = F_U2;
                f.t0 = g.b[1];
                f.t1 = g.b[2];
                f.cmask = f.cval = 1ull << g.b[0];
                for (int e = 0; e < 16; ++e) f.m[e] = 0;
                f.m[0] = f.m[15] = 1;
                f.m[1 * 4 + 2] = f.m[2 * 4 + 1] = 1;
                break;
            default:   // SWAP, ISWAP, RXX, RYY: 4x4 on (w0 = MSB, w1)
                f.kind = F_U2;
                f.t0 = g.b[0];
                f.t1 = g.b[1];
                for (int e = 0; e < 16; ++e) f.m[e] = M[e];
        }
        ops.push_back(f);
    }
    void finish() {
        flush_all();
        emit_diag();
    }
};

bool is_exact_h(const FOp &f) {
    return f.kind == F_U1 && f.cmask == 0 && f.m[0] == cd(kSqrtHalf, 0) && f.m[1] == cd(kSqrtHalf, 0) &&
           f.m[2] == cd(kSqrtHalf, 0) && f.m[3] == cd(-kSqrtHalf, 0);
}
bool is_exact_x(const FOp &f) {
    return f.kind == F_U1 && f.m[0] == cd(0, 0) && f.m[1] == cd(1, 0) && f.m[2] == cd(1, 0) &&
           f.m[3] == cd(0, 0);
}
bool is_exact_swap(const FOp &f) {
    if (f.kind != F_U2 || f.cmask) return false;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            int want = ((i == 0 && j == 0) || (i == 3 && j == 3) || (i == 1 && j == 2) || (i == 2 && j == 1));
            if (f.m[i * 4 + j] != cd(want, 0)) return false;
        }
    return true;
}
// X, CNOT (one control) or SWAP: affine over GF(2)
bool is_gf2(const FOp &f) {
    if (is_exact_x(f) && popc64(f.cmask) <= 1 && f.cmask == f.cval) return true;
    return is_exact_swap(f);
}

// QFT stage: an exact H on bit p followed by a diagonal that is exactly the
// stage's controlled-phase ladder sum_{b in [lo,p)} x_b x_p pi / 2^(p-b).
bool match_ladder(const Diag &d, int p, int &lo) {
    if (d.g0 != 0.0 || d.pairs.empty()) return false;
    for (auto &kv : d.a)
        if (kv.second != 0.0) return false;
    int cnt = 0;
    int mn = p;
    for (auto &kv : d.pairs) {
        int b = kv.first.first, c = kv.first.second;
        if (c != p || b >= p) return false;
        if (kv.second != std::ldexp(kPi, -(p - b))) return false;
        mn = std::min(mn, b);
        cnt++;
    }
    if (cnt != p - mn) return false;   // contiguous bits [mn, p)
    lo = mn;
    return true;
}
}  // namespace

// RX-type 1q ops between two diagonal runs: U = [[c, i s], [i s, c]] equals
// S M S^dagger with S = diag(1, i) and the real M = [[c, -s], [s, c]] (a basis
// conjugation, as for the XX / YY layers of Sec. 5.1).  S^dagger commutes with
// the 1q ops on other bits back to the previous diagonal and S forward to the
// next one, so both fold into diagonals that run anyway; in a Trotter stream
// the S of one step and the S^dagger of the next cancel exactly (the phase
// adjustments are counted in units of pi/2).  The real M runs on the packed
// FP32x2 pipe at half the instructions of the complex form.
static void conjugate_rx_runs(std::vector<FOp> &ops) {
    std::vector<std::map<int, int>> adj(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        if (ops[i].kind != F_DIAG) continue;
        size_t j = i + 1;
        uint64_t seen = 0;
        bool distinct = true;
        while (j < ops.size() && ops[j].kind == F_U1 && ops[j].cmask == 0) {
            if ((seen >> ops[j].t0) & 1) distinct = false;
            seen |= 1ull << ops[j].t0;
            ++j;
        }
        if (j >= ops.size() || ops[j].kind != F_DIAG || j == i + 1 || !distinct) continue;
        for (size_t k = i + 1; k < j; ++k) {
            FOp &f = ops[k];
            const cd *m = f.m;
            const bool rxc = m[0].imag() == 0 && m[0] == m[3] && m[1].real() == 0 && m[1] == m[2] && m[1].imag() != 0;
            if (!rxc) continue;
            const double c = m[0].real(), sv = m[1].imag();
            f.m[0] = cd(c, 0);
            f.m[1] = cd(-sv, 0);
            f.m[2] = cd(sv, 0);
            f.m[3] = cd(c, 0);
            adj[i][f.t0] -= 1;   // S^dagger, applied before M
            adj[j][f.t0] += 1;   // S, applied after M
        }
        i = j - 1;
    }
    for (size_t i = 0; i < ops.size(); ++i)
        for (auto &kv : adj[i]) {
            const int q = ((kv.second % 4) + 4) % 4;   // multiples of pi/2, mod 2 pi
            if (q) ops[i].diag.a[kv.first] += q * (kPi / 2);
        }
}

// Basis-conjugated Pauli-pair layers (Sec. 5.1): a run of >= 2 consecutive
// RXX gates commutes term by term, so it equals H^{(x)S} exp(-i sum t/2 Z Z)
// H^{(x)S} over the run's qubits S; a run of RYY gates the same with V = S H
// (V Z V^dagger = Y): S^dagger then H before the ZZ phases, H then S after.
// The ZZ phases then form one diagonal run and the outer 1q gates merge with
// their neighbours (H H pairs between consecutive layers cancel symbolically).
static void conjugate_pauli_pair_runs(int n, const std::vector<RGate> &in, std::vector<RGate> &out) {
    out.clear();
    auto one = [&](int kind, int q) {
        RGate g;
        g.kind = kind;
        g.nw = 1;
        g.q[0] = q;
        g.b[0] = n - 1 - q;
        return g;
    };
    for (size_t i = 0; i < in.size();) {
        const int k = in[i].kind;
        size_t j = i;
        if (k == QS_RXX || k == QS_RYY)
            while (j < in.size() && in[j].kind == k) ++j;
        if (j - i < 2) {
            out.push_back(in[i]);
            ++i;
            continue;
        }
        std::vector<int> qs;
        for (size_t t = i; t < j; ++t)
            for (int w = 0; w < 2; ++w)
                if (std::find(qs.begin(), qs.end(), in[t].q[w]) == qs.end()) qs.push_back(in[t].q[w]);
        for (int q : qs) {
            if (k == QS_RYY) out.push_back(one(QS_SDG, q));
            out.push_back(one(QS_H, q));
        }
        for (size_t t = i; t < j; ++t) {
            RGate z = in[t];
            z.kind = QS_RZZ;
            out.push_back(z);
        }
        for (int q : qs) {
            out.push_back(one(QS_H, q));
            if (k == QS_RYY) out.push_back(one(QS_S, q));
        }
        i = j;
    }
}

// Decomposed two-qubit diagonals (App. B.1: imported circuits spell CPHASE
// and ZZ terms out as CX . diagonal . CX, which hides them from the layer
// detectors).  A sandwich CX(c,t) . M . CX(c,t), where every gate of M
// either misses c and t or is diagonal on wires within {c, t}, equals M with
// each of those diagonals conjugated, phi'(xc, xt) = phi(xc, xc ^ xt) (CX
// maps xt to xc ^ xt and is its own inverse), and both CX removed.  The
// conjugated diagonals, and the runs of unconjugated diagonal gates on
// {c, t} right before and right after the sandwich, multiply into one
// two-qubit diagonal gate at the second CX's place (only adjacent runs, so
// that a gate stream spelling one CPHASE per sandwich gives one CPHASE each).  So u1 / cx / u1 / cx
// / u1 spelling CPHASE(l) becomes diag(1, 1, 1, e^{il}) exactly (the +-l/2
// terms cancel exactly in FP64), and cx / rz / cx becomes RZZ.  Circuits
// without such a sandwich pass through unchanged.
static void fold_cx_sandwiches(int n, const std::vector<RGate> &in, std::vector<RGate> &out) {
    constexpr size_t kReach = 64;   // gates scanned on each side: linear time
    std::vector<RGate> g(in);
    std::vector<char> dead(g.size(), 0);
    auto touches = [](const RGate &x, int c, int t) {
        for (int m = 0; m < x.nw; ++m)
            if (x.b[m] == c || x.b[m] == t) return true;
        return false;
    };
    auto diag_within = [](const RGate &x, int c, int t) {
        if (!gate_is_diagonal(x.kind)) return false;
        for (int m = 0; m < x.nw; ++m)
            if (x.b[m] != c && x.b[m] != t) return false;
        return true;
    };
    // phases of a diagonal gate within {c, t} as a function of (xc, xt), index xc * 2 + xt
    auto phases = [](const RGate &x, int c, double ph[4]) {
        double p[4];
        diag_phases(x, p);
        for (int s = 0; s < 4; ++s) {
            const int xc = s >> 1, xt = s & 1;
            if (x.nw == 1) {
                ph[s] = p[x.b[0] == c ? xc : xt];
            } else {
                const int v0 = x.b[0] == c ? xc : xt, v1 = x.b[1] == c ? xc : xt;
                ph[s] = p[v0 * 2 + v1];
            }
        }
    };
    bool any = false;
    for (size_t i = 0; i < g.size(); ++i) {
        if (dead[i] || g[i].kind != QS_CX) continue;
        const int c = g[i].b[0], t = g[i].b[1];
        size_t j = i + 1, seen = 0;
        bool found = false;
        for (; j < g.size() && seen < kReach; ++j) {
            if (dead[j]) continue;
            ++seen;
            const RGate &x = g[j];
            if (!touches(x, c, t)) continue;
            if (x.kind == QS_CX && x.b[0] == c && x.b[1] == t) {
                found = true;
                break;
            }
            if (diag_within(x, c, t)) continue;
            break;
        }
        if (!found) continue;
        double ph[4] = {0, 0, 0, 0}, p[4];
        seen = 0;
        for (size_t k = i; k-- > 0 && seen < kReach;) {   // just before the sandwich
            if (dead[k]) continue;
            ++seen;
            if (!diag_within(g[k], c, t)) break;
            phases(g[k], c, p);
            for (int s = 0; s < 4; ++s) ph[s] += p[s];
            dead[k] = 1;
        }
        for (size_t k = i + 1; k < j; ++k) {   // inside: conjugated by the CX
            if (dead[k] || !touches(g[k], c, t)) continue;
            phases(g[k], c, p);
            for (int s = 0; s < 4; ++s) ph[s] += p[(s & 2) | ((s >> 1) ^ (s & 1))];
            dead[k] = 1;
        }
        seen = 0;
        for (size_t k = j + 1; k < g.size() && seen < kReach; ++k) {   // just after the sandwich
            if (dead[k]) continue;
            ++seen;
            if (!diag_within(g[k], c, t)) break;
            phases(g[k], c, p);
            for (int s = 0; s < 4; ++s) ph[s] += p[s];
            dead[k] = 1;
        }
        RGate d;
        d.kind = K_DIAG2;
        d.nw = 2;
        d.b[0] = c;
        d.b[1] = t;
        d.q[0] = n - 1 - c;
        d.q[1] = n - 1 - t;
        for (int s = 0; s < 4; ++s) d.dense[s] = cd(ph[s], 0.0);
        dead[i] = 1;
        g[j] = d;
        any = true;
    }
    if (!any) {
        out = in;
        return;
    }
    out.clear();
    for (size_t k = 0; k < g.size(); ++k)
        if (!dead[k]) out.push_back(g[k]);
}

void detect(int n, const std::vector<RGate> &gates, std::vector<FOp> &ops) {
    std::vector<RGate> folded, conj;
    fold_cx_sandwiches(n, gates, folded);
    conjugate_pauli_pair_runs(n, folded, conj);
    std::vector<FOp> raw;
    Detector det(n, raw);
    for (const RGate &g : conj) det.gate(g);
    det.finish();

    // QFT stages
    std::vector<FOp> s1;
    for (size_t i = 0; i < raw.size(); ++i) {
        if (is_exact_h(raw[i]) && i + 1 < raw.size() && raw[i + 1].kind == F_DIAG) {
            int lo;
            if (match_ladder(raw[i + 1].diag, raw[i].t0, lo)) {
                FOp f;
                f.kind = F_QFT;
                f.p = raw[i].t0;
                f.lo = lo;
                f.n_gates = raw[i].n_gates + raw[i + 1].n_gates;
                s1.push_back(f);
                ++i;
                continue;
            }
        }
        s1.push_back(raw[i]);
    }
    // GF(2) runs of length >= 2
    ops.clear();
    for (size_t i = 0; i < s1.size();) {
        size_t j = i;
        while (j < s1.size() && is_gf2(s1[j])) ++j;
        if (j - i < 2) {
            ops.push_back(s1[i]);
            ++i;
            continue;
        }
        {
            FOp f;
            f.kind = F_GF2;
            f.rows.resize(n);
            for (int b = 0; b < n; ++b) f.rows[b] = 1ull << b;
            f.c = 0;
            f.n_gates = 0;
            for (size_t k = i; k < j; ++k) {
                const FOp &g = s1[k];
                f.n_gates += g.n_gates;
                if (g.kind == F_U1 && g.cmask == 0) {
                    f.c ^= 1ull << g.t0;
                } else if (g.kind == F_U1) {
                    int cb = __builtin_ctzll(g.cmask);
                    f.rows[g.t0] ^= f.rows[cb];
                    if ((f.c >> cb) & 1) f.c ^= 1ull << g.t0;
                } else {
                    std::swap(f.rows[g.t0], f.rows[g.t1]);
                    uint64_t ba = (f.c >> g.t0) & 1, bb = (f.c >> g.t1) & 1;
                    if (ba != bb) f.c ^= (1ull << g.t0) | (1ull << g.t1);
                }
            }
            ops.push_back(f);
            i = j;
        }
    }
    conjugate_rx_runs(ops);
}

// ---------------------------------------------------------------------------
// dense blocks: greedy, order-preserving regrouping of the detector's output
// into blocks of at most k index bits (generic matrix fusion).
//
// The output is a sequence of items: blocks and ops passed through.  A block
// is "open" while no later item touches its bits; an open block can therefore
// move to the end of the sequence, so merging open blocks with each other and
// with the next op is exact.  A 1q/2q op joins the open blocks on its bits
// (and, while there is room, the most recent open block, which packs a layer
// of 1q ops into blocks of k neighbouring bits).  A diagonal splits: terms
// whose bits lie in one open block fold into it, the rest (global phase,
// bonds across blocks) passes through and closes the blocks it touches.
// Everything else passes through and closes the blocks on its bits.
// ---------------------------------------------------------------------------
namespace {

struct DBlock {
    std::vector<int> bits;   // local bit j <-> index bit bits[j]
    std::vector<cd> m;       // 2^k x 2^k row-major
    int slot = -1;           // position in the item sequence
    bool open = true;
    int n_gates = 0;
};

uint64_t dblock_glob(const std::vector<int> &bits, int i) {
    uint64_t g = 0;
    for (size_t j = 0; j < bits.size(); ++j)
        if ((i >> j) & 1) g |= 1ull << bits[j];
    return g;
}

int dblock_local(const std::vector<int> &bits, int b) {
    for (size_t j = 0; j < bits.size(); ++j)
        if (bits[j] == b) return (int)j;
    return -1;
}

// M <- I (x) M : append index bits as the new most significant local bits
void dblock_grow(DBlock &b, const std::vector<int> &extra) {
    if (extra.empty()) return;
    const int k0 = (int)b.bits.size(), d0 = 1 << k0;
    const int k1 = k0 + (int)extra.size(), d1 = 1 << k1;
    std::vector<cd> m(d1 * d1, cd(0, 0));
    for (int i = 0; i < d1; ++i)
        for (int j = 0; j < d1; ++j)
            if ((i >> k0) == (j >> k0)) m[i * d1 + j] = b.m[(i & (d0 - 1)) * d0 + (j & (d0 - 1))];
    b.m.swap(m);
    b.bits.insert(b.bits.end(), extra.begin(), extra.end());
}

// M <- F M for a 1q / 2q op on bits inside the block
void dblock_apply(DBlock &b, const FOp &f) {
    const int k = (int)b.bits.size(), d = 1 << k;
    if (f.kind == F_U1) {
        const int ja = dblock_local(b.bits, f.t0);
        for (int i = 0; i < d; ++i) {
            if ((i >> ja) & 1) continue;
            if ((dblock_glob(b.bits, i) & f.cmask) != f.cval) continue;
            const int i1 = i | (1 << ja);
            for (int col = 0; col < d; ++col) {
                const cd v0 = b.m[i * d + col], v1 = b.m[i1 * d + col];
                b.m[i * d + col] = f.m[0] * v0 + f.m[1] * v1;
                b.m[i1 * d + col] = f.m[2] * v0 + f.m[3] * v1;
            }
        }
    } else {   // F_U2: matrix index = x_t0 * 2 + x_t1
        const int ja = dblock_local(b.bits, f.t0), jb = dblock_local(b.bits, f.t1);
        for (int i = 0; i < d; ++i) {
            if (((i >> ja) & 1) || ((i >> jb) & 1)) continue;
            if ((dblock_glob(b.bits, i) & f.cmask) != f.cval) continue;
            int idx[4];
            for (int q = 0; q < 4; ++q) idx[q] = i | (((q >> 1) & 1) << ja) | ((q & 1) << jb);
            for (int col = 0; col < d; ++col) {
                cd v[4], w[4];
                for (int q = 0; q < 4; ++q) v[q] = b.m[idx[q] * d + col];
                for (int r = 0; r < 4; ++r) {
                    w[r] = 0;
                    for (int q = 0; q < 4; ++q) w[r] += f.m[r * 4 + q] * v[q];
                }
                for (int q = 0; q < 4; ++q) b.m[idx[q] * d + col] = w[q];
            }
        }
    }
}

// M <- diag(e^{i phase}) M for a quadratic-form diagonal on the block's bits
void dblock_diag(DBlock &b, const Diag &dg) {
    const int k = (int)b.bits.size(), d = 1 << k;
    for (int i = 0; i < d; ++i) {
        const uint64_t x = dblock_glob(b.bits, i);
        double ph = dg.g0;
        for (auto &kv : dg.a)
            if ((x >> kv.first) & 1) ph += kv.second;
        for (auto &kv : dg.pairs)
            if (((x >> kv.first.first) & 1) && ((x >> kv.first.second) & 1)) ph += kv.second;
        const cd e = std::polar(1.0, ph);
        for (int col = 0; col < d; ++col) b.m[i * d + col] *= e;
    }
}

}  // namespace

void dense_cells(int n, int T, int L, int k, int *cell_of) {
    int id = 0;
    const int W = T - L;
    int top = n;
    while (top > 0) {
        // windows of T - L high bits from the top; the last one takes the low bits
        int lo = top - W;
        if (lo <= L) lo = 0;
        const int sz = top - lo, nc = (sz + k - 1) / k;
        int b = top;
        for (int c = 0; c < nc; ++c) {   // near-equal cells, larger ones on top
            const int w = sz / nc + (c < sz % nc ? 1 : 0);
            for (int x = b - w; x < b; ++x) cell_of[x] = id;
            b -= w;
            id++;
        }
        top = lo;
    }
}

void fuse_dense(int n, int k, const int *cell_of, const std::vector<FOp> &in, std::vector<FOp> &out) {
    (void)n;
    std::vector<DBlock> blocks;
    struct Item {
        int block = -1;   // block id, or -1: the op below
        bool live = true;
        FOp op;
    };
    std::vector<Item> items;
    int last_touch[64], open_of[64];
    for (int b = 0; b < 64; ++b) last_touch[b] = open_of[b] = -1;
    auto close_block = [&](int id) {
        DBlock &b = blocks[id];
        if (!b.open) return;
        b.open = false;
        for (int x : b.bits) {
            open_of[x] = -1;
            last_touch[x] = std::max(last_touch[x], b.slot);
        }
    };
    auto close_touching = [&](uint64_t S) {
        for (int x = 0; x < 64; ++x)
            if (((S >> x) & 1) && open_of[x] >= 0) close_block(open_of[x]);
    };
    auto emit = [&](const FOp &f, uint64_t S) {
        close_touching(S);
        Item it;
        it.op = f;
        items.push_back(it);
        const int slot = (int)items.size() - 1;
        for (int x = 0; x < 64; ++x)
            if ((S >> x) & 1) last_touch[x] = slot;
    };
    // move open block `id` to the end of the sequence
    auto to_end = [&](int id) {
        DBlock &b = blocks[id];
        if (b.slot >= 0) items[b.slot].live = false;
        Item it;
        it.block = id;
        items.push_back(it);
        b.slot = (int)items.size() - 1;
    };
    int recent = -1;   // most recently created or grown open block
    for (const FOp &f : in) {
        if (f.kind == F_U1 || f.kind == F_U2) {
            uint64_t S = (1ull << f.t0) | f.cmask;
            if (f.kind == F_U2) S |= 1ull << f.t1;
            if (__builtin_popcountll(S) > k) {
                emit(f, S);
                continue;
            }
            std::vector<int> B;
            uint64_t U = S;
            for (int x = 0; x < 64; ++x)
                if (((S >> x) & 1) && open_of[x] >= 0 &&
                    std::find(B.begin(), B.end(), open_of[x]) == B.end()) {
                    B.push_back(open_of[x]);
                    for (int y : blocks[open_of[x]].bits) U |= 1ull << y;
                }
            if (__builtin_popcountll(U) > k) {
                for (int id : B) close_block(id);
                B.clear();
                U = S;
            }
            // pack into the most recent open block while there is room in its cell
            bool same_cell = recent >= 0 && blocks[recent].open;
            if (same_cell) {
                const int cc = cell_of[blocks[recent].bits[0]];
                for (int x = 0; x < 64; ++x)
                    if (((S >> x) & 1) && cell_of[x] != cc) same_cell = false;
            }
            if (B.empty() && same_cell && (int)blocks[recent].bits.size() + __builtin_popcountll(S) <= k) {
                B.push_back(recent);
                for (int y : blocks[recent].bits) U |= 1ull << y;
            }
            int id;
            if (B.empty()) {
                id = (int)blocks.size();
                blocks.emplace_back();
                blocks[id].m.assign(1, cd(1, 0));
            } else {
                id = B[0];
                for (size_t i = 1; i < B.size(); ++i) {   // merge: M = M_i (x) M_id (disjoint bits)
                    DBlock &a = blocks[id], &o = blocks[B[i]];
                    const int ka = (int)a.bits.size(), da = 1 << ka, dob = 1 << o.bits.size(), dd = da * dob;
                    std::vector<cd> m(dd * dd);
                    for (int r = 0; r < dd; ++r)
                        for (int c = 0; c < dd; ++c)
                            m[r * dd + c] = a.m[(r & (da - 1)) * da + (c & (da - 1))] * o.m[(r >> ka) * dob + (c >> ka)];
                    a.m.swap(m);
                    a.bits.insert(a.bits.end(), o.bits.begin(), o.bits.end());
                    a.n_gates += o.n_gates;
                    o.open = false;
                    if (o.slot >= 0) items[o.slot].live = false;
                    for (int y : o.bits) open_of[y] = id;
                }
            }
            to_end(id);
            DBlock &b = blocks[id];
            std::vector<int> extra;
            for (int x = 0; x < 64; ++x)
                if (((S >> x) & 1) && dblock_local(b.bits, x) < 0) extra.push_back(x);
            dblock_grow(b, extra);
            for (int x : b.bits) open_of[x] = id;
            dblock_apply(b, f);
            b.n_gates += f.n_gates;
            recent = id;
            continue;
        }
        if (f.kind == F_DIAG) {
            std::map<int, Diag> part;
            Diag rest;
            rest.g0 = f.diag.g0;
            for (auto &kv : f.diag.a) {
                const int id = open_of[kv.first];
                if (id >= 0) part[id].a[kv.first] += kv.second;
                else rest.a[kv.first] += kv.second;
            }
            for (auto &kv : f.diag.pairs) {
                const int i0 = open_of[kv.first.first], i1 = open_of[kv.first.second];
                if (i0 >= 0 && i0 == i1) part[i0].pairs[kv.first] += kv.second;
                else rest.pairs[kv.first] += kv.second;
            }
            for (auto &kv : part) dblock_diag(blocks[kv.first], kv.second);
            if (rest.a.empty() && rest.pairs.empty() && !part.empty()) {
                // only a global phase is left: it commutes with everything
                DBlock &b0 = blocks[part.begin()->first];
                if (rest.g0 != 0.0) {
                    Diag g;
                    g.g0 = rest.g0;
                    dblock_diag(b0, g);
                }
                b0.n_gates += f.n_gates;
                continue;
            }
            FOp r = f;
            r.diag = rest;
            emit(r, rest.support());
            continue;
        }
        emit(f, f.kind == F_GF2 ? ~0ull : (f.N() | f.D()));
    }
    out.clear();
    for (const Item &it : items) {
        if (!it.live) continue;
        if (it.block < 0) {
            out.push_back(it.op);
            continue;
        }
        const DBlock &b = blocks[it.block];
        FOp f;
        f.n_gates = b.n_gates;
        const int kb = (int)b.bits.size();
        if (kb == 1) {
            f.kind = F_U1;
            f.t0 = b.bits[0];
            for (int e = 0; e < 4; ++e) f.m[e] = b.m[e];
        } else if (kb == 2) {   // F_U2 index = x_t0 * 2 + x_t1: t0 is local bit 1
            f.kind = F_U2;
            f.t0 = b.bits[1];
            f.t1 = b.bits[0];
            for (int e = 0; e < 16; ++e) f.m[e] = b.m[e];
        } else {
            f.kind = F_DENSE;
            f.dbits = b.bits;
            f.dm = b.m;
        }
        out.push_back(f);
    }
}

// ---------------------------------------------------------------------------
// diagonal -> device descriptors and tables
// ---------------------------------------------------------------------------
namespace {
double wrap_angle(double x) {
    double r = std::remainder(x, 2.0 * kPi);
    return r;
}
float2 cexp_f(double ph) {
    double r = wrap_angle(ph);
    float2 v;
    v.x = (float)std::cos(r);
    v.y = (float)std::sin(r);
    return v;
}

struct DiagPlan {            // one Diag split into device descriptors
    std::vector<DiagDesc> descs;
    std::vector<std::vector<float2>> tables;   // per desc: its constants (offsets relative)
    bool count = false;        // applied as a count lookup (MK_DIAGC) instead
    int count_const = 0;       // its constants per sweep that applies it
};

// The count form of a diagonal (sweep-independent part of MK_DIAGC):
// phase(x) = g0 + gamma c1(x) + h c2(x), c1 = edges whose bits differ (zz)
// or are both set (!zz), c2 = popcount(x & mz).
struct CountForm {
    bool zz = true;
    double gamma = 0.0, h = 0.0;
    uint64_t mz = 0;
    std::map<int, uint64_t> cls;   // distance d -> mask of lower endpoints
    int stride = 1, n_z = 0;
};

bool count_form(const Diag &dg, CountForm &cf) {
    if (dg.pairs.empty() && dg.a.empty()) return false;
    const double w = dg.pairs.empty() ? 0.0 : dg.pairs.begin()->second;
    for (auto &kv : dg.pairs)
        if (std::fabs(kv.second - w) > 1e-12 * std::fabs(w)) return false;
    std::map<int, int> deg;
    for (auto &kv : dg.pairs) {
        deg[kv.first.first]++;
        deg[kv.first.second]++;
    }
    // ZZ type: pair weight -2 gamma, single-bit weight gamma deg(b); CZ type:
    // pair weight gamma.  What is left of the single-bit weights must be one
    // value h on a set of bits.
    auto residual_ok = [&](double gam_deg, uint64_t &mz, double &h) {
        mz = 0;
        h = 0.0;
        bool first = true;
        std::set<int> bits;
        for (auto &kv : dg.a) bits.insert(kv.first);
        for (auto &kv : deg) bits.insert(kv.first);
        for (int b : bits) {
            auto it = dg.a.find(b);
            const double have = it == dg.a.end() ? 0.0 : it->second;
            const double want = gam_deg * (deg.count(b) ? deg[b] : 0);
            const double r = have - want;
            if (std::fabs(r) <= 1e-12 * std::max(1.0, std::fabs(want))) continue;
            if (first) {
                h = r;
                first = false;
            } else if (std::fabs(r - h) > 1e-12 * std::max(1.0, std::fabs(h))) {
                return false;
            }
            mz |= 1ull << b;
        }
        return true;
    };
    cf.zz = residual_ok(-w / 2, cf.mz, cf.h);
    if (!cf.zz && !residual_ok(0.0, cf.mz, cf.h)) return false;
    cf.gamma = cf.zz ? -w / 2 : w;
    cf.cls.clear();
    for (auto &kv : dg.pairs) cf.cls[kv.first.second - kv.first.first] |= 1ull << kv.first.first;
    cf.stride = (int)dg.pairs.size() + 1;
    cf.n_z = __builtin_popcountll(cf.mz);
    if ((int)cf.cls.size() > kMaxCountClasses || cf.stride > 4095) return false;
    if ((size_t)cf.stride * (cf.n_z + 1) > 2048) return false;
    return true;
}

// constants of one MK_DIAGC op: the table, alignment, and the data slots
int count_const_size(const CountForm &cf, int R) {
    return cf.stride * (cf.n_z + 1) + 1 + R + 3 + 2 * (int)cf.cls.size();
}

// Slices: window s covers bits [8s, 8s+w), w = min(9, n-8s).  A single-bit
// term on b goes to slice b/8; a pair (b, c) goes to slice b/8 when c is
// inside that window; other pairs are grouped by (distance, angle) into
// popcount LUTs of the CZ type.
void plan_diag(int n, const Diag &d, DiagPlan &out) {
    const int ns = (n + 7) / 8;
    std::vector<std::map<int, double>> s_single(ns);
    std::vector<std::map<std::pair<int, int>, double>> s_pair(ns);
    std::map<std::pair<int, double>, uint64_t> groups;   // (d, gamma) -> mask of low bits
    for (auto &kv : d.a) {
        if (kv.second == 0.0) continue;
        s_single[kv.first / 8][kv.first] += kv.second;
    }
    for (auto &kv : d.pairs) {
        if (kv.second == 0.0) continue;
        int b = kv.first.first, c = kv.first.second;
        int s = b / 8;
        if (c < 8 * s + 9) {
            s_pair[s][kv.first] += kv.second;
        } else {
            groups[{c - b, kv.second}] |= 1ull << b;
        }
    }
    DiagDesc cur;
    std::memset(&cur, 0, sizeof cur);
    std::vector<float2> tab;
    bool g0_done = false;
    for (int s = 0; s < ns; ++s) {
        if (s_single[s].empty() && s_pair[s].empty()) continue;
        int lo = 8 * s, w = std::min(9, n - 8 * s);
        int k = cur.n_slices++;
        cur.slice_lo[k] = lo;
        cur.slice_w[k] = w;
        cur.slice_off[k] = (int)tab.size();
        // entry(v) = exp(i phase(v)), phase a quadratic form in v's bits: build it
        // multiplicatively in FP64 from entry(v without its lowest bit) times that
        // bit's single-term factor and the factors of the pairs it completes
        std::vector<cd> e1(w, cd(1, 0));
        std::vector<std::vector<std::pair<int, cd>>> e2(w);
        for (auto &kv : s_single[s]) e1[kv.first - lo] = std::polar(1.0, wrap_angle(kv.second));
        for (auto &kv : s_pair[s]) {
            const int b0 = kv.first.first - lo, b1 = kv.first.second - lo;
            const cd z = std::polar(1.0, wrap_angle(kv.second));
            e2[b0].push_back({b1, z});
            e2[b1].push_back({b0, z});
        }
        std::vector<cd> z((size_t)1 << w);
        z[0] = g0_done ? cd(1, 0) : std::polar(1.0, wrap_angle(d.g0));
        for (int v = 1; v < (1 << w); ++v) {
            const int b = __builtin_ctz(v), vp = v & (v - 1);
            cd f = z[vp] * e1[b];
            for (auto &pr : e2[b])
                if ((vp >> pr.first) & 1) f *= pr.second;
            z[v] = f;
        }
        for (int v = 0; v < (1 << w); ++v) {
            const double m = std::abs(z[v]);   // keep exactly unit modulus before rounding
            tab.push_back(float2{(float)(z[v].real() / m), (float)(z[v].imag() / m)});
        }
        g0_done = true;
    }
    if (!g0_done) {
        // a constant even when g0 = 0, so that the descriptor does not depend on
        // the angle values (plans of batch items with other angles stay alike)
        cur.gph_off = (int)tab.size();
        tab.push_back(cexp_f(d.g0));
        cur.pad0 = 1;
    }
    for (auto &kv : groups) {
        if (cur.n_groups == kMaxLutGroups) {
            out.descs.push_back(cur);
            out.tables.push_back(tab);
            std::memset(&cur, 0, sizeof cur);
            tab.clear();
        }
        int k = cur.n_groups++;
        cur.grp_type[k] = 1;   // CZ-type: popcount(x & (x >> d) & m)
        cur.grp_d[k] = kv.first.first;
        cur.grp_mask[k] = kv.second;
        cur.grp_off[k] = (int)tab.size();
        int cnt = popc64(kv.second);
        for (int c = 0; c <= cnt; ++c) tab.push_back(cexp_f(c * kv.first.second));
    }
    out.descs.push_back(cur);
    out.tables.push_back(tab);
}

size_t diag_const_size(const DiagPlan &dp) {
    size_t s = 0;
    for (auto &t : dp.tables) s += t.size();
    return s;
}
}  // namespace

// ---------------------------------------------------------------------------
// scheduler: greedy commutation-aware packing of fused ops into tile passes
// ---------------------------------------------------------------------------
namespace {
struct OpCost {
    int n_const = 0;
    int n_micro = 1;
    int n_diag = 0;
};

// constants (complex64 entries) of one dense block's tables (see DenseKind)
int dense_const_size(int dprec) {
    switch (dprec) {
        case DS_FP32: return 32 * 32;
        case DS_TF32X3: return 2 * 32 * 32;
        default: return 4 * 8 * 32;   // DS_BF16
    }
}

OpCost op_cost(int n, const FOp &f, int R, const DiagPlan *dp, int dprec) {
    OpCost c;
    switch (f.kind) {
        case F_DENSE: c.n_const = dense_const_size(dprec) + 1; break;   // + alignment padding
        case F_U1: c.n_const = 5; break;   // 4 entries + the even-offset pad of the real form
        case F_U2: c.n_const = 16; break;
        case F_QFT: c.n_const = 1 << R; break;
        case F_DIAG:
            if (dp->count) {
                c.n_const = dp->count_const;
                c.n_diag = 0;
                c.n_micro = 1;
                break;
            }
            c.n_const = (int)diag_const_size(*dp);
            c.n_diag = (int)dp->descs.size();
            c.n_micro = c.n_diag;
            break;
        default: break;
    }
    (void)n;
    return c;
}

int tile_local(const TilePass &tp, int b) {
    if (b < tp.L) return b;
    for (int k = 0; k < tp.H; ++k)
        if (tp.hb[k] == b) return tp.L + k;
    return -1;
}

uint64_t glob_of_local(const TilePass &tp, int tb) {
    return tb < tp.L ? (1ull << tb) : (1ull << tp.hb[tb - tp.L]);
}

// choose item-bit order so that a warp's 32 lanes hit distinct banks; smem
// offsets are XOR-linear (tp.smem_contrib); vec sweeps access 16 bytes
void choose_item_bits(const TilePass &tp, Sweep &sw) {
    std::vector<int> cand;
    uint64_t gmask = 0;
    for (int j = 0; j < sw.r; ++j) gmask |= 1ull << sw.gbit[j];
    for (int tb = 0; tb < tp.T; ++tb)
        if (!((gmask >> tb) & 1)) cand.push_back(tb);
    const int k = (int)cand.size();
    const int nl = std::min(5, k);
    const int words_per = sw.vec ? 2 : 1;
    // memoised: the answer depends only on the candidate bits' offsets
    thread_local std::map<std::vector<int>, std::vector<int>> memo;
    std::vector<int> key;
    key.push_back(words_per);
    for (int i = 0; i < k; ++i) key.push_back(tp.smem_contrib[cand[i]]);
    auto hit = memo.find(key);
    if (hit != memo.end()) {
        for (int i = 0; i < k; ++i) sw.tbit[i] = cand[hit->second[i]];
        return;
    }
    std::vector<int> best;
    int best_cost = 1 << 30;
    std::vector<int> idx(nl);
    for (int i = 0; i < nl; ++i) idx[i] = i;
    while (true) {
        int words[32];
        for (int l = 0; l < (1 << nl); ++l) {
            int w = 0;
            for (int i = 0; i < nl; ++i)
                if ((l >> i) & 1) w ^= tp.smem_contrib[cand[idx[i]]];
            words[l] = w;
        }
        // the offsets are XOR combinations of independent bits: all distinct
        int bank_cnt[32] = {0};
        for (int l = 0; l < (1 << nl); ++l)
            for (int e = 0; e < 2 * words_per; ++e) bank_cnt[(2 * words[l] + e) & 31]++;
        int cost = 0;
        for (int b = 0; b < 32; ++b) cost = std::max(cost, bank_cnt[b]);
        if (cost < best_cost) {
            best_cost = cost;
            best.assign(idx.begin(), idx.end());
        }
        int i = nl - 1;
        while (i >= 0 && idx[i] == k - nl + i) --i;
        if (i < 0) break;
        idx[i]++;
        for (int j = i + 1; j < nl; ++j) idx[j] = idx[j - 1] + 1;
    }
    std::vector<int> order_idx;
    std::vector<bool> used(k, false);
    for (int i : best) {
        order_idx.push_back(i);
        used[i] = true;
    }
    for (int i = 0; i < k; ++i)
        if (!used[i]) order_idx.push_back(i);
    if (memo.size() < 4096) memo[key] = order_idx;
    for (int i = 0; i < k; ++i) sw.tbit[i] = cand[order_idx[i]];
}

// TMA geometry for the tile bit set S: dims = low bits, runs of tile bits
// (split into <= 8-bit boxes), gaps of non-tile bits; the batch rides on the
// top gap or gets a dim of its own.
TmaPlan tma_geometry(int n, int L, uint64_t S, int batch) {
    TmaPlan g;
    int nd = 0;
    auto add = [&](int kind, int lo_bit, int bits, int off) {
        if (nd >= 5) {
            nd = 6;
            return;
        }
        g.kind[nd] = kind;
        g.off[nd] = off;
        g.w[nd] = bits;
        g.gdim[nd] = kind == 2 ? (uint64_t)batch : (1ull << bits);
        g.gstride[nd] = kind == 2 ? (8ull << n) : (8ull << lo_bit);
        g.box[nd] = kind == 0 ? (1u << bits) : 1u;
        nd++;
    };
    add(0, 0, L, 0);
    int b = L, outer = 0;
    while (b < n && nd <= 5) {
        bool t = (S >> b) & 1;
        int e = b;
        while (e < n && (((S >> e) & 1) != 0) == t) ++e;
        if (t) {
            for (int c = b; c < e; c += 8) add(0, c, std::min(8, e - c), 0);
        } else {
            add(1, b, e - b, outer);
            outer += e - b;
        }
        b = e;
    }
    if (nd <= 5 && batch > 1) {
        if (g.kind[nd - 1] == 1 && !((S >> (n - 1)) & 1)) {
            g.batch_dim = nd - 1;
            g.gdim[nd - 1] *= (uint64_t)batch;
        } else {
            add(2, n, 0, 0);
            g.batch_dim = nd - 1;
        }
    }
    if (nd > 5) return TmaPlan();
    g.ndims = nd;
    for (int d = nd; d < 5; ++d) {   // pad to 5-D with extent-1 dims
        g.kind[d] = 0;
        g.w[d] = 0;
        g.gdim[d] = 1;
        g.box[d] = 1;
        const uint64_t prev = (d - 1 == 0) ? 8ull : g.gstride[d - 1];
        g.gstride[d] = prev * g.gdim[d - 1];
    }
    for (int d = 1; d < 5; ++d)
        if (g.gstride[d] >= (1ull << 40) || (g.gstride[d] & 15)) return TmaPlan();
    g.ok = true;
    return g;
}

// Complete a tile's bit set S (the low bits and the high bits its ops need)
// to T bits.  The lowest unused high bits, unless that leaves more than the 5
// tensor dims one TMA copy can take (each run of tile bits and each gap of
// other bits is a dim): then the smallest gaps below the highest tile bit are
// filled first, which merges runs, and the rest of the room extends the top
// run upward.  Where neither fits the tensor copy, the default stays (the
// pass then copies its tile row by row).
static uint64_t pad_tile_bits(int n, int L, int T, uint64_t S, int batch) {
    uint64_t def = S;
    for (int b = L; b < n && popc64(def) < T; ++b) def |= 1ull << b;
    if (tma_geometry(n, L, def, batch).ok) return def;
    int top = -1;
    for (int b = n - 1; b >= L; --b)
        if ((S >> b) & 1) {
            top = b;
            break;
        }
    if (top < 0) return def;
    int slack = T - popc64(S);
    std::vector<std::pair<int, int>> gaps;   // (length, first bit) of the runs of other bits in [L, top)
    for (int b = L; b < top;) {
        if ((S >> b) & 1) {
            ++b;
            continue;
        }
        int e = b;
        while (e < top && !((S >> e) & 1)) ++e;
        gaps.push_back({e - b, b});
        b = e;
    }
    std::sort(gaps.begin(), gaps.end());
    uint64_t P = S;
    for (auto &g : gaps)
        if (g.first <= slack) {
            for (int b = g.second; b < g.second + g.first; ++b) P |= 1ull << b;
            slack -= g.first;
        }
    for (int b = top + 1; b < n && slack > 0; ++b)
        if (!((P >> b) & 1)) {
            P |= 1ull << b;
            --slack;
        }
    for (int b = L; b < n && slack > 0; ++b)
        if (!((P >> b) & 1)) {
            P |= 1ull << b;
            --slack;
        }
    return tma_geometry(n, L, P, batch).ok ? P : def;
}

// FP64 -> TF32 (FP32 with 10 explicit mantissa bits), round to nearest even
float tf32_round(double x) {
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0xfffu + ((u >> 13) & 1u);
        u &= 0xffffe000u;
    }
    std::memcpy(&f, &u, 4);
    return f;
}

// FP64 -> BF16 bits, round to nearest even (through FP32)
uint16_t bf16_bits(double x) {
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Set while build_fused_plan builds one of several per-item plans: the pass
// builder then keeps to micro-op forms that do not depend on angle values.
thread_local bool t_item_plan = false;

struct PassBuilder {
    int n, L, T, R, dprec;
    HostPass hp;
    TilePass &tp;
    std::vector<float2> &cst;
    uint64_t cur_group = 0;   // tile-local bits of the open sweep
    int open = -1;
    PassBuilder(int n_, int L_, int T_, int R_, uint64_t S, int batch, int dprec_)
        : n(n_), L(L_), T(T_), R(R_), dprec(dprec_), tp(hp.tile), cst(hp.consts) {
        std::memset(&tp, 0, sizeof(TilePass));
        hp.type = HostPass::TILE;
        tp.n = n;
        tp.L = L;
        tp.T = T;
        tp.R = R;
        tp.H = T - L;
        int k = 0;
        for (int b = L; b < n; ++b)
            if ((S >> b) & 1) tp.hb[k++] = b;
        hp.tma = tma_geometry(n, L, S, batch);
        // 128-byte swizzle: 16-byte chunk bits [1,4) of the float2 offset are
        // XORed with row bits [4,7) (rows of 128 bytes = 16 amplitudes)
        tp.swizzle = (hp.tma.ok && L == 4 && T >= 7) ? 1 : 0;
        for (int tb = 0; tb < T; ++tb) {
            int c = 1 << tb;
            if (tp.swizzle && tb >= 4 && tb < 7) c ^= 1 << (tb - 3);
            tp.smem_contrib[tb] = c;
        }
    }
    int group_index(int tb) {
        for (int j = 0; j < tp.sweeps[open].r; ++j)
            if (tp.sweeps[open].gbit[j] == tb) return j;
        return -1;
    }
    // ensure the open sweep's group holds tile-local bits `need`
    void need_bits(uint64_t need) {
        if (open >= 0 && (popc64(cur_group | need) <= R)) {
            Sweep &sw = tp.sweeps[open];
            for (int tb = 0; tb < T; ++tb)
                if (((need >> tb) & 1) && !((cur_group >> tb) & 1)) sw.gbit[sw.r++] = tb;
            cur_group |= need;
            return;
        }
        close_sweep();
        open = tp.n_sweeps++;
        Sweep &sw = tp.sweeps[open];
        std::memset(&sw, 0, sizeof sw);
        sw.op_begin = sw.op_end = tp.n_micro;
        cur_group = need;
        for (int tb = 0; tb < T; ++tb)
            if ((need >> tb) & 1) sw.gbit[sw.r++] = tb;
    }
    void close_sweep() {
        if (open < 0) return;
        Sweep &sw = tp.sweeps[open];
        // pad the group to R bits: tile bit 0 first (16-byte pair accesses),
        // then unused tile bits, highest first
        if (sw.r < std::min(R, T) && !(cur_group & 1ull)) {
            sw.gbit[sw.r++] = 0;
            cur_group |= 1ull;
        }
        // (padding bits that share a bank bit with a group bit last)
        for (int pass = 0; pass < 2; ++pass)
            for (int tb = T - 1; tb >= 0 && sw.r < std::min(R, T); --tb) {
                if ((cur_group >> tb) & 1) continue;
                const int partner = tp.swizzle ? swizzle_partner(tb) : -1;
                if (pass == 0 && partner >= 0 && ((cur_group >> partner) & 1)) continue;
                sw.gbit[sw.r++] = tb;
                cur_group |= 1ull << tb;
            }
        std::sort(sw.gbit, sw.gbit + sw.r);
        // A sweep of rotations and diagonals: the bits of its first rotation run
        // come right after tile bit 0 (which stays first: 16-byte pair
        // accesses), so that a rotation program's first layer owns a contiguous
        // run of low group positions and runs without its padded identities.
        {
            uint64_t first = 0;
            bool ok = true, in_first = true;
            for (int k = sw.op_begin; k < tp.n_micro; ++k) {
                const int kd = tp.micro[k].kind;
                if (kd == MK_ROT) {
                    if (in_first) first |= 1ull << tp.micro[k].a;
                } else if (kd == MK_DIAGC || kd == MK_DIAG || kd == MK_DIAGQ) {
                    in_first = false;
                } else {
                    ok = false;
                }
            }
            if (ok && first) {
                int g[kMaxGroup], m = 0;
                const bool b0 = sw.gbit[0] == 0;
                if (b0) g[m++] = 0;
                for (int j = b0 ? 1 : 0; j < sw.r; ++j)
                    if ((first >> sw.gbit[j]) & 1) g[m++] = sw.gbit[j];
                for (int j = b0 ? 1 : 0; j < sw.r; ++j)
                    if (!((first >> sw.gbit[j]) & 1)) g[m++] = sw.gbit[j];
                for (int j = 0; j < sw.r; ++j) sw.gbit[j] = g[j];
            }
        }
        sw.vec = (sw.r >= 2 && sw.gbit[0] == 0) ? 1 : 0;
        sw.op_end = tp.n_micro;
        choose_item_bits(tp, sw);
        open = -1;
        cur_group = 0;
    }
    // A dense block gets a sweep of its own: 5 group bits (the block's tile
    // bits, padded with the identity on the lowest free tile bits) and the
    // block's tables in the layout its arithmetic reads (DenseKind).
    void add_dense(const FOp &f) {
        close_sweep();
        const int si = tp.n_sweeps++;
        Sweep &sw = tp.sweeps[si];
        std::memset(&sw, 0, sizeof sw);
        sw.dense = dprec;
        sw.r = 5;
        sw.scale = 1.f;
        sw.op_begin = sw.op_end = tp.n_micro;
        const int kb = (int)f.dbits.size();
        int G[5];
        uint64_t used = 0;
        for (int j = 0; j < kb; ++j) {
            G[j] = tile_local(tp, f.dbits[j]);
            used |= 1ull << G[j];
        }
        int ng = kb;
        for (int tb = 0; tb < T && ng < 5; ++tb)
            if (!((used >> tb) & 1)) {
                G[ng++] = tb;
                used |= 1ull << tb;
            }
        std::vector<int> cols;
        for (int tb = 0; tb < T; ++tb)
            if (!((used >> tb) & 1)) cols.push_back(tb);
        int order[5] = {0, 1, 2, 3, 4};   // group bit q is G[order[q]]
        if (dprec == DS_FP32 || dprec == DS_TF32X3) {
            // a thread per column (its 32 amplitudes at the group bits' offsets)
            for (int q = 0; q < 5; ++q) sw.gbit[q] = G[q];
            sw.vec = 0;
            choose_item_bits(tp, sw);
        } else {
            // tensor-core operand loads: lane bits 0-1 are group bits 0-1 (block
            // rows), lane bits 2-4 are item bits 0-2 (columns); pick the five
            // bits whose 8-byte accesses spread over the most banks
            const int nc = (int)cols.size(), m = std::min(3, nc);
            int best = 1 << 30, ba = 0, bb = 1;
            uint32_t bmask = (1u << m) - 1;
            // memoised on the bits' shared-memory offsets
            thread_local std::map<std::vector<int>, std::array<int, 3>> memo;
            std::vector<int> key;
            for (int e = 0; e < 5; ++e) key.push_back(tp.smem_contrib[G[e]]);
            for (int i = 0; i < nc; ++i) key.push_back(tp.smem_contrib[cols[i]]);
            auto hit = memo.find(key);
            if (hit != memo.end()) {
                best = 0;
                ba = hit->second[0];
                bb = hit->second[1];
                bmask = (uint32_t)hit->second[2];
            }
            for (int a = 0; a < 5 && best > 0; ++a)
                for (int b = a + 1; b < 5; ++b)
                    for (uint32_t cm = 0; cm < (1u << nc); ++cm) {
                        if (__builtin_popcount(cm) != m) continue;
                        int v[5] = {tp.smem_contrib[G[a]], tp.smem_contrib[G[b]], 0, 0, 0}, e = 2;
                        for (int i = 0; i < nc; ++i)
                            if ((cm >> i) & 1) v[e++] = tp.smem_contrib[cols[i]];
                        // distinct 8-byte words per bank pair (with fewer than 3
                        // column bits, lanes alias onto the same words)
                        const int nl = 1 << (2 + m);
                        int cnt[16] = {0}, cost = 0;
                        for (int lane = 0; lane < nl; ++lane) {
                            int o = 0;
                            for (int x = 0; x < 2 + m; ++x)
                                if ((lane >> x) & 1) o ^= v[x];
                            cost = std::max(cost, ++cnt[o & 15]);
                        }
                        if (cost < best) {
                            best = cost;
                            ba = a;
                            bb = b;
                            bmask = cm;
                        }
                    }
            if (memo.size() < 4096) memo[key] = {ba, bb, (int)bmask};
            order[0] = ba;
            order[1] = bb;
            int q = 2;
            for (int e = 0; e < 5; ++e)
                if (e != ba && e != bb) order[q++] = e;
            for (int e = 0; e < 5; ++e) sw.gbit[e] = G[order[e]];
            int t = 0;
            for (int i = 0; i < nc; ++i)
                if ((bmask >> i) & 1) sw.tbit[t++] = cols[i];
            for (int i = 0; i < nc; ++i)
                if (!((bmask >> i) & 1)) sw.tbit[t++] = cols[i];
        }
        // the 32 x 32 matrix in group-bit order (identity on the padding bits)
        const int dim = 1 << kb;
        std::vector<cd> U(32 * 32, cd(0, 0));
        for (int i = 0; i < 32; ++i)
            for (int j = 0; j < 32; ++j) {
                int bi = 0, bj = 0, pi = 0, pj = 0;
                for (int q = 0; q < 5; ++q) {
                    const int e = order[q];
                    if (e < kb) {
                        bi |= ((i >> q) & 1) << e;
                        bj |= ((j >> q) & 1) << e;
                    } else {
                        pi |= ((i >> q) & 1) << (e - kb);
                        pj |= ((j >> q) & 1) << (e - kb);
                    }
                }
                if (pi == pj) U[i * 32 + j] = f.dm[bi * dim + bj];
            }
        if (cst.size() & 1) cst.push_back(float2{0.f, 0.f});   // 16-byte aligned tables (float4 reads)
        sw.dcst = (int)cst.size();
        if (dprec == DS_FP32) {
            for (int e = 0; e < 32 * 32; ++e) cst.push_back(float2{(float)U[e].real(), (float)U[e].imag()});
        } else if (dprec == DS_TF32X3) {
            // tcgen05 B operands: Re U hi, Im U hi, Re U lo, Im U lo, each 32 x 32
            // K-major (row = output i, 32 inputs j of 4 bytes) with the 128-byte
            // swizzle (16-byte chunk j / 4 of row i at chunk (j / 4) ^ (i % 8)),
            // starting on a 1024-byte boundary of the constant table
            while (cst.size() % 128) cst.push_back(float2{0.f, 0.f});
            sw.dcst = (int)cst.size();
            std::vector<float> t(4 * 32 * 32, 0.f);
            for (int i = 0; i < 32; ++i)
                for (int j = 0; j < 32; ++j) {
                    const cd u = U[i * 32 + j];
                    const float hr = tf32_round(u.real()), hm = tf32_round(u.imag());
                    const int e = i * 32 + (((j >> 2) ^ (i & 7)) << 2) + (j & 3);
                    t[e] = hr;
                    t[1024 + e] = hm;
                    t[2048 + e] = tf32_round(u.real() - (double)hr);
                    t[3072 + e] = tf32_round(u.imag() - (double)hm);
                }
            for (int e = 0; e < 4 * 1024; e += 2) cst.push_back(float2{t[e], t[e + 1]});
        } else {
            // m16n8k16 B operand: k = 2 * row + (0: re, 1: im) within a 16-wide
            // k-step, n = 2 * out_row + (0: re, 1: im) within an 8-wide n-tile
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 8; ++t)
                    for (int lane = 0; lane < 32; ++lane) {
                        const int g = lane >> 2, q = lane & 3, orow = 4 * t + (g >> 1);
                        const bool im = (g & 1) != 0;
                        uint32_t w[2];
                        for (int h = 0; h < 2; ++h) {
                            const cd u = U[orow * 32 + 8 * s + 4 * h + q];
                            const double b0 = im ? u.imag() : u.real(), b1 = im ? u.real() : -u.imag();
                            w[h] = (uint32_t)bf16_bits(b0) | ((uint32_t)bf16_bits(b1) << 16);
                        }
                        float2 v;
                        std::memcpy(&v.x, &w[0], 4);
                        std::memcpy(&v.y, &w[1], 4);
                        cst.push_back(v);
                    }
        }
    }
    // Uncontrolled one-qubit ops on distinct bits commute, so a run of them
    // (a layer) is held back and added in the order that fills the open sweep
    // first: the layer's ops on the open group's bits join it, e.g. the
    // sweep that holds a diagonal applies the next layer on its own bits too.
    std::vector<FOp> pend;
    uint64_t pend_bits = 0;
    int pending_ops() const { return (int)pend.size(); }
    void add(const FOp &f, const DiagPlan *dp) {
        if (f.kind == F_U1 && f.cmask == 0) {
            if ((pend_bits >> f.t0) & 1) flush_pending();
            pend.push_back(f);
            pend_bits |= 1ull << f.t0;
            return;
        }
        flush_pending();
        add_now(f, dp);
    }
    void flush_pending() {
        if (pend.empty()) return;
        std::vector<FOp> ops;
        ops.swap(pend);
        pend_bits = 0;
        std::vector<char> in_open(ops.size(), 0);
        if (open >= 0)
            for (size_t i = 0; i < ops.size(); ++i) in_open[i] = (cur_group >> tile_local(tp, ops[i].t0)) & 1;
        for (size_t i = 0; i < ops.size(); ++i)
            if (in_open[i]) add_now(ops[i], nullptr);
        // The rest fill groups of R bits in the order given.  With the 128-byte
        // swizzle, tile bits t and t + 3 (t = 1..3) select the same bank bit of
        // an access; a group that holds both leaves a warp's lanes one bank bit
        // short (two-way conflicts on every access of the sweep), so each group
        // is filled with the first remaining op whose partner it does not hold.
        std::vector<size_t> rest;
        for (size_t i = 0; i < ops.size(); ++i)
            if (!in_open[i]) rest.push_back(i);
        if (tp.swizzle) {
            std::vector<size_t> order;
            uint64_t grp = open >= 0 ? cur_group : 0;
            int room = open >= 0 ? std::max(0, R - popc64(cur_group)) : R;
            while (!rest.empty()) {
                if (room == 0) {
                    grp = 0;
                    room = R;
                }
                size_t pick = 0;
                for (size_t k = 0; k < rest.size(); ++k) {
                    const int tb = tile_local(tp, ops[rest[k]].t0);
                    const int partner = swizzle_partner(tb);
                    if (partner < 0 || !((grp >> partner) & 1)) {
                        pick = k;
                        break;
                    }
                }
                grp |= 1ull << tile_local(tp, ops[rest[pick]].t0);
                --room;
                order.push_back(rest[pick]);
                rest.erase(rest.begin() + (long)pick);
            }
            rest.swap(order);
        }
        for (size_t i : rest) add_now(ops[i], nullptr);
    }
    // the tile bit whose 128-byte-swizzle contribution shares a bank bit with tb
    static int swizzle_partner(int tb) {
        if (tb >= 1 && tb <= 3) return tb + 3;
        if (tb >= 4 && tb <= 6) return tb - 3;
        return -1;
    }
    void add_now(const FOp &f, const DiagPlan *dp) {
        switch (f.kind) {
            case F_DENSE:
                add_dense(f);
                break;
            case F_U1: case F_U2: case F_QFT: {
                uint64_t need = 0;
                int ta = tile_local(tp, f.kind == F_QFT ? f.p : f.t0);
                need |= 1ull << ta;
                int tb2 = -1;
                if (f.kind == F_U2) {
                    tb2 = tile_local(tp, f.t1);
                    need |= 1ull << tb2;
                }
                need_bits(need);
                MicroOp mo;
                std::memset(&mo, 0, sizeof mo);
                mo.a = ta;   // tile-local for now; converted to group index at finalize
                mo.b = tb2;
                mo.cmask = f.cmask;
                mo.cval = f.cval;
                mo.cst = (int)cst.size();
                if (f.kind == F_U1) {
                    const cd *m = f.m;
                    bool h = f.cmask == 0 && m[0] == cd(kSqrtHalf, 0) && m[1] == cd(kSqrtHalf, 0) &&
                             m[2] == cd(kSqrtHalf, 0) && m[3] == cd(-kSqrtHalf, 0);
                    // RX family [[c, i s], [i s, c]] and real matrices have cheaper forms
                    bool rxc = f.cmask == 0 && m[0].imag() == 0 && m[0] == m[3] && m[1].real() == 0 &&
                               m[1] == m[2];
                    bool real = f.cmask == 0 && m[0].imag() == 0 && m[1].imag() == 0 && m[2].imag() == 0 &&
                                m[3].imag() == 0;
                    // a real rotation c [[1, t], [-t, 1]] with |t| <= 1: one packed FMA per
                    // amplitude, c folded into the sweep scale (finalize)
                    bool rot = !t_item_plan && real && m[0] == m[3] && m[1] == -m[2] && m[0].real() != 0.0 &&
                               std::abs(m[1].real()) <= std::abs(m[0].real());
                    if (h) {
                        mo.kind = MK_H;
                    } else if (rot) {
                        mo.kind = MK_ROT;
                        const double c = m[0].real(), t = m[1].real() / c;
                        cst.push_back(float2{(float)t, (float)t});
                        cst.push_back(float2{(float)-t, (float)-t});
                        // c travels to finalize in the (otherwise unused) control value
                        std::memcpy(&mo.cval, &c, sizeof c);
                    } else if (rxc) {
                        mo.kind = MK_RXC;
                        cst.push_back(float2{(float)m[0].real(), (float)m[1].imag()});
                    } else if (real) {
                        mo.kind = MK_U1R;
                        if (cst.size() & 1) cst.push_back(float2{0.f, 0.f});
                        mo.cst = (int)cst.size();
                        for (int e = 0; e < 4; ++e) {
                            const float v = (float)m[e].real();
                            cst.push_back(float2{v, v});
                        }
                    } else {
                        mo.kind = MK_U1;
                        for (int e = 0; e < 4; ++e) {
                            float2 v;
                            v.x = (float)m[e].real();
                            v.y = (float)m[e].imag();
                            cst.push_back(v);
                        }
                        // the FP64 matrix, for a layer that becomes MK_ZYZ (merge_layers)
                        mo.p = (int)u1_fp64.size();
                        u1_fp64.push_back({m[0], m[1], m[2], m[3]});
                    }
                } else if (f.kind == F_U2) {
                    mo.kind = MK_U2;
                    for (int e = 0; e < 16; ++e) {
                        float2 v;
                        v.x = (float)f.m[e].real();
                        v.y = (float)f.m[e].imag();
                        cst.push_back(v);
                    }
                } else {
                    mo.kind = MK_QFT;
                    mo.p = f.p;
                    mo.lo = f.lo;
                    hp.uses_roots = 1;
                    // group twiddle table filled at finalize (needs final group)
                    for (int e = 0; e < (1 << R); ++e) cst.push_back(float2{1.f, 0.f});
                }
                tp.micro[tp.n_micro++] = mo;
                tp.sweeps[open].op_end = tp.n_micro;
                break;
            }
            case F_DIAG: {
                if (open < 0) need_bits(0);
                if (dp->count) {   // completed per sweep at finalize (to_diagc)
                    MicroOp mo;
                    std::memset(&mo, 0, sizeof mo);
                    mo.kind = MK_DIAGC;
                    mo.cst = (int)count_src.size();
                    count_src.push_back(&f.diag);
                    tp.micro[tp.n_micro++] = mo;
                    tp.sweeps[open].op_end = tp.n_micro;
                    break;
                }
                for (size_t k = 0; k < dp->descs.size(); ++k) {
                    DiagDesc dd = dp->descs[k];
                    int base = (int)cst.size();
                    for (int s = 0; s < dd.n_slices; ++s) dd.slice_off[s] += base;
                    for (int g = 0; g < dd.n_groups; ++g) dd.grp_off[g] += base;
                    if (dd.pad0) dd.gph_off += base;
                    cst.insert(cst.end(), dp->tables[k].begin(), dp->tables[k].end());
                    int di = count_diags++;
                    tp.diags[di] = dd;
                    diag_src[di] = (dp->descs.size() == 1 && dd.n_tw == 0) ? &f.diag : nullptr;
                    MicroOp mo;
                    std::memset(&mo, 0, sizeof mo);
                    mo.kind = MK_DIAG;
                    mo.cst = di;
                    tp.micro[tp.n_micro++] = mo;
                }
                tp.sweeps[open].op_end = tp.n_micro;
                break;
            }
            default: break;
        }
    }
    int count_diags = 0;
    const Diag *diag_src[kMaxDiag] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<const Diag *> count_src;   // MK_DIAGC ops before finalize: cst = index here
    bool count_failed = false;
    std::vector<std::array<cd, 4>> u1_fp64;   // FP64 matrices of the MK_U1 ops (index in MicroOp::p)
    std::vector<std::pair<int, int>> count_luts;   // (offset, entries) of the count tables built
    // A diagonal g0 + gamma c1(x) + h c2(x) (count_form: uniform-angle RZZ sets
    // such as TFIM chains and QAOA cost layers, uniform CZ / CP sets, uniform
    // single-qubit phases) is applied as a count lookup (Sec. 5.1 phase LUT
    // indexed by popcounts): one table entry and one complex multiply per
    // amplitude.  Fills the sweep-dependent part of the MK_DIAGC op.
    bool to_diagc(MicroOp &mo, const Sweep &sw, const Diag &dg) {
        CountForm cf;
        if (!count_form(dg, cf)) return false;
        int gb[kMaxGroup];
        uint64_t gm = 0;
        for (int m = 0; m < sw.r; ++m) {
            gb[m] = __builtin_ctzll(glob_of_local(tp, sw.gbit[m]));
            gm |= 1ull << gb[m];
        }
        // neighbours outside the group, edges inside it
        uint64_t nb[kMaxGroup] = {0, 0, 0, 0, 0};
        uint64_t qc[2] = {0, 0};
        std::vector<std::pair<int, int>> inner;
        for (auto &kv : dg.pairs) {
            const int u = kv.first.first, v = kv.first.second;
            const bool iu = (gm >> u) & 1, iv = (gm >> v) & 1;
            for (int m = 0; m < sw.r; ++m) {
                if (iu && !iv && gb[m] == u) nb[m] |= 1ull << v;
                if (iv && !iu && gb[m] == v) nb[m] |= 1ull << u;
            }
            if (iu && iv) {
                int mu = 0, mv = 0;
                for (int m = 0; m < sw.r; ++m) {
                    if (gb[m] == u) mu = m;
                    if (gb[m] == v) mv = m;
                }
                inner.push_back({mu, mv});
            }
        }
        for (int j = 0; j < (1 << sw.r); ++j) {
            uint64_t q = 0;
            for (auto &e : inner) {
                const int bu = (j >> e.first) & 1, bv = (j >> e.second) & 1;
                q += cf.zz ? (uint64_t)(bu ^ bv) : (uint64_t)(bu & bv);
            }
            if (q > 15) return false;   // at most C(5, 2) = 10 edges inside a group
            qc[j >> 4] |= q << (4 * (j & 15));
        }
        uint64_t degs = 0, zinc = 0;
        for (int m = 0; m < sw.r; ++m) {
            degs |= (uint64_t)__builtin_popcountll(nb[m]) << (6 * m);
            if ((cf.mz >> gb[m]) & 1) zinc |= (uint64_t)cf.stride << (12 * m);
        }
        const int lut = (int)cst.size();
        const size_t n_e = dg.pairs.size();
        for (int c2 = 0; c2 <= cf.n_z; ++c2)
            for (size_t c1 = 0; c1 <= n_e; ++c1) cst.push_back(cexp_f(dg.g0 + cf.gamma * (double)c1 + cf.h * c2));
        count_luts.push_back({lut, (int)((cf.n_z + 1) * (n_e + 1))});
        if (cst.size() & 1) cst.push_back(float2{0.f, 0.f});   // 16-byte aligned data
        const int dat = (int)cst.size();
        auto slot64 = [&](uint64_t v) {
            float2 f;
            std::memcpy(&f, &v, 8);
            cst.push_back(f);
        };
        for (int m = 0; m < sw.r; ++m) slot64(nb[m]);
        slot64(degs);
        slot64(cf.mz);
        slot64(zinc);
        for (auto &kv : cf.cls) {
            slot64(kv.second);
            slot64((uint64_t)kv.first);
        }
        mo.kind = MK_DIAGC;
        mo.cst = lut;
        mo.lo = dat;
        mo.a = (int)cf.cls.size();
        mo.b = cf.zz ? 0 : 1;
        mo.p = cf.stride;
        mo.cmask = qc[0];
        mo.cval = qc[1];
        return true;
    }

    // A diagonal whose sweep group spans more than two slice tables (or a LUT
    // group) would take the per-amplitude general path; factor it instead as
    // (tables at group bits 0) x Q(group bits) x couplings(group bit, other bit).
    bool to_diagq(MicroOp &mo, const Sweep &sw) {
        const Diag *dg = diag_src[mo.cst];
        if (!dg) return false;
        int gb[kMaxGroup];
        uint64_t gm = 0;
        for (int m = 0; m < sw.r; ++m) {
            gb[m] = __builtin_ctzll(glob_of_local(tp, sw.gbit[m]));
            gm |= 1ull << gb[m];
        }
        std::vector<std::vector<std::pair<int, double>>> cpl(sw.r);
        for (auto &kv : dg->pairs) {
            const int b0 = kv.first.first, b1 = kv.first.second;
            const bool i0 = (gm >> b0) & 1, i1 = (gm >> b1) & 1;
            if (i0 == i1) continue;
            const int gbit = i0 ? b0 : b1, other = i0 ? b1 : b0;
            for (int m = 0; m < sw.r; ++m)
                if (gb[m] == gbit) cpl[m].push_back({other, kv.second});
        }
        for (int m = 0; m < sw.r; ++m)
            if ((int)cpl[m].size() > kMaxCouple) return false;
        const int qoff = (int)cst.size();
        for (int j = 0; j < (1 << sw.r); ++j) {
            double ph = 0.0;
            for (int m = 0; m < sw.r; ++m) {
                if (!((j >> m) & 1)) continue;
                auto it = dg->a.find(gb[m]);
                if (it != dg->a.end()) ph += it->second;
                for (int m2 = m + 1; m2 < sw.r; ++m2) {
                    if (!((j >> m2) & 1)) continue;
                    auto pt = dg->pairs.find({std::min(gb[m], gb[m2]), std::max(gb[m], gb[m2])});
                    if (pt != dg->pairs.end()) ph += pt->second;
                }
            }
            cst.push_back(cexp_f(ph));
        }
        const int coff = (int)cst.size();
        uint64_t counts = 0;
        for (int m = 0; m < sw.r; ++m) {
            for (int e = 0; e < kMaxCouple; ++e) {
                float2 idx{0.f, 0.f}, w{1.f, 0.f};
                if (e < (int)cpl[m].size()) {
                    const int b = cpl[m][e].first;
                    std::memcpy(&idx.x, &b, 4);
                    w = cexp_f(cpl[m][e].second);
                }
                cst.push_back(idx);
                cst.push_back(w);
            }
            counts |= (uint64_t)cpl[m].size() << (6 * m);
        }
        mo.kind = MK_DIAGQ;
        mo.p = qoff;
        mo.lo = coff;
        mo.cmask = counts;
        mo.cval = 0;
        return true;
    }
    void finalize() {
        flush_pending();
        close_sweep();
        std::vector<double> sw_scale(tp.n_sweeps, 1.0);
        // convert tile-local bit references to group indices, fill QFT
        // tables, fold butterfly normalisations, mark diagonal factors that
        // depend on the group bits
        for (int s = 0; s < tp.n_sweeps; ++s) {
            Sweep &sw = tp.sweeps[s];
            uint64_t ggl = 0;
            for (int m = 0; m < sw.r; ++m) ggl |= glob_of_local(tp, sw.gbit[m]);
            int n_butterfly = 0;
            double rot_scale = 1.0;   // product of the factors c of the sweep's rotations
            for (int i = sw.op_begin; i < sw.op_end; ++i) {
                MicroOp &mo = tp.micro[i];
                if (mo.kind == MK_H || mo.kind == MK_QFT) n_butterfly++;
                if (mo.kind == MK_ROT) {
                    double c;
                    std::memcpy(&c, &mo.cval, sizeof c);
                    rot_scale *= c;
                    mo.cval = 0;
                }
                if (mo.kind == MK_DIAGC) {
                    if (!to_diagc(mo, sw, *count_src[mo.cst])) count_failed = true;
                    continue;
                }
                if (mo.kind == MK_DIAG) {
                    const DiagDesc &d = tp.diags[mo.cst];
                    uint32_t ds = 0, dg = 0;
                    for (int k = 0; k < d.n_slices; ++k) {
                        uint64_t win = (((1ull << d.slice_w[k]) - 1) << d.slice_lo[k]);
                        if (win & ggl) ds |= 1u << k;
                    }
                    for (int k = 0; k < d.n_groups; ++k) {
                        uint64_t bits = d.grp_mask[k] | (d.grp_mask[k] << d.grp_d[k]);
                        if (bits & ggl) dg |= 1u << k;
                    }
                    mo.a = (int)ds;
                    mo.b = (int)dg;
                    const int cap = dprec ? kMaxConstDense : kMaxConst;
                    if ((dg != 0 || __builtin_popcount(ds) > 2) &&
                        (int)cst.size() + (1 << sw.r) + 2 * kMaxCouple * sw.r <= cap)
                        to_diagq(mo, sw);
                    continue;
                }
                int ga = -1, gb = -1;
                for (int j = 0; j < sw.r; ++j) {
                    if (sw.gbit[j] == mo.a) ga = j;
                    if (mo.kind == MK_U2 && sw.gbit[j] == mo.b) gb = j;
                }
                mo.a = ga;
                if (mo.kind == MK_U2) mo.b = gb;
                if (mo.kind == MK_QFT) {
                    uint64_t M = (mo.p > mo.lo) ? (((1ull << mo.p) - 1) & ~((1ull << mo.lo) - 1)) : 0;
                    for (int jj = 0; jj < (1 << R); ++jj) {
                        uint64_t u = 0;
                        for (int m = 0; m < sw.r; ++m)
                            if ((jj >> m) & 1) u |= glob_of_local(tp, sw.gbit[m]);
                        u &= M;
                        double ph = kPi * std::ldexp((double)u, -mo.p);
                        cst[mo.cst + jj] = cexp_f(ph);
                    }
                }
            }
            sw_scale[s] = std::pow(kSqrtHalf, (double)n_butterfly) * rot_scale;
        }
        // The sweeps' scale factors commute with every op, so the pass applies
        // their product once: folded into its first count table when it has one
        // (the table's entries are multiplied in FP64 and rounded once), else
        // on its last sweep.
        // (Kept per sweep when the unscaled values could leave FP32's range:
        // any partial product outside [2^-40, 2^40].)
        double total = 1.0;
        bool foldable = true;
        int last = -1;
        for (int s = 0; s < tp.n_sweeps; ++s) {
            total *= sw_scale[s];
            if (!(total >= 0x1p-40 && total <= 0x1p40)) foldable = false;
            if (!tp.sweeps[s].dense) last = s;
        }
        if (foldable && last >= 0) {
            for (int s = 0; s < tp.n_sweeps; ++s) tp.sweeps[s].scale = 1.f;
            if (total != 1.0) {
                if (!count_luts.empty()) {
                    const auto &lt = count_luts.front();
                    for (int e = 0; e < lt.second; ++e) {
                        float2 &v = cst[lt.first + e];
                        v = float2{(float)((double)v.x * total), (float)((double)v.y * total)};
                    }
                } else {
                    tp.sweeps[last].scale = (float)total;
                }
            }
        } else {
            for (int s = 0; s < tp.n_sweeps; ++s) tp.sweeps[s].scale = (float)sw_scale[s];
        }
        merge_layers();
        tp.n_const = (int)cst.size();
    }
    // Merge runs of consecutive micro-ops that act on distinct group bits and
    // commute (same 2x2 family, no controls) into one layer op, and runs of
    // QFT stages in descending bit order into one QFT layer: the kernel then
    // runs them as straight-line code with one dispatch.
    void merge_layers() {
        std::vector<MicroOp> out;
        for (int s = 0; s < tp.n_sweeps; ++s) {
            Sweep &sw = tp.sweeps[s];
            const int begin = (int)out.size();
            int i = sw.op_begin;
            while (i < sw.op_end) {
                const MicroOp &m0 = tp.micro[i];
                auto layer_kind = [&](const MicroOp &m) {
                    if (m.cmask) return -1;
                    if (m.kind == MK_RXC || m.kind == MK_U1R || m.kind == MK_U1 || m.kind == MK_H || m.kind == MK_ROT)
                        return (int)m.kind;
                    return -1;
                };
                const int lk = layer_kind(m0);
                if (lk >= 0) {
                    uint32_t mask = 0;
                    int j = i;
                    while (j < sw.op_end && layer_kind(tp.micro[j]) == lk && !((mask >> tp.micro[j].a) & 1)) {
                        mask |= 1u << tp.micro[j].a;
                        ++j;
                    }
                    // a layer of two or more 2x2 unitaries that ends its sweep, or any
                    // that is the whole sweep (the kernel's straight-line program),
                    // becomes one MK_ZYZ op on all R group bits (identity on the others):
                    // phases, rotations, phases (unitary matrices only: the
                    // factorisation assumes it), the sweep's scale folded into the
                    // output phases.  It is last so that the kernel can undo the
                    // exchanged pairs of cotangent-form rotations at the store.
                    if (lk == MK_U1 && (j - i >= 2 || i == sw.op_begin) && j == sw.op_end && sw.r == R && !sw.dense) {
                        std::vector<std::array<cd, 4>> mats(R, std::array<cd, 4>{cd(1, 0), cd(0, 0), cd(0, 0), cd(1, 0)});
                        bool unitary = true;
                        for (int k = i; k < j; ++k) {
                            const auto &u = u1_fp64[tp.micro[k].p];
                            mats[tp.micro[k].a] = u;
                            // U^H U = I to 1e-9
                            const cd g00 = std::conj(u[0]) * u[0] + std::conj(u[2]) * u[2];
                            const cd g11 = std::conj(u[1]) * u[1] + std::conj(u[3]) * u[3];
                            const cd g01 = std::conj(u[0]) * u[1] + std::conj(u[2]) * u[3];
                            if (std::abs(g00 - 1.0) > 1e-9 || std::abs(g11 - 1.0) > 1e-9 || std::abs(g01) > 1e-9)
                                unitary = false;
                        }
                        const int P = 1 << R;
                        if (unitary && (int)cst.size() + 2 * P + 2 * R + 1 <= kMaxConst) {
                            MicroOp Z;
                            std::memset(&Z, 0, sizeof Z);
                            Z.kind = MK_ZYZ;
                            Z.cst = (int)cst.size();
                            std::vector<cd> pin(P, cd(1, 0)), pout(P, cd(1, 0));
                            std::vector<float2> kk;
                            int form = 0;
                            for (int m = 0; m < R; ++m) {
                                const auto &u = mats[m];
                                double c = std::abs(u[0]), sn = std::abs(u[2]);
                                const double nr = std::hypot(c, sn);
                                c /= nr;
                                sn /= nr;
                                double a, b, d;   // U = diag(e^{ia}, e^{ib}) [[c, -s], [s, c]] diag(1, e^{id})
                                if (sn == 0.0) {
                                    a = std::arg(u[0]);
                                    b = std::arg(u[3]);
                                    d = 0.0;
                                } else if (c == 0.0) {
                                    a = 0.0;
                                    b = std::arg(u[2]);
                                    d = std::arg(-u[1]);
                                } else {
                                    a = std::arg(u[0]);
                                    b = std::arg(u[2]);
                                    d = std::arg(-u[1]) - a;
                                }
                                const bool cot = sn > c;
                                double k0, k1, f;
                                if (!cot) {
                                    k0 = -sn / c;
                                    k1 = sn / c;
                                    f = c;
                                } else {
                                    // cotangent form: the kernel computes the pair
                                    // (a0 + (c/s) a1, a1 - (c/s) a0), the two outputs exchanged
                                    k0 = c / sn;
                                    k1 = -c / sn;
                                    f = sn;
                                    form |= 1 << m;
                                }
                                kk.push_back(float2{(float)k0, (float)k0});
                                kk.push_back(float2{(float)k1, (float)k1});
                                const cd e0 = std::polar(f * (cot ? -1.0 : 1.0), a), e1 = std::polar(f, b);
                                const cd ed = std::polar(1.0, d);
                                for (int jj = 0; jj < P; ++jj) {
                                    pout[jj] *= ((jj >> m) & 1) ? e1 : e0;
                                    if ((jj >> m) & 1) pin[jj] *= ed;
                                }
                            }
                            const double scl = sw.scale;
                            sw.scale = 1.f;
                            for (int jj = 0; jj < P; ++jj) cst.push_back(float2{(float)pin[jj].real(), (float)pin[jj].imag()});
                            // output phases in the order of the exchanged results: entry i
                            // multiplies the value that is stored as element i ^ form
                            for (int jj = 0; jj < P; ++jj)
                                cst.push_back(float2{(float)(pout[jj ^ form].real() * scl), (float)(pout[jj ^ form].imag() * scl)});
                            cst.insert(cst.end(), kk.begin(), kk.end());
                            float fm;
                            std::memcpy(&fm, &form, sizeof fm);
                            cst.push_back(float2{fm, 0.f});
                            out.push_back(Z);
                            i = j;
                            continue;
                        }
                    }
                    const int stride = lk == MK_RXC ? 1 : lk == MK_U1R ? 4 : lk == MK_U1 ? 4 : lk == MK_ROT ? 2 : 0;
                    // a lone rotation becomes a one-bit layer too (see the padding below)
                    if (j - i >= (lk == MK_ROT ? 1 : 2) && (int)cst.size() + R * stride + 1 <= kMaxConst) {
                        MicroOp L;
                        std::memset(&L, 0, sizeof L);
                        L.kind = MK_LAYER;
                        L.a = lk;
                        L.b = (int)mask;
                        if (lk == MK_U1R && (cst.size() & 1)) cst.push_back(float2{0.f, 0.f});
                        L.cst = (int)cst.size();
                        for (int m = 0; m < R * stride; ++m) cst.push_back(float2{0.f, 0.f});
                        for (int k = i; k < j; ++k) {
                            const MicroOp &mk = tp.micro[k];
                            for (int e = 0; e < stride; ++e) cst[L.cst + mk.a * stride + e] = cst[mk.cst + e];
                        }
                        out.push_back(L);
                        i = j;
                        continue;
                    }
                }
                if (m0.kind == MK_QFT && m0.lo == 0) {
                    uint32_t mask = 0;
                    int j = i, last = 1 << 30;
                    while (j < sw.op_end && tp.micro[j].kind == MK_QFT && tp.micro[j].lo == 0 &&
                           tp.micro[j].a < last) {
                        last = tp.micro[j].a;
                        mask |= 1u << last;
                        ++j;
                    }
                    if (j - i >= 2 && (int)cst.size() + R * (1 << R) <= kMaxConst) {
                        MicroOp L;
                        std::memset(&L, 0, sizeof L);
                        L.kind = MK_QFTL;
                        L.b = (int)mask;
                        L.cst = (int)cst.size();
                        uint64_t pp = 0;
                        for (int m = 0; m < R * (1 << R); ++m) cst.push_back(float2{1.f, 0.f});
                        for (int k = i; k < j; ++k) {
                            const MicroOp &mk = tp.micro[k];
                            pp |= (uint64_t)(mk.p & 63) << (6 * mk.a);
                            for (int e = 0; e < (1 << R); ++e) cst[L.cst + mk.a * (1 << R) + e] = cst[mk.cst + e];
                        }
                        L.cmask = pp;
                        out.push_back(L);
                        i = j;
                        continue;
                    }
                }
                out.push_back(m0);
                ++i;
            }
            sw.op_begin = begin;
            sw.op_end = (int)out.size();
            // A sweep of rotation layers and count-table diagonals in one of the
            // kernel's rotation programs (layer; diagonal, layer; layer,
            // diagonal; layer, diagonal, layer) gets its layers on all R group
            // bits: the constants of a bit without a rotation are t = 0 (set
            // above), an exact identity, and the sweep runs as straight-line code.
            auto rot_layer = [&](const MicroOp &m) { return m.kind == MK_LAYER && m.a == MK_ROT; };
            auto diagc = [&](const MicroOp &m) { return m.kind == MK_DIAGC; };
            const int n_ops = sw.op_end - sw.op_begin;
            const MicroOp *o = out.data() + begin;
            const bool program = sw.r == R && ((n_ops == 1 && rot_layer(o[0])) ||
                                               (n_ops == 2 && diagc(o[0]) && rot_layer(o[1])) ||
                                               (n_ops == 2 && rot_layer(o[0]) && diagc(o[1])) ||
                                               (n_ops == 3 && rot_layer(o[0]) && diagc(o[1]) && rot_layer(o[2])));
            // (the layer's own bits stay in `lo`: the kernel skips the padded ones
            // when they are the lowest three or four group positions, or those
            // above position 0)
            if (program)
                for (int k = begin; k < sw.op_end; ++k)
                    if (rot_layer(out[k])) {
                        out[k].lo = out[k].b;
                        out[k].b = (1 << R) - 1;
                    }
        }
        tp.n_micro = (int)out.size();
        for (int k = 0; k < tp.n_micro; ++k) tp.micro[k] = out[k];
    }
};
}  // namespace

static void build_perm_or_gather(int n, const FOp &f, HostPass &hp) {
    bool perm = true;
    for (int i = 0; i < n; ++i)
        if (popc64(f.rows[i]) != 1) perm = false;
    if (perm) {
        hp.type = HostPass::PERM;
        std::memset(&hp.perm, 0, sizeof hp.perm);
        hp.perm.n = n;
        hp.perm.L = std::min(5, n);
        for (int i = 0; i < n; ++i) hp.perm.out_pos[__builtin_ctzll(f.rows[i])] = i;
        hp.perm.xor_mask = f.c;
        return;
    }
    // inverse of the forward matrix over GF(2): columns of M^-1 via Gauss-Jordan
    hp.type = HostPass::GATHER;
    std::memset(&hp.gather, 0, sizeof hp.gather);
    hp.gather.n = n;
    std::vector<uint64_t> A(f.rows.begin(), f.rows.end());   // row i: coefficients of x
    std::vector<uint64_t> Inv(n);
    for (int i = 0; i < n; ++i) Inv[i] = 1ull << i;
    for (int col = 0; col < n; ++col) {
        int piv = -1;
        for (int r = col; r < n; ++r)
            if ((A[r] >> col) & 1) {
                piv = r;
                break;
            }
        std::swap(A[col], A[piv]);
        std::swap(Inv[col], Inv[piv]);
        for (int r = 0; r < n; ++r)
            if (r != col && ((A[r] >> col) & 1)) {
                A[r] ^= A[col];
                Inv[r] ^= Inv[col];
            }
    }
    // Inv rows: x_i = parity(Inv[i] & (y ^ c)); column j of M^-1 = bits i with Inv[i] bit j
    auto apply_inv = [&](uint64_t v) {
        uint64_t x = 0;
        for (int i = 0; i < n; ++i)
            if (popc64(Inv[i] & v) & 1) x |= 1ull << i;
        return x;
    };
    hp.gather.c = apply_inv(f.c);
    hp.gather.n_slices = (n + 7) / 8;
    for (int k = 0; k < hp.gather.n_slices; ++k)
        for (int bte = 0; bte < 256; ++bte) {
            uint64_t v = (uint64_t)bte << (8 * k);
            if (8 * k + 8 > n) v &= (n >= 64 ? ~0ull : ((1ull << n) - 1));
            hp.gather.tab[k][bte] = apply_inv(v);
        }
}

static qs_status build_fused_plan_cfg(int n, int batch, const std::vector<FOp> &detected, int n_gates,
                                      const qs_opts &o, Plan &plan, std::string &err);

// Tile shape actually used for T tile bits with L low bits: T <= 13 (two
// 2^13-amplitude buffers fill the 227 KB of shared memory) and <= n, L in
// [1, T]; a tile that does not cover the whole state keeps at least two
// high-bit slots (so that a 4x4 op on any two high bits fits a pass): T >= 3
// and L <= T - 2.
static void clamp_tile_shape(int n, int &T, int &L) {
    if (T > 13) T = 13;
    if (T > n) T = n;
    if (T < n && T < 3) T = std::min(n, 3);
    if (L > T) L = T;
    if (T < n && L > T - 2) L = T - 2;
    if (L < 1) L = 1;
}

// Default tile shape: 12-bit tiles with 4-bit register groups (two CTAs per
// SM hide each other's copy latency) unless they need more HBM passes than
// 13-bit tiles with 5-bit groups.
qs_status build_fused_plan(int n, int batch, const std::vector<RGate> &gates, const qs_opts &o, Plan &plan,
                           std::string &err, bool item_plan) {
    struct ItemPlanScope {   // the pass builder reads the flag on this thread
        explicit ItemPlanScope(bool v) { t_item_plan = v; }
        ~ItemPlanScope() { t_item_plan = false; }
    } item_scope(item_plan);
    if (o.dense_prec < QS_DENSE_OFF || o.dense_prec > QS_DENSE_BF16) {
        err = "dense_prec must be one of QS_DENSE_OFF / FP32 / TF32X3 / BF16";
        return QS_ERR_INVALID_ARG;
    }
    if (o.block_qubits != 0 && (o.block_qubits < 3 || o.block_qubits > 5)) {
        err = "block_qubits must be 0 (default 5) or in [3, 5]";
        return QS_ERR_INVALID_ARG;
    }
    std::vector<FOp> detected;
    detect(n, gates, detected);
    if (o.dense_prec != QS_DENSE_OFF && n >= 5) {
        // dense blocks: cells of <= k bits laid out so that the cells of one
        // tile window (the low bits plus T - L high bits) share a pass
        qs_opts c = o;
        const int k = o.block_qubits > 0 ? o.block_qubits : 5;
        if (c.tile_qubits <= 0) c.tile_qubits = 13;
        c.tile_qubits = std::max(5, std::min(c.tile_qubits, std::min(n, 13)));
        if (c.low_qubits <= 0) c.low_qubits = 4;
        // a block may hold k high bits (its ops' bits, controls included, need
        // not share a cell): a tile that does not cover the state keeps k
        // high-bit slots
        if (c.tile_qubits < n) {
            c.tile_qubits = std::max(c.tile_qubits, std::min(n, k + 1));
            if (c.tile_qubits < n) c.low_qubits = std::max(1, std::min(c.low_qubits, c.tile_qubits - k));
        }
        clamp_tile_shape(n, c.tile_qubits, c.low_qubits);
        c.group_qubits = 5;   // dense passes run in the 5-bit-group kernel
        int cell_of[64];
        for (int b = 0; b < 64; ++b) cell_of[b] = 63;
        dense_cells(n, c.tile_qubits, c.low_qubits, k, cell_of);
        std::vector<FOp> blocks;
        fuse_dense(n, k, cell_of, detected, blocks);
        return build_fused_plan_cfg(n, batch, blocks, (int)gates.size(), c, plan, err);
    }
    qs_opts od = o;
    od.dense_prec = QS_DENSE_OFF;
    if (o.tile_qubits > 0 || o.group_qubits > 0 || n < 13)
        return build_fused_plan_cfg(n, batch, detected, (int)gates.size(), od, plan, err);
    bool has_qft = false;
    for (const FOp &f : detected)
        if (f.kind == F_QFT) has_qft = true;
    // candidates in order of measured per-pass speed for general passes (the
    // first wins a tie in HBM passes).  13-bit tiles with 5-bit groups win a
    // tie for QFT stages (25q QFT 0.60 against 0.73 ms) and for layer plans:
    // every pass a tensor copy of uncontrolled one-qubit layers and diagonals,
    // none evaluated factor by factor (the warp-specialised kernel's rotation,
    // U(2) and straight-line layer sweeps; 25q Trotter, Heisenberg, ansatz,
    // QCBM and QAOA circuits 9-31% faster than with 12-bit tiles and 4-bit
    // groups).  Otherwise the 4-bit groups stay ahead (25q random circuit 11.1
    // against 18.6 ms, long-range Ising 7.9 against 14.8 ms, quantum walk 13.4
    // against 15.5 ms).
    const int cfg[3][2] = {{12, 4}, {13, 4}, {13, 5}};
    // the third candidate can win only for QFT stages or a layer plan: not
    // built when an op is controlled or acts on two bits non-diagonally
    bool may_layer = true;
    for (const FOp &f : detected)
        if ((f.kind == F_U1 && f.cmask != 0) || f.kind == F_U2 || f.kind == F_DENSE) may_layer = false;
    const int n_cand = (has_qft || may_layer) ? 3 : 2;
    Plan cand[3];
    for (int i = 0; i < n_cand; ++i) {
        qs_opts c = od;
        c.tile_qubits = cfg[i][0];
        c.group_qubits = cfg[i][1];
        qs_status s = build_fused_plan_cfg(n, batch, detected, (int)gates.size(), c, cand[i], err);
        if (s != QS_OK) return s;
    }
    int best = 0;
    for (int i = 1; i < 2; ++i)
        if (cand[i].passes.size() < cand[best].passes.size()) best = i;
    bool layer_plan = n_cand == 3;
    for (const HostPass &hp : cand[2].passes)
        if (hp.type == HostPass::TILE &&
            (!hp.tma.ok || !layer_only(hp.tile) || general_diags(hp.tile) > 0 ||
             std::any_of(hp.tile.micro, hp.tile.micro + hp.tile.n_micro,
                         [](const MicroOp &m) { return m.kind == MK_U1 && m.cmask != 0; })))
            layer_plan = false;
    if (n_cand == 3 && (has_qft || layer_plan) && cand[2].passes.size() <= cand[best].passes.size()) best = 2;
    plan = std::move(cand[best]);
    return QS_OK;
}

// Runs of uncontrolled one-qubit ops on distinct bits commute; the scheduler
// takes ops into a pass in stream order, so a run's order decides which bits
// share a tile.  Each run is ordered: the L tile-resident low bits, then the
// a = (T - L) - b bits right above them, then the top b = (T - L) / 3 bits,
// then the rest ascending.  The first pass of a layer then holds one long
// contiguous block (rows of 2^(L+a) amplitudes) and a few top bits, and the
// others contiguous middle blocks; a tile of top bits only (rows of 2^L
// amplitudes, each in another far-apart page) streams ~15% slower through the
// TMA.  (30q Trotter steps: 7.71 -> 7.30 ms with the same 201 passes.)  The
// order is a second candidate plan (build_fused_plan_cfg keeps the one with
// the lower locality cost): it can also fragment passes past the 5 tensor
// dimensions of one copy (Heisenberg chains, where each layer's bits follow
// the conjugated pair terms).
// Only runs of real 2x2 ops (rotations, Hadamards) are reordered: with complex
// layers the first pass of each layer also holds the random-angle diagonal
// that precedes it, and with the low bits in that sweep's group its slice-table
// lookups vary across a warp's lanes (28q layered suite: 79 -> 88 ms).
static void order_layer_runs(int n, int T, int L, std::vector<FOp> &ops) {
    const int b = std::max(0, (T - L) / 3), a = std::max(0, (T - L) - b);
    std::vector<int> rank(n, 0);
    int r = 0;
    for (int q = 0; q < L && q < n; ++q) rank[q] = r++;
    for (int q = L; q < L + a && q < n; ++q) rank[q] = r++;
    for (int q = n - 1; q >= n - b && q >= L + a; --q) rank[q] = r++;
    for (int q = L + a; q < n - b; ++q) rank[q] = r++;
    auto one_q = [&](const FOp &f) {
        return f.kind == F_U1 && f.cmask == 0 && f.t0 >= 0 && f.t0 < n && f.m[0].imag() == 0.0 &&
               f.m[1].imag() == 0.0 && f.m[2].imag() == 0.0 && f.m[3].imag() == 0.0;
    };
    size_t i = 0;
    while (i < ops.size()) {
        if (!one_q(ops[i])) {
            ++i;
            continue;
        }
        size_t j = i;
        uint64_t seen = 0;
        while (j < ops.size() && one_q(ops[j]) && !((seen >> ops[j].t0) & 1)) {
            seen |= 1ull << ops[j].t0;
            ++j;
        }
        std::stable_sort(ops.begin() + (long)i, ops.begin() + (long)j,
                         [&](const FOp &x, const FOp &y) { return rank[x.t0] < rank[y.t0]; });
        i = j;
    }
}

static qs_status build_fused_plan_once(int n, int batch, const std::vector<FOp> &detected, int n_gates,
                                      const qs_opts &o, bool order, Plan &plan, std::string &err);

// Locality cost of a plan's tile passes.  A tile with many bits among the
// 2 MB-page bits (index bit 18 and up, for 8-byte amplitudes) whose rows also
// reach the top of a state of 1 GB and more streams slowest through the TMA
// (30q, one two-sweep pass: tile bits 20-28 3.44 ms, 18-26 3.10 ms, 4-8 with
// 26-29 2.87 ms): such a pass costs its count of page bits.  A pass copied
// row by row (more than 5 tensor dimensions) is counted apart.
static void locality_cost(const Plan &p, int &row_copies, int &spread) {
    row_copies = 0;
    spread = 0;
    for (const HostPass &hp : p.passes) {
        if (hp.type != HostPass::TILE) continue;
        if (!hp.tma.ok) ++row_copies;
        const TilePass &tp = hp.tile;
        int page_bits = 0, top = -1;
        for (int k = 0; k < tp.H; ++k) {
            if (tp.hb[k] >= 18) ++page_bits;
            top = std::max(top, tp.hb[k]);
        }
        if (page_bits >= 6 && top >= 27) spread += page_bits;
    }
}

// Plan with the scheduler's stream order and, for states of 2^28 amplitudes
// and more, with the layer order below as well; the latter is kept when it
// needs no more HBM passes and no more row-copy passes and has the lower
// locality cost.
static qs_status build_fused_plan_cfg(int n, int batch, const std::vector<FOp> &detected, int n_gates,
                                      const qs_opts &o, Plan &plan, std::string &err) {
    qs_status s = build_fused_plan_once(n, batch, detected, n_gates, o, false, plan, err);
    if (s != QS_OK || n < 28) return s;
    Plan alt;
    std::string err2;
    if (build_fused_plan_once(n, batch, detected, n_gates, o, true, alt, err2) != QS_OK) return s;
    int rc0, sp0, rc1, sp1;
    locality_cost(plan, rc0, sp0);
    locality_cost(alt, rc1, sp1);
    if (alt.passes.size() <= plan.passes.size() && rc1 <= rc0 && sp1 < sp0) plan = std::move(alt);
    return s;
}

static qs_status build_fused_plan_once(int n, int batch, const std::vector<FOp> &detected, int n_gates,
                                      const qs_opts &o, bool order, Plan &plan, std::string &err) {
    plan = Plan();
    plan.n = n;
    plan.mode = QS_MODE_FUSED;
    plan.n_gates = n_gates;
    std::vector<FOp> ops(detected);

    int T = o.tile_qubits > 0 ? o.tile_qubits : 13;
    int L = o.low_qubits > 0 ? o.low_qubits : 4;
    clamp_tile_shape(n, T, L);
    int R = o.group_qubits > 0 ? std::min(o.group_qubits, kMaxGroup) : kMaxGroup;
    R = std::min(R, T);
    const int dprec = o.dense_prec;
    const int max_const = dprec ? kMaxConstDense : kMaxConst;

    // split oversized diagonals; pre-plan each diagonal's tables
    std::vector<FOp> ops2;
    for (auto &f : ops) {
        if (f.kind != F_DIAG) {
            ops2.push_back(f);
            continue;
        }
        CountForm cf0;
        if (count_form(f.diag, cf0)) {   // one count lookup, whatever its size
            ops2.push_back(f);
            continue;
        }
        DiagPlan dp;
        plan_diag(n, f.diag, dp);
        if ((int)dp.descs.size() <= kMaxDiag && (int)diag_const_size(dp) <= kMaxConst / 2) {
            ops2.push_back(f);
            continue;
        }
        // split pairs into chunks (diagonal factors commute)
        FOp base = f;
        base.diag.pairs.clear();
        std::vector<std::pair<std::pair<int, int>, double>> prs(f.diag.pairs.begin(), f.diag.pairs.end());
        const size_t chunk = 16;
        ops2.push_back(base);
        for (size_t i = 0; i < prs.size(); i += chunk) {
            FOp g;
            g.kind = F_DIAG;
            g.n_gates = 0;
            for (size_t k = i; k < std::min(prs.size(), i + chunk); ++k) g.diag.pairs[prs[k].first] = prs[k].second;
            ops2.push_back(g);
        }
    }
    ops.swap(ops2);
    if (order) order_layer_runs(n, T, L, ops);
    for (FOp &f : ops) f.cache_masks();
    std::vector<DiagPlan> dplans(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        if (ops[i].kind != F_DIAG) continue;
        CountForm cf;
        if (count_form(ops[i].diag, cf)) {
            dplans[i].count = true;
            dplans[i].count_const = count_const_size(cf, R);
        } else {
            plan_diag(n, ops[i].diag, dplans[i]);
        }
    }

    // the ops still to schedule are rem[head..]: a pass moves `head` past what
    // it placed (O(ops scanned) per pass, not O(ops left))
    std::vector<int> rem(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) rem[i] = (int)i;
    size_t head = 0;
    std::vector<char> placed(ops.size(), 0);
    const uint64_t lowmask = (L >= 64) ? ~0ull : ((1ull << L) - 1);
    const int kLookahead = 4096, kMaxDeferred = 96;

    while (head < rem.size()) {
        const FOp &f0 = ops[rem[head]];
        if (f0.kind == F_GF2) {
            HostPass hp;
            build_perm_or_gather(n, f0, hp);
            hp.note = hp.type == HostPass::PERM ? "perm" : "gather";
            plan.passes.push_back(hp);
            ++head;
            continue;
        }
        uint64_t S = lowmask;
        int slots = T - L;
        std::vector<int> taken, deferred;
        size_t j = 0;
        int c_const = 0, c_micro = 0, c_diag = 0;
        int sim_sweeps = 0;          // mirrors PassBuilder::need_bits grouping
        uint64_t sim_group = 0;
        bool sim_open = false;
        for (; head + j < rem.size() && (int)j < kLookahead; ++j) {
            const FOp &f = ops[rem[head + j]];
            if (f.kind == F_GF2) break;
            bool ok = true;
            for (int d : deferred)
                if (!commute(f, ops[d])) {
                    ok = false;
                    break;
                }
            if (ok) {
                uint64_t need = f.cN & ~S;
                OpCost c = op_cost(n, f, R, f.kind == F_DIAG ? &dplans[rem[head + j]] : nullptr, dprec);
                uint64_t nb = f.cN;
                int ns = sim_sweeps;
                uint64_t ng = sim_group;
                bool no = sim_open;
                if (f.kind == F_DENSE) {   // a sweep of its own
                    ns++;
                    ng = 0;
                    no = false;
                } else if (nb) {
                    if (no && popc64(ng | nb) <= R) {
                        ng |= nb;
                    } else {
                        ns++;
                        ng = nb;
                        no = true;
                    }
                } else if (!no) {
                    ns++;
                    ng = 0;
                    no = true;
                }
                bool fits = popc64(need) <= slots - (popc64(S) - L) && c_const + c.n_const <= max_const &&
                            c_micro + c.n_micro <= kMaxMicro - 8 && c_diag + c.n_diag <= kMaxDiag &&
                            ns <= kMaxSweeps - 1;
                if (fits) {
                    sim_sweeps = ns;
                    sim_group = ng;
                    sim_open = no;
                    S |= need;
                    c_const += c.n_const;
                    c_micro += c.n_micro;
                    c_diag += c.n_diag;
                    taken.push_back(rem[head + j]);
                    continue;
                }
            }
            deferred.push_back(rem[head + j]);
            if ((int)deferred.size() >= kMaxDeferred) {
                ++j;
                break;
            }
        }
        if (taken.empty()) {
            err = "scheduler could not place an op (internal)";
            return QS_ERR_INTERNAL;
        }
        S = pad_tile_bits(n, L, T, S, batch);
        // the sweep and constant estimates above can fall short of what the
        // builder makes: ops past its sweep / micro-op limit stay in the
        // queue (below), and a pass whose constants come out over the budget
        // (the optional factored diagonals of finalize and the count tables
        // share it) is rebuilt from a shorter prefix of its ops
        size_t limit = taken.size();
        std::unique_ptr<PassBuilder> pbp;
        for (;;) {
            pbp.reset(new PassBuilder(n, L, T, R, S, batch, dprec));
            size_t added = 0;
            for (size_t k = 0; k < limit; ++k) {
                const int id = taken[k];
                pbp->add(ops[id], ops[id].kind == F_DIAG ? &dplans[id] : nullptr);
                ++added;
                // held-back layer ops may each still open a sweep
                if (pbp->tp.n_sweeps + pbp->pending_ops() >= kMaxSweeps - 1 ||
                    pbp->tp.n_micro + pbp->pending_ops() >= kMaxMicro - 16)
                    break;
            }
            pbp->finalize();
            if (pbp->tp.n_const <= max_const) {
                for (size_t k = 0; k < added; ++k) placed[taken[k]] = 1;
                break;
            }
            if (added <= 1) {
                // one op alone needs more constants than a pass holds: the
                // kernel sizes its shared memory from them, so refuse here
                err = "an op needs " + std::to_string(pbp->tp.n_const) + " pass constants, more than the " +
                      std::to_string(max_const) + " a tile pass holds (op kind " + std::to_string(ops[taken[0]].kind) +
                      ")";
                return QS_ERR_UNSUPPORTED;
            }
            limit = added - std::max<size_t>(1, added / 8);
        }
        PassBuilder &pb = *pbp;
        if (pb.count_failed) {
            err = "count-table diagonal could not be placed (internal)";
            return QS_ERR_INTERNAL;
        }
        pb.hp.note = "tile";
        plan.passes.push_back(pb.hp);
        // everything scanned but not placed, in stream order: the deferred ops
        // and any taken op past the builder's limit (each placed op commutes
        // with every deferred op before it, so the order stays exact)
        std::vector<int> carry;
        for (size_t k = 0; k < j; ++k)
            if (!placed[rem[head + k]]) carry.push_back(rem[head + k]);
        for (int id : taken) placed[id] = 0;
        head += j - carry.size();
        std::copy(carry.begin(), carry.end(), rem.begin() + head);
    }
    return QS_OK;
}

// ---------------------------------------------------------------------------
// per-gate plan: the structured pure path (Sec. 3.2.2; Sec. 4.1 dispatch)
// ---------------------------------------------------------------------------
qs_status build_pergate_plan(int n, const std::vector<RGate> &gates, Plan &plan, std::string &err) {
    (void)err;
    plan = Plan();
    plan.n = n;
    plan.mode = QS_MODE_PERGATE;
    plan.n_gates = (int)gates.size();
    for (const RGate &g : gates) {
        PgOp op;
        std::memset(&op, 0, sizeof op);
        auto setm = [&](const cd *M, int cnt) {
            for (int e = 0; e < cnt; ++e) {
                op.m[e].x = (float)M[e].real();
                op.m[e].y = (float)M[e].imag();
            }
        };
        cd M[64];
        gate_matrix(g, M);
        double ph[4];
        switch (g.kind) {
            case QS_I:
                continue;
            case QS_Z: case QS_S: case QS_SDG: case QS_T: case QS_TDG: case QS_P:
                op.kind = PG_PHASE;   // touch only the bit = 1 half
                op.t0 = g.b[0];
                op.cmask = op.cval = 1ull << g.b[0];
                op.nbits_phase = 0;
                diag_phases(g, ph);
                op.m[0] = cexp_f(ph[1]);
                break;
            case QS_RZ:
                op.kind = PG_PHASE;
                op.t0 = g.b[0];
                op.nbits_phase = 1;
                diag_phases(g, ph);
                op.m[0] = cexp_f(ph[0]);
                op.m[1] = cexp_f(ph[1]);
                break;
            case QS_CZ: case QS_CP:
                op.kind = PG_PHASE;   // only the |11> quarter
                op.cmask = op.cval = (1ull << g.b[0]) | (1ull << g.b[1]);
                op.nbits_phase = 0;
                diag_phases(g, ph);
                op.m[0] = cexp_f(ph[3]);
                break;
            case QS_CRZ:
                op.kind = PG_PHASE;   // control = 1 half, phase by target
                op.t0 = g.b[1];
                op.cmask = op.cval = 1ull << g.b[0];
                op.nbits_phase = 1;
                diag_phases(g, ph);
                op.m[0] = cexp_f(ph[2]);
                op.m[1] = cexp_f(ph[3]);
                break;
            case QS_RZZ:
                op.kind = PG_PHASE;
                op.t0 = g.b[0];
                op.t1 = g.b[1];
                op.nbits_phase = 2;
                diag_phases(g, ph);
                // table index = bit t0 | bit t1 << 1; ph index = x_w0*2 + x_w1
                op.m[0] = cexp_f(ph[0]);
                op.m[1] = cexp_f(ph[2]);
                op.m[2] = cexp_f(ph[1]);
                op.m[3] = cexp_f(ph[3]);
                break;
            case QS_CX: case QS_CY: case QS_CH: case QS_CRX: case QS_CRY: {
                op.kind = PG_U1;   // masked half-state update
                op.t0 = g.b[1];
                op.cmask = op.cval = 1ull << g.b[0];
                cd U[4] = {M[10], M[11], M[14], M[15]};
                setm(U, 4);
                break;
            }
            case QS_CCX: {
                op.kind = PG_U1;
                op.t0 = g.b[2];
                op.cmask = op.cval = (1ull << g.b[0]) | (1ull << g.b[1]);
                cd U[4] = {0, 1, 1, 0};
                setm(U, 4);
                break;
            }
            case QS_SWAP:
                op.kind = PG_SWAP;
                op.t0 = g.b[0];
                op.t1 = g.b[1];
                break;
            case QS_CSWAP:
                op.kind = PG_SWAP;
                op.t0 = g.b[1];
                op.t1 = g.b[2];
                op.cmask = op.cval = 1ull << g.b[0];
                break;
            case QS_ISWAP: case QS_RXX: case QS_RYY:
                op.kind = PG_U2;
                op.t0 = g.b[0];
                op.t1 = g.b[1];
                setm(M, 16);
                break;
            default:   // remaining 1q kinds: general 2x2
                op.kind = PG_U1;
                op.t0 = g.b[0];
                setm(M, 4);
        }
        plan.pg.push_back(op);
    }
    return QS_OK;
}

static bool same_tma(const TmaPlan &a, const TmaPlan &b) {   // field by field (the struct has padding)
    if (a.ok != b.ok || a.ndims != b.ndims || a.batch_dim != b.batch_dim) return false;
    for (int d = 0; d < 5; ++d)
        if (a.kind[d] != b.kind[d] || a.off[d] != b.off[d] || a.w[d] != b.w[d] || a.gdim[d] != b.gdim[d] ||
            a.gstride[d] != b.gstride[d] || a.box[d] != b.box[d])
            return false;
    return true;
}

bool merge_item_plans(std::vector<Plan> &plans, Plan &out, int batch) {
    if (plans.empty()) return false;
    const Plan &p0 = plans[0];
    if (p0.mode != QS_MODE_FUSED) return false;
    for (const Plan &p : plans) {
        if (p.mode != p0.mode || p.items != 1 || p.passes.size() != p0.passes.size()) return false;
        for (size_t i = 0; i < p.passes.size(); ++i) {
            const HostPass &a = p0.passes[i], &b = p.passes[i];
            if (a.type != b.type || a.uses_roots != b.uses_roots) return false;
            if (a.type == HostPass::TILE) {
                if (std::memcmp(&a.tile, &b.tile, sizeof(TilePass)) != 0 || a.consts.size() != b.consts.size() ||
                    !same_tma(a.tma, b.tma))
                    return false;
            } else if (a.type == HostPass::PERM) {
                if (std::memcmp(&a.perm, &b.perm, sizeof(PermPass)) != 0) return false;
            } else if (std::memcmp(&a.gather, &b.gather, sizeof(GatherPass)) != 0) {
                return false;
            }
        }
    }
    out = p0;
    out.items = (int)plans.size();
    for (size_t i = 0; i < out.passes.size(); ++i) {
        HostPass &hp = out.passes[i];
        if (hp.type != HostPass::TILE) continue;
        // the batch may need a tensor dim of its own: keep the merge only if the
        // tensor-copy path survives (the layout and swizzle assume it)
        uint64_t S = (1ull << hp.tile.L) - 1;
        for (int k = 0; k < hp.tile.H; ++k) S |= 1ull << hp.tile.hb[k];
        const TmaPlan g = tma_geometry(out.n, hp.tile.L, S, batch);
        if (g.ok != hp.tma.ok) return false;
        hp.tma = g;
        hp.consts.clear();
        for (const Plan &p : plans) hp.consts.insert(hp.consts.end(), p.passes[i].consts.begin(), p.passes[i].consts.end());
    }
    return true;
}

int Plan::hbm_passes() const {
    if (mode == QS_MODE_PERGATE) return (int)pg.size();
    return (int)passes.size();
}

// sweeps of a tile pass that the kernel runs as a specialised program: a
// rotation program (rotation layer on all group bits; count-table diagonal
// and layer in either order; layer, diagonal, layer) or a lone U(2) layer op
int program_sweeps(const TilePass &tp) {
    const int F = (1 << tp.R) - 1;
    int k = 0;
    for (int s = 0; s < tp.n_sweeps; ++s) {
        const Sweep &S = tp.sweeps[s];
        if (S.dense) continue;
        const MicroOp *o = tp.micro + S.op_begin;
        const int n = S.op_end - S.op_begin;
        auto rot = [&](int i) { return o[i].kind == MK_LAYER && o[i].a == MK_ROT && o[i].b == F; };
        auto dgc = [&](int i) { return o[i].kind == MK_DIAGC; };
        if ((n == 1 && rot(0)) || (n == 2 && dgc(0) && rot(1)) || (n == 2 && rot(0) && dgc(1)) ||
            (n == 3 && rot(0) && dgc(1) && rot(2)) || (n == 1 && o[0].kind == MK_ZYZ && S.scale == 1.f))
            ++k;
    }
    return k;
}

// sweeps whose only op is one layer on all group bits (or all but bit 0)
// that the kernel runs as straight-line code from load to store
int straight_sweeps(const TilePass &tp) {
    if (tp.R != 4 && tp.R != 5) return 0;
    const uint32_t F = (1u << tp.R) - 1;
    int k = 0;
    for (int s = 0; s < tp.n_sweeps; ++s) {
        const Sweep &S = tp.sweeps[s];
        if (S.dense || S.op_end - S.op_begin != 1) continue;
        const MicroOp &o = tp.micro[S.op_begin];
        if (o.kind != MK_LAYER || (o.a != MK_H && o.a != MK_ROT && S.scale != 1.f)) continue;
        if ((uint32_t)o.b == F || (uint32_t)o.b == (F & ~1u)) ++k;
    }
    return k;
}

// every micro-op of the pass is a one-qubit layer kind or a diagonal (the
// kernels compiled for that op set, KS_LAYER)
bool layer_only(const TilePass &tp) {
    for (int i = 0; i < tp.n_micro; ++i) {
        const int k = tp.micro[i].kind;
        if (!(k == MK_LAYER || k == MK_RXC || k == MK_U1R || k == MK_ROT || k == MK_H || k == MK_U1 ||
              k == MK_ZYZ || k == MK_DIAG || k == MK_DIAGQ || k == MK_DIAGC))
            return false;
    }
    return true;
}

// diagonal micro-ops that the kernel evaluates factor by factor per amplitude
// (tables whose indices vary with more than two slices of the group)
int general_diags(const TilePass &tp) {
    int k = 0;
    for (int i = 0; i < tp.n_micro; ++i)
        if (tp.micro[i].kind == MK_DIAG && (tp.micro[i].b != 0 || __builtin_popcount((unsigned)tp.micro[i].a) > 2))
            ++k;
    return k;
}

std::string Plan::describe() const {
    std::ostringstream os;
    if (mode == QS_MODE_PERGATE) {
        os << "PERGATE n=" << n << " gates=" << n_gates << " launches=" << pg.size() << "\n";
        return os.str();
    }
    os << "FUSED n=" << n << " gates=" << n_gates << " passes=" << passes.size() << "\n";
    for (size_t i = 0; i < passes.size(); ++i) {
        const HostPass &hp = passes[i];
        if (hp.type == HostPass::TILE) {
            const TilePass &t = hp.tile;
            int cnt[16] = {0};
            for (int k = 0; k < t.n_micro; ++k) {
                const MicroOp &mo = t.micro[k];
                if (mo.kind == MK_LAYER) cnt[mo.a] += __builtin_popcount((unsigned)mo.b);
                else if (mo.kind == MK_QFTL) cnt[MK_QFT] += __builtin_popcount((unsigned)mo.b);
                else if (mo.kind == MK_DIAGQ || mo.kind == MK_DIAGC) cnt[MK_DIAG]++;
                else cnt[mo.kind]++;
            }
            os << "TILE T=" << t.T << " L=" << t.L << " hb=[";
            for (int k = 0; k < t.H; ++k) os << (k ? "," : "") << t.hb[k];
            os << "] tma=" << (hp.tma.ok ? 1 : 0) << " sweeps=" << t.n_sweeps << " R=" << t.R << " prog=" << program_sweeps(t) << " straight=" << straight_sweeps(t)
               << " U1=" << cnt[MK_U1] + cnt[MK_H] + cnt[MK_RXC] + cnt[MK_U1R] + cnt[MK_ROT] << " ZYZ=" << cnt[MK_ZYZ]
               << " U2=" << cnt[MK_U2]
               << " DIAG=" << cnt[MK_DIAG] << " QFT=" << cnt[MK_QFT];
            int nd = 0, slow = 0, fq = 0, fc = 0;
            for (int k = 0; k < t.n_sweeps; ++k) nd += t.sweeps[k].dense ? 1 : 0;
            for (int k = 0; k < t.n_micro; ++k) {
                if (t.micro[k].kind == MK_DIAG && (t.micro[k].b != 0 || __builtin_popcount((unsigned)t.micro[k].a) > 2))
                    slow++;
                if (t.micro[k].kind == MK_DIAGQ) fq++;
                if (t.micro[k].kind == MK_DIAGC) fc++;
            }
            if (nd) os << " DENSE=" << nd;
            if (fq) os << " DIAGQ=" << fq;
            if (fc) os << " DIAGC=" << fc;
            if (slow) os << " DIAG_GENERAL=" << slow;
            os << " consts=" << t.n_const << "\n";
        } else if (hp.type == HostPass::PERM) {
            os << "PERM xor=" << hp.perm.xor_mask << "\n";
        } else {
            os << "GATHER\n";
        }
    }
    return os.str();
}

}  // namespace qs
