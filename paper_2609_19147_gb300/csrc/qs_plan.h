// Host-side planner: gate validation, gate matrices (FP64), the fusion
// detector (Sec. 5.2 "Semantics-Preserving Fusion") and the HBM-pass
// scheduler.  No CUDA calls; qs_plan_describe runs it without a GPU.
#pragma once

#include <complex>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "qs.h"
#include "qs_internal.h"

namespace qs {

using cd = std::complex<double>;

// A validated gate with its angles bound (index bits, not qubits).
struct RGate {
    int kind = 0, nw = 0;
    int q[3] = {0, 0, 0};   // qubits as given
    int b[3] = {0, 0, 0};   // index bits: b = n-1-q
    double p[3] = {0, 0, 0};
    cd dense[4];
};

// Internal kind of the fused detector (never accepted from callers): a
// two-qubit diagonal with phases dense[k].real(), k = x_b0 * 2 + x_b1.
constexpr int K_DIAG2 = 1000;

// Diagonal phase as a quadratic form over the index bits (FP64, radians):
//   phase(x) = g0 + sum_b a[b] x_b + sum_{b<c} pairs[(b,c)] x_b x_c
// Every diagonal gate of the library (Z, S, T, RZ, P, CZ, CP, CRZ, RZZ) is of
// this form, and so is any product of them (Sec. 5.1 phase-LUT layers).
struct Diag {
    double g0 = 0.0;
    std::map<int, double> a;
    std::map<std::pair<int, int>, double> pairs;
    bool empty() const { return a.empty() && pairs.empty() && g0 == 0.0; }
    uint64_t support() const;
    void add1(int b, double ph0, double ph1);
    void add2(int b0, int b1, const double ph[4]);   // ph index = x_b0*2 + x_b1
    void merge(const Diag &o);
};

enum FKind { F_U1 = 0, F_U2, F_DIAG, F_QFT, F_GF2, F_DENSE };

// A fused op in index-bit space.
struct FOp {
    FKind kind = F_U1;
    int t0 = -1, t1 = -1;          // U1: t0; U2: t0 = matrix MSB, t1 = LSB
    uint64_t cmask = 0, cval = 0;  // control condition on the index
    cd m[16];                      // U1: 2x2, U2: 4x4 (row-major)
    Diag diag;                     // F_DIAG
    int p = -1, lo = -1;           // F_QFT
    // F_GF2: forward affine map f(x) = M x ^ c as rows (bit i of f(x) =
    // parity(rows[i] & x) ^ bit i of c); the state moves psi'[f(x)] = psi[x].
    std::vector<uint64_t> rows;
    uint64_t c = 0;
    // F_DENSE: block on index bits dbits (k <= 5); dm is 2^k x 2^k row-major,
    // bit j of a matrix index is the value of index bit dbits[j]
    std::vector<int> dbits;
    std::vector<cd> dm;
    int n_gates = 1;               // source gates absorbed
    uint64_t N() const;            // bits acted on non-diagonally
    uint64_t D() const;            // bits the op depends on diagonally
    uint64_t cN = 0, cD = 0;       // cached N() / D() (set by cache_masks)
    void cache_masks() {
        cN = N();
        cD = D();
    }
};

// TMA tensor geometry of a tile pass (see TmaGeom): dims in ascending bit
// order with their global extents, byte strides and box extents.
struct TmaPlan {
    bool ok = false;
    int ndims = 0;
    int kind[5] = {0, 0, 0, 0, 0};
    int off[5] = {0, 0, 0, 0, 0};
    int w[5] = {0, 0, 0, 0, 0};
    int batch_dim = -1;
    uint64_t gdim[5] = {1, 1, 1, 1, 1};
    uint64_t gstride[5] = {0, 0, 0, 0, 0};   // bytes, dims 1..4
    uint32_t box[5] = {1, 1, 1, 1, 1};
};

struct HostPass {
    enum Type { TILE = 0, PERM = 1, GATHER = 2 } type = TILE;
    TilePass tile;                 // TILE
    std::vector<float2> consts;    // TILE constants
    TmaPlan tma;                   // TILE: tensor-copy geometry
    int uses_roots = 0;
    PermPass perm;                 // PERM
    GatherPass gather;             // GATHER
    int out_of_place = 0;          // set by the executor's buffer routing
    std::string note;
};

int program_sweeps(const TilePass &tp);   // sweeps the kernel runs as a specialised program
int straight_sweeps(const TilePass &tp);  // sweeps of one layer run as straight-line code
int general_diags(const TilePass &tp);    // diagonals evaluated factor by factor per amplitude
bool layer_only(const TilePass &tp);      // only one-qubit layer kinds and diagonals

struct Plan {
    int n = 0;
    int mode = QS_MODE_FUSED;
    // items > 1: one plan for a batch whose items differ only in constant
    // values; every TILE pass holds items x n_const constants, item after item
    int items = 1;
    std::vector<HostPass> passes;  // fused mode
    std::vector<PgOp> pg;          // per-gate mode: one entry per launch
    int n_gates = 0;
    std::string describe() const;
    int hbm_passes() const;
};

// Validate gates and bind parameters for batch item `bi`.  Returns QS_OK or
// QS_ERR_INVALID_ARG / QS_ERR_UNSUPPORTED with `err` set.
qs_status resolve_gates(int n, const qs_gate *gates, size_t n_gates, const double *params,
                        int n_params, int bi, std::vector<RGate> &out, std::string &err);

// Full unitary of one gate in the kind's own wire order (2^nw x 2^nw).
void gate_matrix(const RGate &g, cd *M);
bool gate_is_diagonal(int kind);

// item_plan: the plan is one of several per-item plans that merge_item_plans
// is to combine (they must agree in everything but constant values), so no
// micro-op form is chosen by angle value (the real-rotation form MK_ROT, whose
// factor sits in the sweep scale, is left out).
qs_status build_fused_plan(int n, int batch, const std::vector<RGate> &gates, const qs_opts &o, Plan &plan,
                           std::string &err, bool item_plan = false);
qs_status build_pergate_plan(int n, const std::vector<RGate> &gates, Plan &plan, std::string &err);

// Merge per-item fused plans into one plan for `batch` states (a multiple of
// the item count) with per-item constants, when they agree in everything but
// constant values and every pass keeps its TMA tensor path at that batch.
bool merge_item_plans(std::vector<Plan> &plans, Plan &out, int batch);

// Fusion detector only (exposed for tests through qs_plan_describe).
void detect(int n, const std::vector<RGate> &gates, std::vector<FOp> &ops);

// Regroup detected ops into dense blocks of at most k index bits (qs_opts
// dense_prec / block_qubits); blocks of 1-2 bits come back as F_U1 / F_U2.
// cell_of[b] partitions the index bits: ops on disjoint bits share a block
// only within one cell (dense_cells: cells that fill the tile windows of
// T-bit tiles with L low bits).
void dense_cells(int n, int T, int L, int k, int *cell_of);
void fuse_dense(int n, int k, const int *cell_of, const std::vector<FOp> &in, std::vector<FOp> &out);

}  // namespace qs
