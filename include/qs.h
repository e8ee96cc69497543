/*
 * qs.h -- C ABI of the structured-layer state-vector engine (libqs.so).
 *
 * The engine applies gate lists to 2^n-amplitude complex64 state vectors on
 * one CUDA GPU (sm_103a).  A fusion detector routes the gate stream into the
 * layer families of the paper's Sec. 5.1 (phase-LUT diagonals, GF(2) affine
 * permutation gathers, fused tensor-product single-qubit layers, radix-2^r
 * QFT / Walsh butterflies, basis-conjugated XX/YY layers) plus dense blocks,
 * each run by a hand-written CUDA kernel.  The calls follow the paper's
 * statement of the problem: state initialisation, gate application and Pauli
 * expectation (Sec. 3.2.1-3.2.2), gradients of parameterised circuits (Sec.
 * 3.2.3; here by the adjoint method rather than parameter shift).
 *
 * Conventions (all calls):
 *  - State: complex64 interleaved (re, im) float pairs, 2^n amplitudes per
 *    state, `batch` states stored back to back (state b starts at element
 *    b * 2^n).  Qubit q is bit n-1-q of the basis index (most significant
 *    first; Sec. 3.2.2 reshape (2^q, 2, 2^(n-q-1)) and App. A).
 *  - Gate matrices follow the gate library of Sec. 3.2.2 and the OpenQASM
 *    table of Sec. 3.3: R_P(t) = exp(-i t P / 2); RZZ(t) = exp(-i t/2 Z(x)Z)
 *    (the theta = -2 J dt mapping of Sec. 4.1); CP(t) = diag(1,1,1,e^{it});
 *    P(l) = U1(l) = diag(1, e^{il}); U2/U3 as in OpenQASM 2.0.  For multi-qubit
 *    gates w[0] is the most significant bit of the gate matrix index (the
 *    control for controlled gates).
 *  - Pauli masks: bit q of x_mask / z_mask refers to qubit q; a qubit with both
 *    bits set carries Y.
 *  - Errors: every call returns a qs_status.  On failure nothing of the
 *    requested operation has been applied (validation precedes any launch),
 *    and qs_last_error() gives a message for the calling thread.  Asynchronous
 *    CUDA faults surface as QS_ERR_CUDA on the next synchronous call.
 *  - Streams: all device work of a state runs on the state's stream (set at
 *    qs_wrap / qs_set_stream; the legacy default stream otherwise).
 *    qs_apply_circuit is asynchronous with respect to the host; qs_expect,
 *    qs_grad and the amplitude copies synchronise the state's stream.
 *  - Threads: a qs_state must not be used from two host threads at once.
 */
#ifndef QS_ABI_H_INCLUDED
#define QS_ABI_H_INCLUDED

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qs_status;
enum {
    QS_OK = 0,
    QS_ERR_INVALID_ARG = 1,  /* bad pointer, size, wire, kind or arity      */
    QS_ERR_UNSUPPORTED = 2,  /* valid request the library does not support  */
    QS_ERR_OOM = 3,          /* device allocation failed / cap exceeded     */
    QS_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed        */
    QS_ERR_TIMEOUT = 5,      /* a bounded device wait ran out               */
    QS_ERR_INTERNAL = 6      /* a device-side consistency check failed      */
};

/* Gate kinds: the gate library of Sec. 3.2.2, the OpenQASM 2.0 coverage table
 * of Sec. 3.3 and the Trotter-term gates of Sec. 5.1. */
enum qs_gate_kind {
    QS_I = 0, QS_X = 1, QS_Y = 2, QS_Z = 3, QS_H = 4, QS_S = 5, QS_SDG = 6,
    QS_T = 7, QS_TDG = 8, QS_SX = 9,
    QS_RX = 10, QS_RY = 11, QS_RZ = 12,   /* p[0] = theta                   */
    QS_P = 13,                            /* U1 / phase gate, p[0] = lambda */
    QS_U2 = 14,                           /* p[0] = phi, p[1] = lambda      */
    QS_U3 = 15,                           /* p[0..2] = theta, phi, lambda   */
    QS_U = 16,                            /* dense 2x2: `dense` -> 8 doubles */
    QS_CX = 32, QS_CY = 33, QS_CZ = 34, QS_CH = 35, QS_SWAP = 36,
    QS_ISWAP = 37, QS_CRX = 38, QS_CRY = 39, QS_CRZ = 40,
    QS_CP = 41,                           /* CPHASE, p[0] = theta           */
    QS_RZZ = 42, QS_RXX = 43, QS_RYY = 44,/* exp(-i p[0]/2 P(x)P)           */
    QS_CCX = 64, QS_CSWAP = 65            /* Toffoli, Fredkin               */
};

/* One gate record.  Arrays of records are owned by the caller, read during
 * the call and not retained. */
typedef struct qs_gate {
    uint16_t kind;       /* enum qs_gate_kind                                */
    uint8_t nw;          /* number of wires; must equal the kind's arity     */
    uint8_t flags;       /* reserved, 0                                      */
    int32_t w[3];        /* wires (qubit indices), distinct, in [0, n)       */
    double p[3];         /* angles in radians                                */
    int32_t param_idx;   /* -1: fixed; else p[0] := params[b*n_params + idx] */
    int32_t reserved;    /* 0                                                */
    const double *dense; /* QS_U only: row-major 2x2 complex128 as (re, im);
                            finite entries; unitarity is the caller's     */
} qs_gate;

/* One Pauli term coeff * P, P = prod_q sigma_q from (x_mask, z_mask). */
typedef struct qs_pauli {
    double coeff;
    uint64_t x_mask;
    uint64_t z_mask;
} qs_pauli;

enum qs_mode {
    QS_MODE_FUSED = 0,   /* detector + fused layer kernels (default)         */
    QS_MODE_PERGATE = 1  /* one kernel launch per gate: the baseline path    */
};

/* Dense k-qubit blocks (fused mode only).  With dense_prec != QS_DENSE_OFF
 * the detector's output is regrouped into dense blocks of at most
 * block_qubits qubits (generic matrix fusion, which the paper's appendix
 * "Complete Per-Workload Speedups" names as the next extension):
 * consecutive 1- and 2-qubit ops and the in-block part of diagonal layers
 * are multiplied into one 2^k x 2^k complex matrix in FP64; the parts of
 * diagonal layers that cross blocks (the boundary bonds of a ZZ layer) stay
 * diagonal.  Blocks of 3..5 qubits are applied inside the tile pass as
 * out = U X over 5 tile bits (smaller blocks padded with the identity), in
 * the chosen arithmetic:
 *   QS_DENSE_FP32   -- FP32 FMA on the CUDA cores;
 *   QS_DENSE_TF32X3 -- tensor cores, split precision: U = U_hi + U_lo and
 *                      X = X_hi + X_lo in TF32, U_hi X_hi + U_hi X_lo +
 *                      U_lo X_hi accumulated in FP32 (about FP32 accuracy);
 *   QS_DENSE_BF16   -- tensor cores, U and X rounded to BF16 with FP32
 *                      accumulation (about 3 significant digits per block).
 * Blocks of 1-2 qubits run as the ordinary FP32 2x2 / 4x4 micro-ops. */
enum qs_dense_prec {
    QS_DENSE_OFF = 0,
    QS_DENSE_FP32 = 1,
    QS_DENSE_TF32X3 = 2,
    QS_DENSE_BF16 = 3
};

/* Options for qs_apply_circuit / qs_plan_describe; NULL means defaults. */
typedef struct qs_opts {
    int32_t mode;         /* enum qs_mode                                    */
    int32_t tile_qubits;  /* qubits per tile pass, 0 = default (13)          */
    int32_t low_qubits;   /* contiguous low bits per tile row, 0 = default;
                             the planner clamps the shape: tile_qubits <= 13
                             and <= n; a tile smaller than the state keeps
                             >= 2 high bits (with dense blocks: >= the block
                             size), raising tile_qubits to 3 (block size + 1)
                             or lowering low_qubits as needed              */
    int32_t group_qubits; /* tile bits held in registers per sweep (1..5),
                             0 = default (5)                                 */
    int32_t dense_prec;   /* enum qs_dense_prec, 0 = off                      */
    int32_t block_qubits; /* largest dense block (3..5), 0 = default (5)      */
} qs_opts;

typedef struct qs_state qs_state;

/* Allocate `batch` states of n qubits in device memory owned by the library,
 * each initialised to |0...0> (Sec. 3.2.1 state management: an n-qubit
 * register starts in |0...0> and is held as 2^n amplitudes; Sec. 2.1 for the
 * state-vector representation).  n in [1, 33]; batch >= 1.  Errors:
 * QS_ERR_INVALID_ARG (out == NULL, batch < 1), QS_ERR_UNSUPPORTED (n out of
 * range), QS_ERR_OOM (allocation failed).  Free with qs_free. */
qs_status qs_alloc(int n, int batch, qs_state **out);

/* Wrap caller-owned device memory (e.g. a torch tensor) of batch * 2^n
 * complex64 amplitudes, 16-byte aligned (the amplitude array of Sec. 3.2.1,
 * owned by the caller instead of the library).  The library never frees
 * `dev_ptr`; `cuda_stream` (a cudaStream_t, may be NULL) becomes the state's
 * stream.  The contents are left as they are. */
qs_status qs_wrap(void *dev_ptr, int n, int batch, void *cuda_stream, qs_state **out);

/* Release the handle, library-owned memory and scratch buffers.  NULL is a
 * no-op.  Waits for the state's stream first. */
qs_status qs_free(qs_state *st);

/* Replace the state's stream (cudaStream_t, NULL = legacy default). */
qs_status qs_set_stream(qs_state *st, void *cuda_stream);

/* Hand the library a caller-owned device scratch buffer of `bytes` bytes
 * (>= batch * 2^n * 8 for out-of-place gathers).  Without one the library
 * allocates its own on first need.  The buffer must stay valid until
 * qs_free or the next qs_set_scratch. */
qs_status qs_set_scratch(qs_state *st, void *dev_ptr, size_t bytes);

/* Device pointer of the amplitudes (batch * 2^n complex64). */
qs_status qs_device_ptr(const qs_state *st, void **out);

/* Reset every state of the batch to |0...0> (Sec. 3.2.1); asynchronous. */
qs_status qs_init_zero(qs_state *st);

/* Copy batch * 2^n complex64 amplitudes in (src) or out (dst); `is_device`
 * says whether the pointer is device memory (Sec. 3.2.1: the amplitudes of
 * the state are readable and settable as one array, index bit n-1-q =
 * qubit q).  Synchronous: returns after
 * the copy is complete. */
qs_status qs_set_amplitudes(qs_state *st, const void *src, int is_device);
qs_status qs_get_amplitudes(const qs_state *st, void *dst, int is_device);

/* Apply the gate list to every state of the batch, in order (Sec. 3.2.2
 * gate application on the reshaped state; Sec. 5.1 layer families and
 * Sec. 5.2 semantics-preserving fusion, which the fused mode follows).
 * params: NULL, or batch x n_params doubles (row b resolves param_idx for
 * state b).  Every gate is validated before anything runs: kind and nw
 * consistent, wires distinct and in [0, n), param_idx < n_params, dense != NULL
 * for QS_U; a failure returns QS_ERR_INVALID_ARG with the state untouched.
 * In QS_MODE_FUSED the detector builds layer passes whose result equals the
 * gate-by-gate product up to float rounding (permutations exactly).
 * Asynchronous on the state's stream. */
qs_status qs_apply_circuit(qs_state *st, const qs_gate *gates, size_t n_gates,
                           const double *params, int n_params, const qs_opts *opts);

/* out[b] = <psi_b| sum_k coeff_k P_k |psi_b> (real part) for each state b,
 * accumulated in FP64 on the device (Sec. 3.2.1 Pauli expectation).
 * Masks must lie within the n qubits.  Synchronous. */
qs_status qs_expect(qs_state *st, const qs_pauli *terms, size_t n_terms, double *out);

/* Adjoint-method gradient of E_b(theta) = <psi_b(theta)|H|psi_b(theta)> with
 * psi_b(theta) = U(theta_b)|0...0>, H = sum_k coeff_k P_k.  The paper's
 * variational algorithms (Sec. 3.2.3, VQE with a hardware-efficient ansatz)
 * take gradients by parameter shift, two energy evaluations per parameter;
 * this call returns all of them from one reverse sweep instead (the adjoint
 * method of Jones and Gacon 2020, arXiv:2009.02823: lambda = H psi carried
 * back through the inverse gates, dE/dt = Im <lambda| G |psi> at each
 * rotation exp(-i t G / 2)).  The results equal the parameter-shift values
 * up to float rounding.  The state is
 * overwritten: on return it holds psi_b(theta).  energy: batch doubles;
 * grad: batch x n_params doubles (zero for unused indices).  Parameterised
 * gates must be QS_RX, QS_RY, QS_RZ, QS_RZZ or QS_CP (else
 * QS_ERR_UNSUPPORTED); each index may feed several gates (contributions add).
 * Workspace: when the device has room, K + 1 states per batch item (K =
 * gradient points: psi is stored at each during the forward pass and the
 * reverse sweep un-applies only lambda); otherwise two (the psi / lambda
 * pairs, both un-applied).  It is allocated at the first call and kept with
 * the state until qs_free (a later call that needs more reallocates it).
 * Synchronous. */
qs_status qs_grad(qs_state *st, const qs_gate *gates, size_t n_gates,
                  const double *params, int n_params,
                  const qs_pauli *terms, size_t n_terms,
                  double *energy, double *grad);

/* One MaxCut graph: n vertices (one qubit each), edges as 2 * n_edges
 * vertex indices (u0, v0, u1, v1, ...), no self-loops. */
typedef struct qs_graph {
    int32_t n;
    int32_t n_edges;
    const int32_t *edges;
} qs_graph;

/* Batched QAOA MaxCut (Sec. 3.2.3: H_C = 1/2 sum_edges (I - Z_u Z_v),
 * H_M = sum_q X_q).  For graph g and angle set a (n_sets per graph):
 *   |psi> = prod_{l=1..p} e^{-i beta_l H_M} e^{-i gamma_l H_C} |+>^n,
 *   out[g * n_sets + a] = <psi|H_C|psi>   (FP64 accumulation).
 * gammas / betas: n_graphs x n_sets x p doubles (row-major).  Every
 * instance with n <= 24 runs in one persistent launch that needs no host
 * planning: CTAs take instances (largest first) from a device work counter;
 * a state with n <= 14 stays in the CTA's shared memory, a larger one lives
 * in the CTA's slot of device memory and moves through shared memory in
 * 2^14-amplitude tiles, two passes per layer.  Graphs with 24 < n <= 30 run
 * through the fused tile-pass executor, one graph (all its angle sets as a
 * batch) at a time.  Limits: p <= 16, <= 64 edges per graph.  Allocates its
 * own device memory (one state of the largest n above 14 per SM for the
 * persistent launch); synchronous on cuda_stream. */
qs_status qs_qaoa_maxcut(const qs_graph *graphs, size_t n_graphs, int n_sets, int p, const double *gammas,
                         const double *betas, double *out, void *cuda_stream);

/* Autotuner for the fused executor's tile passes (the tile shape, qubits per
 * pass and register-group depth that the kernels of Sec. 5 are built
 * around): applies the circuit to a private copy of the state under each
 * candidate configuration -- tile_qubits T in {12, 13}, low_qubits L in
 * {4, 5}, group_qubits R in {4, 5} (R = 5 only with dense blocks), and the
 * planner's own choice (all three 0) -- one untimed call, then `reps` calls
 * timed with CUDA events on the state's stream, and writes the fastest into
 * *best (the remaining fields copied from *base, which may be NULL) and its
 * milliseconds per call into *best_ms (may be NULL).  The state's amplitudes
 * are left unchanged.  A choice is kept per (GPU name, n, batch, gate
 * structure -- kinds, wires and parameter slots, not angle values -- and
 * dense settings); repeating a request returns the kept choice without
 * timing anything (*best_ms = the time measured then).  cache_path (may be
 * NULL) names a text file of earlier choices, one per line, read on first
 * use and appended to after each new measurement.  Needs device memory for
 * one more copy of the state (and its scratch buffer if the plan has
 * permutation passes); synchronises the state's stream.  Errors:
 * QS_ERR_INVALID_ARG (NULL st or best, reps outside [1, 100], base->mode not
 * QS_MODE_FUSED, invalid gates or parameters), QS_ERR_OOM, QS_ERR_CUDA. */
qs_status qs_autotune(qs_state *st, const qs_gate *gates, size_t n_gates, const double *params, int n_params,
                      const qs_opts *base, int reps, const char *cache_path, qs_opts *best, double *best_ms);

/* Test hook: write the detector's plan for an n-qubit circuit as text
 * (one line per pass: family, qubits, op count) into buf (NUL-terminated,
 * truncated to len).  Needs no GPU.  *passes (if non-NULL) receives the
 * number of full-state HBM passes the plan makes. */
qs_status qs_plan_describe(int n, const qs_gate *gates, size_t n_gates,
                           const qs_opts *opts, char *buf, size_t len, int *passes);

/* OpenQASM 2.0 import (Sec. 3.3 "OpenQASM Integration"; App. B.1): the
 * unitary subset of the NUL-terminated program `src` as gate records for
 * qs_apply_circuit / qs_plan_describe.  Needs no GPU.
 *  - Registers are laid end to end in declaration order (the first qreg
 *    holds qubits 0..k-1, the next continues from k); *n_qubits receives the
 *    total.
 *  - Gate names map to the kinds above: the primitives U (U3) and CX, and
 *    the standard-library names (id, x, y, z, h, s, sdg, t, tdg, sx, rx, ry,
 *    rz, u1 / p, u2, u3 / u, cx, cy, cz, ch, swap, iswap, crx, cry, crz,
 *    cu1 / cp, rzz, rxx, ryy, ccx, cswap), with this library's matrices
 *    (global phases may differ from a textual expansion of qelib1.inc);
 *    cu3 becomes controlled-U3 exactly, spelled with RZ, RY, CX and P;
 *    c3x / c4x become exact ancilla-free phase polynomials (CX, P, H);
 *    sxdg becomes SX^3.
 *  - `gate` definitions in the program take precedence over those names;
 *    they are inlined recursively with parameters and arguments bound.
 *  - A call on whole registers applies the gate once per index.
 *  - Barriers are skipped.  Measurements are accepted after the last unitary
 *    gate only; the records describe the state before them.
 * On success *gates receives a library-allocated array of *n_gates records
 * (param_idx -1, dense NULL; NULL when the program applies no gate), to be
 * released with qs_qasm_free.  Errors (outputs then NULL / 0, message with
 * the line number in qs_last_error): QS_ERR_INVALID_ARG (a NULL argument,
 * syntax, undeclared names, wrong qubit or parameter counts, a repeated
 * qubit, registers of different sizes in one call, an angle that is not
 * finite), QS_ERR_UNSUPPORTED (a gate
 * that is neither defined nor in the list, opaque gates, reset, if, a gate
 * after a measurement, an include other than qelib1.inc, more than 63 qubits,
 * more than 2^25 gate applications counting inlined ones, definitions nested
 * more than 64 deep, expressions nested more than 200 deep). */
qs_status qs_qasm_parse(const char *src, qs_gate **gates, size_t *n_gates, int *n_qubits);
/* Release an array from qs_qasm_parse; NULL is a no-op. */
void qs_qasm_free(qs_gate *gates);

/* Per-kernel-family timing with CUDA events recorded on the state's stream
 * around each launch.  enable != 0 turns it on and clears the counters. */
qs_status qs_profile_enable(qs_state *st, int enable);
/* Copy up to `cap` records: name (NUL-terminated, 32 bytes), launches,
 * total milliseconds, algorithmic bytes moved.  *count = records written.
 * Synchronises the state's stream. */
typedef struct qs_profile_record {
    char name[32];
    int64_t launches;
    double total_ms;
    double bytes;
} qs_profile_record;
qs_status qs_profile_read(qs_state *st, qs_profile_record *out, int cap, int *count);

/* Pauli expectation values without any device allocation.  The paper has
 * no counterpart: this call exists for callers that cannot call cudaMalloc.
 * A plug-in inside a host application that owns every device allocation
 * through its own arena may not allocate behind the host's back; a process
 * that sized its states to fill the GPU has no room for a late allocation;
 * a real-time loop cannot take the implicit device synchronisation of
 * cudaMalloc / cudaFree.  It computes what qs_expect computes
 * (out[b] = <psi_b| sum_k coeff_k P_k |psi_b>, FP64 accumulation), but takes
 * the state as a plain device pointer and keeps its scratch (block partial
 * sums, finished sums, the term table) in one file-scope static __device__
 * array of 694,272 bytes compiled into the library.  Every GPU that loads
 * the library holds that array until the process exits.
 *   dev_state: device pointer, batch * 2^n complex64, 16-byte aligned (read only)
 *   n in [1, 33]; batch in [1, 16]; n_terms <= 256 (larger -> QS_ERR_UNSUPPORTED,
 *   nothing launched); n_terms == 0 gives out[b] = 0; out: host array of
 *   batch doubles; cuda_stream: the cudaStream_t to run on (NULL = legacy
 *   default).  Synchronous: returns after the stream has finished the sums.
 * The first call on each device (per CUDA context) looks up the array's
 * device address with cudaGetSymbolAddress, with that device current, and
 * keeps it; that first call should come before any stream capture.  All
 * calls share the one array and it keeps the previous call's contents:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it.  Nothing in it needs clearing -- every slot a call reads is
 * written earlier in the same call.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
qs_status qs_expect_noalloc(const void *dev_state, int n, int batch, const qs_pauli *terms, size_t n_terms,
                            double *out, void *cuda_stream);

/* Message for the last failed call on this host thread ("" if none). */
const char *qs_last_error(void);

/* Library version string. */
const char *qs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QS_ABI_H_INCLUDED */
