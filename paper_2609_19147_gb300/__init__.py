"""Python binding of libqs (the structured-layer state-vector engine).

Argument marshalling only: every step of gate application, expectation and
gradient runs in the library's CUDA kernels behind the C ABI of include/qs.h.
PyTorch supplies device memory and streams.  There is no CPU fallback: if
the compiled library is missing, importing this package raises.

Gate records are the ``workloads.Gate`` objects (kind name, wires, angles,
optional 2x2 matrix, parameter index); Pauli terms are (coeff, x_mask,
z_mask) with bit q = qubit q.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqs.so is not built ({LIB_PATH}); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")

_lib = ctypes.CDLL(LIB_PATH)

# --- enums (include/qs.h) ---------------------------------------------------
QS_OK, QS_ERR_INVALID_ARG, QS_ERR_UNSUPPORTED, QS_ERR_OOM, QS_ERR_CUDA, QS_ERR_TIMEOUT, QS_ERR_INTERNAL = range(7)
MODE_FUSED, MODE_PERGATE = 0, 1
KIND = {"I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8, "SX": 9,
        "RX": 10, "RY": 11, "RZ": 12, "P": 13, "U2": 14, "U3": 15, "U": 16,
        "CX": 32, "CY": 33, "CZ": 34, "CH": 35, "SWAP": 36, "ISWAP": 37, "CRX": 38, "CRY": 39,
        "CRZ": 40, "CP": 41, "RZZ": 42, "RXX": 43, "RYY": 44, "CCX": 64, "CSWAP": 65}


class QsGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint16), ("nw", ctypes.c_uint8), ("flags", ctypes.c_uint8),
                ("w", ctypes.c_int32 * 3), ("p", ctypes.c_double * 3), ("param_idx", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dense", ctypes.POINTER(ctypes.c_double))]


class QsPauli(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64)]


class QsOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_qubits", ctypes.c_int32), ("low_qubits", ctypes.c_int32),
                ("group_qubits", ctypes.c_int32), ("dense_prec", ctypes.c_int32), ("block_qubits", ctypes.c_int32)]


# qs_dense_prec: arithmetic of the dense k-qubit blocks (None / "off" = no dense blocks)
DENSE_PREC = {None: 0, "off": 0, "fp32": 1, "tf32x3": 2, "bf16": 3}


class QsGraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("edges", ctypes.POINTER(ctypes.c_int32))]


class QsProfileRecord(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i32 = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "qs_alloc": ([_i32, _i32, ctypes.POINTER(_vp)], _i32),
    "qs_wrap": ([_vp, _i32, _i32, _vp, ctypes.POINTER(_vp)], _i32),
    "qs_free": ([_vp], _i32),
    "qs_set_stream": ([_vp, _vp], _i32),
    "qs_set_scratch": ([_vp, _vp, _sz], _i32),
    "qs_device_ptr": ([_vp, ctypes.POINTER(_vp)], _i32),
    "qs_init_zero": ([_vp], _i32),
    "qs_set_amplitudes": ([_vp, _vp, _i32], _i32),
    "qs_get_amplitudes": ([_vp, _vp, _i32], _i32),
    "qs_apply_circuit": ([_vp, ctypes.POINTER(QsGate), _sz, _dp, _i32, ctypes.POINTER(QsOpts)], _i32),
    "qs_expect": ([_vp, ctypes.POINTER(QsPauli), _sz, _dp], _i32),
    "qs_grad": ([_vp, ctypes.POINTER(QsGate), _sz, _dp, _i32, ctypes.POINTER(QsPauli), _sz, _dp, _dp], _i32),
    "qs_plan_describe": ([_i32, ctypes.POINTER(QsGate), _sz, ctypes.POINTER(QsOpts), ctypes.c_char_p, _sz,
                          ctypes.POINTER(_i32)], _i32),
    "qs_profile_enable": ([_vp, _i32], _i32),
    "qs_profile_read": ([_vp, ctypes.POINTER(QsProfileRecord), _i32, ctypes.POINTER(_i32)], _i32),
    "qs_expect_noalloc": ([_vp, _i32, _i32, ctypes.POINTER(QsPauli), _sz, _dp, _vp], _i32),
    "qs_qaoa_maxcut": ([ctypes.POINTER(QsGraph), _sz, _i32, _i32, _dp, _dp, _dp, _vp], _i32),
    "qs_autotune": ([_vp, ctypes.POINTER(QsGate), _sz, _dp, _i32, ctypes.POINTER(QsOpts), _i32, ctypes.c_char_p,
                     ctypes.POINTER(QsOpts), _dp], _i32),
    "qs_qasm_parse": ([ctypes.c_char_p, ctypes.POINTER(ctypes.POINTER(QsGate)), ctypes.POINTER(_sz),
                       ctypes.POINTER(_i32)], _i32),
    "qs_qasm_free": ([ctypes.POINTER(QsGate)], None),
    "qs_last_error": ([], ctypes.c_char_p),
    "qs_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class QsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"qs status {status}: {msg}")
        self.status = status


def _check(st: int):
    if st != QS_OK:
        raise QsError(st, _lib.qs_last_error().decode())


def version() -> str:
    return _lib.qs_version().decode()


# --- marshalling ---------------------------------------------------------------
class CGates:
    """ctypes array of qs_gate built from workloads.Gate records (keeps dense
    matrices alive for the duration of the object)."""

    def __init__(self, gates: Sequence):
        self.n = len(gates)
        self.arr = (QsGate * max(1, self.n))()
        self._keep = []
        for i, g in enumerate(gates):
            c = self.arr[i]
            c.kind = KIND[g.kind]
            c.nw = len(g.wires)
            for m, w in enumerate(g.wires):
                c.w[m] = int(w)
            for m, p in enumerate(g.params[:3]):
                c.p[m] = float(p)
            c.param_idx = int(g.pidx)
            if g.matrix is not None:
                d = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128).reshape(-1)).view(np.float64)
                self._keep.append(d)
                c.dense = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _paulis(terms) -> Tuple[ctypes.Array, int]:
    arr = (QsPauli * max(1, len(terms)))()
    for i, (c, x, z) in enumerate(terms):
        arr[i].coeff = float(c)
        arr[i].x_mask = int(x)
        arr[i].z_mask = int(z)
    return arr, len(terms)


def _opts(mode="fused", tile_qubits=0, low_qubits=0, group_qubits=0, dense=None, block_qubits=0) -> QsOpts:
    o = QsOpts()
    o.mode = MODE_PERGATE if mode == "pergate" else MODE_FUSED
    o.tile_qubits = int(tile_qubits)
    o.low_qubits = int(low_qubits)
    o.group_qubits = int(group_qubits)
    if dense not in DENSE_PREC:
        raise ValueError(f"dense must be one of {sorted(k for k in DENSE_PREC if k)}, got {dense!r}")
    o.dense_prec = DENSE_PREC[dense]
    o.block_qubits = int(block_qubits)
    return o


def plan_describe(n: int, gates, mode: str = "fused", tile_qubits: int = 0, low_qubits: int = 0,
                  group_qubits: int = 0, dense=None, block_qubits: int = 0):
    """The detector's plan as text and its number of HBM passes (no GPU needed)."""
    cg = gates if isinstance(gates, CGates) else CGates(gates)
    buf = ctypes.create_string_buffer(1 << 20)
    passes = ctypes.c_int(0)
    o = _opts(mode, tile_qubits, low_qubits, group_qubits, dense, block_qubits)
    _check(_lib.qs_plan_describe(n, cg.arr, cg.n, ctypes.byref(o), buf, len(buf), ctypes.byref(passes)))
    return buf.value.decode(), passes.value


# --- OpenQASM 2.0 import --------------------------------------------------------------
_KIND_NAME = {v: k for k, v in KIND.items()}
_N_PARAMS = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "U2": 2, "U3": 3, "CRX": 1, "CRY": 1, "CRZ": 1, "CP": 1,
             "RZZ": 1, "RXX": 1, "RYY": 1}


class GateRecord(tuple):
    """(kind, wires, params): the fields CGates and the gate-list consumers read."""
    __slots__ = ()

    def __new__(cls, kind, wires, params):
        return super().__new__(cls, (kind, tuple(wires), tuple(params)))

    kind = property(lambda self: self[0])
    wires = property(lambda self: self[1])
    params = property(lambda self: self[2])
    matrix = None
    pidx = -1


def parse_qasm(src: str):
    """OpenQASM 2.0 program -> (n_qubits, [GateRecord]) through qs_qasm_parse
    (the library's parser; no GPU needed)."""
    arr = ctypes.POINTER(QsGate)()
    n_gates = _sz(0)
    n_qubits = _i32(0)
    _check(_lib.qs_qasm_parse(src.encode(), ctypes.byref(arr), ctypes.byref(n_gates), ctypes.byref(n_qubits)))
    try:
        out = []
        for i in range(n_gates.value):
            g = arr[i]
            name = _KIND_NAME[g.kind]
            out.append(GateRecord(name, [g.w[m] for m in range(g.nw)], [g.p[m] for m in range(_N_PARAMS.get(name, 0))]))
    finally:
        _lib.qs_qasm_free(arr)
    return n_qubits.value, out


# --- device state ----------------------------------------------------------------
class State:
    """`batch` n-qubit complex64 states in a torch CUDA tensor of shape
    (batch, 2^n), wrapped by a qs_state handle on torch's current stream."""

    def __init__(self, n: int, batch: int = 1, tensor=None, stream=None):
        import torch
        self.n, self.batch = int(n), int(batch)
        if tensor is None:
            tensor = torch.zeros((self.batch, 1 << self.n), dtype=torch.complex64, device="cuda")
            tensor[:, 0] = 1.0
        assert tensor.is_cuda and tensor.dtype == torch.complex64 and tensor.is_contiguous()
        assert tensor.numel() == self.batch << self.n
        self.tensor = tensor
        s = stream if stream is not None else torch.cuda.current_stream(tensor.device)
        self.stream = s
        h = _vp()
        _check(_lib.qs_wrap(_vp(tensor.data_ptr()), self.n, self.batch, _vp(s.cuda_stream), ctypes.byref(h)))
        self.h = h
        self._scratch = None

    def close(self):
        if getattr(self, "h", None):
            _lib.qs_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def provide_scratch(self):
        """Give the library a torch-allocated scratch buffer for out-of-place passes."""
        import torch
        if self._scratch is None:
            self._scratch = torch.empty_like(self.tensor)
            _check(_lib.qs_set_scratch(self.h, _vp(self._scratch.data_ptr()),
                                       self._scratch.numel() * 8))

    def zero(self):
        _check(_lib.qs_init_zero(self.h))

    def set(self, amps: np.ndarray):
        a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex64).reshape(self.batch, -1))
        _check(_lib.qs_set_amplitudes(self.h, _vp(a.ctypes.data), 0))

    def get(self) -> np.ndarray:
        out = np.empty((self.batch, 1 << self.n), dtype=np.complex64)
        _check(_lib.qs_get_amplitudes(self.h, _vp(out.ctypes.data), 0))
        return out

    def apply(self, gates, params: Optional[np.ndarray] = None, mode: str = "fused",
              tile_qubits: int = 0, low_qubits: int = 0, group_qubits: int = 0, dense=None,
              block_qubits: int = 0):
        cg = gates if isinstance(gates, CGates) else CGates(gates)
        o = _opts(mode, tile_qubits, low_qubits, group_qubits, dense, block_qubits)
        if params is not None:
            p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(self.batch, -1))
            self._params = p
            _check(_lib.qs_apply_circuit(self.h, cg.arr, cg.n, p.ctypes.data_as(_dp), p.shape[1],
                                         ctypes.byref(o)))
        else:
            _check(_lib.qs_apply_circuit(self.h, cg.arr, cg.n, None, 0, ctypes.byref(o)))

    def autotune(self, gates, params: Optional[np.ndarray] = None, reps: int = 2, cache_path: Optional[str] = None,
                 dense=None, block_qubits: int = 0) -> dict:
        """Time the circuit under the candidate tile shapes on a copy of this
        state (the state is unchanged) and return the fastest as keyword
        arguments for apply(), plus 'ms' (milliseconds per call)."""
        cg = gates if isinstance(gates, CGates) else CGates(gates)
        base = _opts("fused", 0, 0, 0, dense, block_qubits)
        out = QsOpts()
        ms = ctypes.c_double(0.0)
        cp = cache_path.encode() if cache_path else None
        if params is not None:
            p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(self.batch, -1))
            _check(_lib.qs_autotune(self.h, cg.arr, cg.n, p.ctypes.data_as(_dp), p.shape[1], ctypes.byref(base),
                                    int(reps), cp, ctypes.byref(out), ctypes.byref(ms)))
        else:
            _check(_lib.qs_autotune(self.h, cg.arr, cg.n, None, 0, ctypes.byref(base), int(reps), cp,
                                    ctypes.byref(out), ctypes.byref(ms)))
        return {"tile_qubits": out.tile_qubits, "low_qubits": out.low_qubits, "group_qubits": out.group_qubits,
                "ms": ms.value}

    def expect(self, terms) -> np.ndarray:
        arr, k = _paulis(terms)
        out = np.zeros(self.batch, dtype=np.float64)
        _check(_lib.qs_expect(self.h, arr, k, out.ctypes.data_as(_dp)))
        return out

    def grad(self, gates, params: np.ndarray, terms) -> Tuple[np.ndarray, np.ndarray]:
        cg = gates if isinstance(gates, CGates) else CGates(gates)
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(self.batch, -1))
        arr, k = _paulis(terms)
        e = np.zeros(self.batch)
        g = np.zeros_like(p)
        _check(_lib.qs_grad(self.h, cg.arr, cg.n, p.ctypes.data_as(_dp), p.shape[1], arr, k,
                            e.ctypes.data_as(_dp), g.ctypes.data_as(_dp)))
        return e, g

    def profile(self, enable: bool = True):
        _check(_lib.qs_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        recs = (QsProfileRecord * 32)()
        cnt = ctypes.c_int(0)
        _check(_lib.qs_profile_read(self.h, recs, 32, ctypes.byref(cnt)))
        return {recs[i].name.decode(): (recs[i].launches, recs[i].total_ms, recs[i].bytes)
                for i in range(cnt.value)}


def qaoa_maxcut(instances, stream=None) -> np.ndarray:
    """Batched QAOA MaxCut: `instances` is a list of dicts with n, edges,
    gammas (n_sets x p), betas (n_sets x p) (the form of
    workloads.qaoa_batch).  Returns <C> per (graph, angle set), shape
    (n_graphs, n_sets)."""
    import torch
    if not instances:
        return np.zeros((0, 0))
    n_sets, p = np.asarray(instances[0]["gammas"]).shape
    arr = (QsGraph * len(instances))()
    keep = []
    gam = np.zeros((len(instances), n_sets, p))
    bet = np.zeros_like(gam)
    for i, inst in enumerate(instances):
        e = np.ascontiguousarray(np.asarray(inst["edges"], dtype=np.int32).reshape(-1))
        keep.append(e)
        arr[i].n = int(inst["n"])
        arr[i].n_edges = len(e) // 2
        arr[i].edges = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        gam[i] = inst["gammas"]
        bet[i] = inst["betas"]
    out = np.zeros((len(instances), n_sets))
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.qs_qaoa_maxcut(arr, len(instances), n_sets, p, gam.ctypes.data_as(_dp), bet.ctypes.data_as(_dp),
                               out.ctypes.data_as(_dp), _vp(s.cuda_stream)))
    return out


_AUTOGRAD_FN = None
_GRAD_STATES = {}   # (device index, n, batch) -> State kept between calls


def _grad_state(device, n: int, batch: int) -> "State":
    """The State that QSExpectation runs on: one per (device, n, batch), kept
    so that repeated calls (a training loop) reuse its device memory and the
    adjoint workspace that qs_grad keeps with it."""
    import torch
    idx = device.index if device.index is not None else torch.cuda.current_device()
    key = (idx, int(n), int(batch))
    st = _GRAD_STATES.get(key)
    if st is None or st.h is None:
        with torch.cuda.device(idx):
            st = State(n, batch=batch)
        _GRAD_STATES[key] = st
    return st


def _autograd():
    global _AUTOGRAD_FN
    if _AUTOGRAD_FN is not None:
        return _AUTOGRAD_FN
    import torch

    class QSExpectation(torch.autograd.Function):
        """E_b(theta_b) = <psi(theta_b)|H|psi(theta_b)> for a batch of parameter
        vectors; the backward pass uses the library's adjoint-method gradient
        (computed in the same qs_grad call as the energies).  Energies and the
        saved gradients live on the device of `params` (a CUDA device; CPU
        params run on the current CUDA device and get CPU results).  The
        angles go to the host once per call: the planner reduces them and
        builds the phase tables in FP64 there."""

        @staticmethod
        def forward(ctx, params, n, gates, terms):
            dev = params.device if params.is_cuda else torch.device("cuda", torch.cuda.current_device())
            p = params.detach().to("cpu", torch.float64).numpy().reshape(params.shape[0], -1)
            st = _grad_state(dev, n, p.shape[0])
            e, g = st.grad(gates, p, terms)
            ctx.save_for_backward(torch.from_numpy(g).to(device=params.device, dtype=params.dtype))
            return torch.from_numpy(e).to(device=params.device, dtype=params.dtype)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout.reshape(-1, 1).to(g.device, g.dtype) * g, None, None, None

    _AUTOGRAD_FN = QSExpectation
    return QSExpectation


def qs_expectation(params, n: int, gates, terms):
    """Differentiable batched energy: params (batch, P) torch tensor -> (batch,),
    on the device of `params`."""
    cg = gates if isinstance(gates, CGates) else CGates(gates)
    return _autograd().apply(params, n, cg, terms)
