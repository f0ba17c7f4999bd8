"""Python binding of libqsim, the GB300 state-vector simulator of the method of
quant-ph/0201042 (Niwa, Matsumoto, Imai).

Argument marshalling only: every gate, reduction and trajectory runs in the
CUDA kernels of libqsim.so behind the C ABI of include/qsim.h.  PyTorch
provides the device memory (a state is a torch complex tensor wrapped with
qs_wrap) and the stream (the current torch stream).  There is no CPU fallback:
if the library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqsim.so")

QS_C64 = 1
QS_C128 = 2
DTYPES = {"c64": QS_C64, "c128": QS_C128}
KIND_CODES = {
    "MATRIX": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "UP1": 5, "UP2": 6,
    "UR": 7, "URP1": 8, "RY": 9, "RZ": 10, "SWAP": 11,
}
STATUS = {0: "QS_OK", 1: "QS_EINVAL", 2: "QS_ERANGE", 3: "QS_ENOMEM", 4: "QS_ECUDA",
          5: "QS_ETIMEOUT", 6: "QS_EUNSUPPORTED"}


class QsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class C128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class QsGate(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("t", ctypes.c_int32), ("t2", ctypes.c_int32),
        ("param", ctypes.c_int32), ("ctrl_mask", ctypes.c_uint64), ("ctrl_val", ctypes.c_uint64),
        ("theta", ctypes.c_double * 2), ("u", C128 * 4),
    ]


class QsExecOpts(ctypes.Structure):
    _fields_ = [("no_fusion", ctypes.c_int32), ("max_ops_per_pass", ctypes.c_int32),
                ("c128_arith", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


ARITH = {"default": 0, "f64": 1, "ds": 2}


class QsNoise(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double), ("sigma", ctypes.c_double), ("mode", ctypes.c_int32),
                ("every", ctypes.c_int32)]


class QsTrajGroup(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("metric", ctypes.c_int32), ("target", ctypes.c_uint64),
                ("gates", ctypes.POINTER(QsGate)), ("m", ctypes.c_size_t), ("first", ctypes.c_uint32),
                ("count", ctypes.c_uint32), ("x0", ctypes.POINTER(ctypes.c_uint64)),
                ("flags", ctypes.c_void_p)]


class QsObservable(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("pauli", ctypes.c_char_p),
                ("ref", ctypes.c_void_p)]


OBS_PAULI = 0
OBS_FIDELITY = 1
NOISE_FLIPS = 0
NOISE_DEPOLARIZING = 1
TRAJ_NO_DEVIATION = 1
TRAJ_NO_FLIPS = 2
TRAJ_FIDELITY = 0
TRAJ_PROB = 1

assert ctypes.sizeof(QsGate) == 112

_lib: Optional[ctypes.CDLL] = None

# exported entry points and their argument types
_SIGS = {
    "qs_alloc": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
    "qs_wrap": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
    "qs_free": [ctypes.c_void_p],
    "qs_set_stream": [ctypes.c_void_p, ctypes.c_void_p],
    "qs_info": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                ctypes.POINTER(ctypes.c_int)],
    "qs_init_basis": [ctypes.c_void_p, ctypes.c_uint64],
    "qs_apply_1q": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(C128)],
    "qs_apply_ctrl": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(C128)],
    "qs_apply_mctrl": [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                       ctypes.POINTER(C128)],
    "qs_apply_swap": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
    "qs_apply_gate": [ctypes.c_void_p, ctypes.POINTER(QsGate)],
    "qs_apply_circuit": [ctypes.c_void_p, ctypes.POINTER(QsGate), ctypes.c_size_t,
                         ctypes.POINTER(QsExecOpts)],
    "qs_plan_create": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(QsGate), ctypes.c_size_t,
                       ctypes.POINTER(QsExecOpts), ctypes.POINTER(ctypes.c_void_p)],
    "qs_plan_execute": [ctypes.c_void_p, ctypes.c_void_p],
    "qs_plan_info": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "qs_plan_free": [ctypes.c_void_p],
    "qs_plan_set_timing": [ctypes.c_void_p, ctypes.c_int],
    "qs_plan_describe": [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "qs_plan_timing": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
    "qs_prob": [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)],
    "qs_prob_qubit": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "qs_expect": [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)],
    "qs_inner": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(C128)],
    "qs_norm": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)],
    "qs_renormalize": [ctypes.c_void_p],
    "qs_qft": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "qs_measure": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                   ctypes.POINTER(ctypes.c_uint64)],
    "qs_norm_noalloc": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "qs_run_trajectories": [ctypes.POINTER(QsTrajGroup), ctypes.c_int, ctypes.POINTER(QsNoise), ctypes.c_uint64,
                            ctypes.c_int, ctypes.POINTER(QsExecOpts), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_uint64)],
    "qs_adjoint_grad": [ctypes.c_void_p, ctypes.POINTER(QsGate), ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                        ctypes.c_size_t, ctypes.POINTER(QsObservable), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double)],
    "qs_adjoint_grad_ex": [ctypes.c_void_p, ctypes.POINTER(QsGate), ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                           ctypes.c_size_t, ctypes.POINTER(QsObservable), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(QsExecOpts)],
    "qs_adjoint_describe": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(QsGate), ctypes.c_size_t, ctypes.c_char_p,
                            ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "qs_shard_plan": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(QsGate), ctypes.c_size_t, ctypes.POINTER(QsGate),
                      ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int32)],
    "qs_shard_localize": [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(QsGate), ctypes.c_size_t,
                          ctypes.POINTER(QsGate), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "qs_shard_pack": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "qs_shard_unpack": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "qs_alu_peak": [ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "qs_copy_out": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "qs_copy_out_async": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "qs_sync": [ctypes.c_void_p],
    "qs_copy_in": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
}


def lib() -> ctypes.CDLL:
    """The loaded libqsim.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libqsim.so is not built (run __graft_entry__.build() or "
                           "python -m paper_quant_ph_0201042_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.qs_last_error.argtypes = []
    L.qs_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(st: int) -> None:
    if st != 0:
        raise QsimError(st, lib().qs_last_error().decode(errors="replace"))


def _mat(U) -> ctypes.Array:
    m = np.asarray(U, dtype=np.complex128).reshape(4)
    return (C128 * 4)(*[C128(float(z.real), float(z.imag)) for z in m])


def gates_to_abi(gates: Sequence) -> ctypes.Array:
    """Marshals gate descriptions (objects with kind, target, target2, controls,
    angles, matrix, param) into a qs_gate array."""
    arr = (QsGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        c = arr[i]
        c.kind = KIND_CODES[g.kind]
        c.t = g.target
        c.t2 = g.target2
        c.param = g.param
        cm = cv = 0
        for q, v in g.controls.items():
            cm |= 1 << q
            if v:
                cv |= 1 << q
        c.ctrl_mask = cm
        c.ctrl_val = cv
        for k, a in enumerate(g.angles):
            c.theta[k] = a
        if g.matrix is not None:
            m = np.asarray(g.matrix, dtype=np.complex128).reshape(4)
            for k in range(4):
                c.u[k].re = float(m[k].real)
                c.u[k].im = float(m[k].imag)
    return arr


def _opts(fuse: bool, max_ops: int = 0, arith: str = "default") -> QsExecOpts:
    o = QsExecOpts()
    o.no_fusion = 0 if fuse else 1
    o.max_ops_per_pass = max_ops
    o.c128_arith = ARITH[arith]
    return o


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: libqsim runs only on the GPU")
    return torch


class State:
    """An n-qubit register on the current CUDA device, held in a torch tensor
    (complex64 or complex128, 2^n elements) and wrapped by qs_wrap.  All
    operations are enqueued on the torch stream that is current when the
    state is created (or on `stream`)."""

    def __init__(self, n: int, dtype: str = "c64", tensor=None, stream=None):
        torch = _torch()
        self.n = n
        self.dtype = dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        if tensor is None:
            tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        assert tensor.dtype == tdt and tensor.numel() == (1 << n) and tensor.is_contiguous()
        self.tensor = tensor
        self._h = ctypes.c_void_p()
        check(lib().qs_wrap(ctypes.c_void_p(tensor.data_ptr()), n, DTYPES[dtype], ctypes.byref(self._h)))
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        check(lib().qs_set_stream(self._h, ctypes.c_void_p(s.cuda_stream)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().qs_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # evolution
    def init_basis(self, x: int = 0):
        check(lib().qs_init_basis(self._h, x))
        return self

    def apply_1q(self, q: int, U):
        check(lib().qs_apply_1q(self._h, q, _mat(U)))
        return self

    def apply_ctrl(self, c: int, t: int, U):
        check(lib().qs_apply_ctrl(self._h, c, t, _mat(U)))
        return self

    def apply_mctrl(self, ctrl_mask: int, ctrl_val: int, t: int, U):
        check(lib().qs_apply_mctrl(self._h, ctrl_mask, ctrl_val, t, _mat(U)))
        return self

    def apply_swap(self, a: int, b: int):
        check(lib().qs_apply_swap(self._h, a, b))
        return self

    def apply_gate(self, g):
        arr = gates_to_abi([g])
        check(lib().qs_apply_gate(self._h, arr))
        return self

    def apply_circuit(self, gates: Sequence, fuse: bool = True, max_ops: int = 0, arith: str = "default"):
        """arith (complex128 fused passes): 'default' / 'ds' double-single, 'f64' doubles."""
        arr = gates_to_abi(gates)
        o = _opts(fuse, max_ops, arith)
        check(lib().qs_apply_circuit(self._h, arr, len(gates), ctypes.byref(o)))
        return self

    # reductions (double precision)
    def prob(self, index: int) -> float:
        r = ctypes.c_double()
        check(lib().qs_prob(self._h, index, ctypes.byref(r)))
        return r.value

    def prob_qubit(self, q: int) -> float:
        r = ctypes.c_double()
        check(lib().qs_prob_qubit(self._h, q, ctypes.byref(r)))
        return r.value

    def expect(self, pauli: str) -> float:
        r = ctypes.c_double()
        check(lib().qs_expect(self._h, pauli.encode(), ctypes.byref(r)))
        return r.value

    def inner(self, other: "State") -> complex:
        r = C128()
        check(lib().qs_inner(self._h, other._h, ctypes.byref(r)))
        return complex(r.re, r.im)

    def norm(self) -> float:
        r = ctypes.c_double()
        check(lib().qs_norm(self._h, ctypes.byref(r)))
        return r.value

    def renormalize(self):
        check(lib().qs_renormalize(self._h))
        return self

    def measure(self, r) -> np.ndarray:
        """Outcomes of the measurement gate for the random numbers r in [0, 1)."""
        rr = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1))
        out = np.zeros(max(1, rr.size), dtype=np.uint64)
        check(lib().qs_measure(self._h, rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rr.size,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out[:rr.size]

    def qft(self, q0: int = 0, L: Optional[int] = None, inverse: bool = False) -> "State":
        """QFT (inverse: its adjoint) of qubits q0 .. q0+L-1 by the library's
        FFT (qs_qft); L defaults to n - q0."""
        if L is None:
            L = self.n - q0
        check(lib().qs_qft(self._h, int(q0), int(L), int(bool(inverse))))
        return self

    # host copies
    def to_numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == "c64" else np.complex128)
        check(lib().qs_copy_out(self._h, out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
        return out

    def from_numpy(self, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=np.complex64 if self.dtype == "c64" else np.complex128)
        assert a.size == 1 << self.n
        check(lib().qs_copy_in(self._h, a.ctypes.data_as(ctypes.c_void_p), a.nbytes))
        return self


class Plan:
    """A circuit compiled once (validation, fusion planning) for repeated
    execution on states of n qubits and the given dtype."""

    def __init__(self, n: int, dtype: str, gates: Sequence, fuse: bool = True, max_ops: int = 0,
                 arith: str = "default"):
        self.n = n
        self.dtype = dtype
        arr = gates_to_abi(gates)
        o = _opts(fuse, max_ops, arith)
        self._h = ctypes.c_void_p()
        check(lib().qs_plan_create(n, DTYPES[dtype], arr, len(gates), ctypes.byref(o),
                                   ctypes.byref(self._h)))
        nl = ctypes.c_int64()
        ng = ctypes.c_int64()
        check(lib().qs_plan_info(self._h, ctypes.byref(nl), ctypes.byref(ng)))
        self.launches = nl.value
        self.n_gates = ng.value

    def execute(self, state: State):
        check(lib().qs_plan_execute(state.handle, self._h))
        return state

    def describe(self) -> str:
        need = ctypes.c_size_t()
        check(lib().qs_plan_describe(self._h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        check(lib().qs_plan_describe(self._h, buf, need.value, None))
        return buf.value.decode()

    def set_timing(self, on: bool = True):
        check(lib().qs_plan_set_timing(self._h, 1 if on else 0))

    def timing(self):
        """(summed device ms, launches) of the launches timed since the last read."""
        ms = ctypes.c_double()
        nl = ctypes.c_int64()
        check(lib().qs_plan_timing(self._h, ctypes.byref(ms), ctypes.byref(nl)))
        return ms.value, nl.value

    def close(self):
        if self._h:
            lib().qs_plan_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_trajectories(groups: Sequence, p: float, sigma: float, seed: int, dtype: str = "c64",
                     mode: int = NOISE_FLIPS, every: int = 1, with_stats: bool = True, fuse: bool = True,
                     max_ops: int = 0):
    """Runs batches of noisy trajectories (qs_run_trajectories).

    groups: sequence of dicts with keys n, gates, x0 (array of basis indices),
    first (trajectory id of the first), metric ('fidelity' or 'prob'),
    target (for 'prob') and optionally flags (one byte per gate:
    TRAJ_NO_DEVIATION | TRAJ_NO_FLIPS).  Returns (metric array, stats array of
    shape (T, 4) or None) in group order."""
    keep = []
    arr = (QsTrajGroup * max(1, len(groups)))()
    total = 0
    for k, g in enumerate(groups):
        ga = gates_to_abi(g["gates"])
        x0 = np.ascontiguousarray(g["x0"], dtype=np.uint64)
        keep += [ga, x0]
        c = arr[k]
        c.n = g["n"]
        c.metric = TRAJ_FIDELITY if g.get("metric", "fidelity") == "fidelity" else TRAJ_PROB
        c.target = int(g.get("target", 0))
        c.gates = ga
        c.m = len(g["gates"])
        c.first = int(g["first"])
        c.count = int(x0.size)
        c.x0 = x0.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        if g.get("flags") is not None:
            fl = np.ascontiguousarray(g["flags"], dtype=np.uint8)
            if fl.size != len(g["gates"]):
                raise ValueError("flags: one byte per gate")
            keep.append(fl)
            c.flags = fl.ctypes.data_as(ctypes.c_void_p)
        total += x0.size
    nz = QsNoise(p, sigma, mode, every)
    met = np.zeros(max(1, total), dtype=np.float64)
    st = np.zeros((max(1, total), 4), dtype=np.uint64) if with_stats else None
    opts = _opts(fuse, max_ops)   # same layout as qs_traj_opts
    check(lib().qs_run_trajectories(arr, len(groups), ctypes.byref(nz), seed, DTYPES[dtype], ctypes.byref(opts),
                                    met.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if st is not None else None))
    return met[:total], (st[:total] if st is not None else None)


def alu_peak(kind: str = "f32") -> float:
    """Measured FMA lane operations per second on the current device
    (qs_alu_peak): kind 'f32' or 'f64'."""
    r = ctypes.c_double()
    check(lib().qs_alu_peak({"f32": 0, "f64": 1}[kind], ctypes.byref(r)))
    return r.value


def batch_groups(batch) -> list:
    """Groups of a workloads.TrajectoryBatch in the form run_trajectories takes."""
    out = []
    for k in range(len(batch.widths)):
        f, c = batch.first[k], batch.count[k]
        g = {"n": batch.widths[k], "gates": batch.circuits[k], "x0": batch.x0[f:f + c], "first": f}
        if batch.kinds[k] == "grover":
            g["metric"] = "prob"
            g["target"] = batch.marked[k]
        out.append(g)
    return out


def adjoint_describe(n: int, dtype: str, gates: Sequence) -> str:
    """The fused reverse sweep's host-side plan for these gates (qs_adjoint_describe):
    step lines, then per tile pass its runs of steps.  Needs no GPU."""
    arr = gates_to_abi(gates)
    need = ctypes.c_size_t()
    check(lib().qs_adjoint_describe(n, DTYPES[dtype], arr, len(gates), None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    check(lib().qs_adjoint_describe(n, DTYPES[dtype], arr, len(gates), buf, need.value, None))
    return buf.value.decode()


def adjoint_grad(work: "State", gates: Sequence, params, pauli: Optional[str] = None,
                 ref: Optional["State"] = None, fuse: bool = True):
    """(E, dE/dparams) by the adjoint reverse sweep (qs_adjoint_grad_ex).  E is
    <psi|pauli|psi> or, with ref, |<ref|psi>|^2; psi is the circuit applied to
    |0...0> in `work` with gate angles taken from params by each gate's param
    index.  fuse=False runs one sweep of both vectors per step."""
    arr = gates_to_abi(gates)
    prm = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
    grad = np.zeros(max(1, prm.size))
    val = ctypes.c_double()
    obs = QsObservable()
    if ref is not None:
        obs.kind = OBS_FIDELITY
        obs.ref = ref.handle
    else:
        obs.kind = OBS_PAULI
        obs.pauli = pauli.encode()
    opts = _opts(fuse)
    check(lib().qs_adjoint_grad_ex(work.handle, arr, len(gates), prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   prm.size, ctypes.byref(obs), ctypes.byref(val),
                                   grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts)))
    return val.value, grad[:prm.size]


def _make_adjoint_function():
    import torch

    class AdjointExpectation(torch.autograd.Function):
        """E(params) for a parameterised circuit, differentiated by the
        library's adjoint reverse sweep.  forward(params, work, gates, pauli,
        ref) returns E as a 0-d float64 tensor; backward returns
        grad_output * dE/dparams for params (None for the others)."""

        @staticmethod
        def forward(ctx, params, work, gates, pauli=None, ref=None):
            val, grad = adjoint_grad(work, gates, params.detach().cpu().numpy(), pauli=pauli, ref=ref)
            ctx.save_for_backward(torch.from_numpy(grad).to(params.device, params.dtype))
            return torch.tensor(val, dtype=torch.float64, device=params.device)

        @staticmethod
        def backward(ctx, grad_output):
            (g,) = ctx.saved_tensors
            return grad_output.to(g.dtype) * g, None, None, None, None

    return AdjointExpectation


def __getattr__(name):
    if name == "AdjointExpectation":
        fn = _make_adjoint_function()
        globals()["AdjointExpectation"] = fn
        return fn
    raise AttributeError(name)
