"""CPU oracle for the state-vector method of quant-ph/0201042 (complex128).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline / reference leg of bench.py, never by the product package.  It
shares no code with the CUDA library; both consume the circuit descriptions of
the `workloads` module.

The arithmetic lives in qs_oracle.c (plain C, double complex, out-of-place
row-by-row gate application); this file compiles it with gcc and exposes it
through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libqs_oracle.so")

KIND_CODES = {
    "MATRIX": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "UP1": 5, "UP2": 6,
    "UR": 7, "URP1": 8, "RY": 9, "RZ": 10, "SWAP": 11,
}
NOISE_FLIPS = 0
NOISE_DEPOLARIZING = 1


class OrGate(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("target", ctypes.c_int32),
        ("target2", ctypes.c_int32),
        ("param", ctypes.c_int32),
        ("ctrl_mask", ctypes.c_uint64),
        ("ctrl_val", ctypes.c_uint64),
        ("angle", ctypes.c_double * 2),
        ("m", ctypes.c_double * 8),
    ]


class OrNoise(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("mode", ctypes.c_int32),
        ("every", ctypes.c_int32),
    ]


# -O3 without contraction: every C operation rounds once, the same on x86 and
# Arm hosts (no -march=native: the library and the oracle are built on
# machines of both kinds and must give the same numbers there).
CFLAGS = ["-O3", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-D_DEFAULT_SOURCE"]


def build(force: bool = False) -> str:
    """Compiles qs_oracle.c into _build/libqs_oracle.so (OpenMP when available)."""
    stamp = _LIB_PATH + ".flags"
    flags = " ".join(CFLAGS)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC) and \
            os.path.exists(stamp) and open(stamp).read() == flags:
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    with open(stamp, "w") as f:
        f.write(flags)
    return _LIB_PATH


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    L = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    gp = ctypes.POINTER(OrGate)
    L.or_apply_gate.argtypes = [dp, ctypes.c_int, gp]
    L.or_apply_circuit.argtypes = [dp, ctypes.c_int, gp, ctypes.c_int64]
    L.or_init_basis.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
    L.or_norm2.argtypes = [dp, ctypes.c_int]
    L.or_norm2.restype = ctypes.c_double
    L.or_prob.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
    L.or_prob.restype = ctypes.c_double
    L.or_prob_qubit.argtypes = [dp, ctypes.c_int, ctypes.c_int]
    L.or_prob_qubit.restype = ctypes.c_double
    L.or_inner.argtypes = [dp, dp, ctypes.c_int, dp]
    L.or_expect_pauli.argtypes = [dp, ctypes.c_int, ctypes.c_char_p]
    L.or_expect_pauli.restype = ctypes.c_double
    L.or_measure.argtypes = [dp, ctypes.c_int, ctypes.c_double]
    L.or_measure.restype = ctypes.c_uint64
    L.or_qft_dft.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.or_gate_matrix.argtypes = [ctypes.c_int, dp, dp, dp]
    L.or_gate_n_angles.argtypes = [ctypes.c_int]
    L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                   ctypes.POINTER(ctypes.c_uint32)]
    L.or_flip_threshold.argtypes = [ctypes.c_double]
    L.or_flip_threshold.restype = ctypes.c_uint32
    L.or_gauss.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
    L.or_gauss.restype = ctypes.c_double
    L.or_run_trajectory.argtypes = [dp, ctypes.c_int, gp, ctypes.c_int64, ctypes.POINTER(OrNoise),
                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
    L.or_cost.argtypes = [ctypes.c_int, gp, ctypes.c_int64, dp, ctypes.c_char_p, dp]
    L.or_cost.restype = ctypes.c_double
    L.or_gradient.argtypes = [ctypes.c_int, gp, ctypes.c_int64, dp, ctypes.c_int64, ctypes.c_char_p,
                              dp, ctypes.c_int, ctypes.c_double, dp]
    L.or_num_threads.restype = ctypes.c_int
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gates_to_c(gates: Sequence) -> ctypes.Array:
    """Translates workloads.Gate descriptions into the oracle's gate array."""
    arr = (OrGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        c = arr[i]
        c.kind = KIND_CODES[g.kind]
        c.target = g.target
        c.target2 = g.target2
        c.param = g.param
        c.ctrl_mask = g.ctrl_mask()
        c.ctrl_val = g.ctrl_val()
        for k, a in enumerate(g.angles):
            c.angle[k] = a
        if g.matrix is not None:
            m = np.asarray(g.matrix, dtype=np.complex128).reshape(4)
            for k in range(4):
                c.m[2 * k] = m[k].real
                c.m[2 * k + 1] = m[k].imag
    return arr


def basis(n: int, x: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    lib().or_init_basis(_dp(psi.view(np.float64)), n, x)
    return psi


def run(n: int, gates: Sequence, psi: Optional[np.ndarray] = None, x0: int = 0) -> np.ndarray:
    """Applies the circuit to psi (a copy) or to |x0>; returns the new state."""
    if psi is None:
        psi = basis(n, x0)
    else:
        psi = np.array(psi, dtype=np.complex128, copy=True)
    if len(gates):
        rc = lib().or_apply_circuit(_dp(psi.view(np.float64)), n, gates_to_c(gates), len(gates))
        if rc != 0:
            raise ValueError("oracle: invalid gate in circuit")
    return psi


def gate_matrix(g) -> np.ndarray:
    c = gates_to_c([g])[0]
    out = np.zeros(8)
    lib().or_gate_matrix(c.kind, ctypes.cast(c.angle, ctypes.POINTER(ctypes.c_double)),
                         ctypes.cast(c.m, ctypes.POINTER(ctypes.c_double)), _dp(out))
    return out.view(np.complex128).reshape(2, 2)


def norm2(psi: np.ndarray) -> float:
    n = int(np.log2(psi.size))
    return lib().or_norm2(_dp(np.ascontiguousarray(psi).view(np.float64)), n)


def prob(psi: np.ndarray, index: int) -> float:
    n = int(np.log2(psi.size))
    return lib().or_prob(_dp(np.ascontiguousarray(psi).view(np.float64)), n, index)


def prob_qubit(psi: np.ndarray, q: int) -> float:
    n = int(np.log2(psi.size))
    return lib().or_prob_qubit(_dp(np.ascontiguousarray(psi).view(np.float64)), n, q)


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    n = int(np.log2(a.size))
    out = np.zeros(2)
    lib().or_inner(_dp(np.ascontiguousarray(a).view(np.float64)),
                   _dp(np.ascontiguousarray(b).view(np.float64)), n, _dp(out))
    return complex(out[0], out[1])


def expect_pauli(psi: np.ndarray, pauli: str) -> float:
    n = int(np.log2(psi.size))
    assert len(pauli) == n
    return lib().or_expect_pauli(_dp(np.ascontiguousarray(psi).view(np.float64)), n,
                                 pauli.encode())


def measure(psi: np.ndarray, r: float) -> int:
    n = int(np.log2(psi.size))
    return int(lib().or_measure(_dp(np.ascontiguousarray(psi).view(np.float64)), n, r))


def qft(psi: np.ndarray, q0: int = 0, L: Optional[int] = None, inverse: bool = False) -> np.ndarray:
    """QFT (or its inverse) of qubits q0 .. q0+L-1 by the plain double sum of
    Sec. 2.3.2; returns a new vector."""
    n = int(np.log2(psi.size))
    if L is None:
        L = n - q0
    out = np.array(psi, dtype=np.complex128, copy=True)
    if lib().or_qft_dft(_dp(out.view(np.float64)), n, q0, L, int(bool(inverse))) != 0:
        raise ValueError("or_qft_dft: bad arguments")
    return out


def philox(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def flip_threshold(p: float) -> int:
    return int(lib().or_flip_threshold(p))


def gauss(seed: int, traj: int, step: int, a: int) -> float:
    return lib().or_gauss(seed, traj, step, a)


NO_DEVIATION = 1   # gate flag: its angles are not deviated
NO_FLIPS = 2       # gate flag: no flips after it


def run_trajectory(n: int, gates: Sequence, p: float, sigma: float, seed: int, traj: int,
                   x0: int, mode: int = NOISE_FLIPS, every: int = 1, flags=None):
    """One noisy trajectory (Sec. 3 error model); returns (state, stats) with
    stats = [#X flips, #Y flips, #Z flips, event fingerprint].  Decoherence acts after
    gate step s when (s + 1) % every == 0 and flags[s] lacks NO_FLIPS."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    nz = OrNoise(p, sigma, mode, every)
    st = (ctypes.c_uint64 * 4)()
    fl = None
    if flags is not None:
        fl = np.ascontiguousarray(flags, dtype=np.uint8)
        assert fl.size == len(gates)
    rc = lib().or_run_trajectory(_dp(psi.view(np.float64)), n, gates_to_c(gates), len(gates),
                                 ctypes.byref(nz), seed, traj, x0, st,
                                 fl.ctypes.data_as(ctypes.c_void_p) if fl is not None else None)
    if rc != 0:
        raise ValueError("oracle: invalid gate in trajectory circuit")
    return psi, np.array(list(st), dtype=np.uint64)


def cost(n: int, gates: Sequence, params: np.ndarray, pauli: Optional[str] = None,
         ref: Optional[np.ndarray] = None) -> float:
    params = np.ascontiguousarray(params, dtype=np.float64)
    refp = _dp(np.ascontiguousarray(ref).view(np.float64)) if ref is not None else None
    return lib().or_cost(n, gates_to_c(gates), len(gates), _dp(params),
                         pauli.encode() if pauli else None, refp)


def gradient(n: int, gates: Sequence, params: np.ndarray, pauli: Optional[str] = None,
             ref: Optional[np.ndarray] = None, method: str = "shift", h: float = 1e-4) -> np.ndarray:
    """d cost / d params by the parameter-shift rule (method='shift') or central
    finite differences (method='fd', step h)."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    grad = np.zeros(params.size)
    refp = _dp(np.ascontiguousarray(ref).view(np.float64)) if ref is not None else None
    rc = lib().or_gradient(n, gates_to_c(gates), len(gates), _dp(params), params.size,
                           pauli.encode() if pauli else None, refp,
                           0 if method == "shift" else 1, h, _dp(grad))
    if rc != 0:
        raise ValueError("oracle: a gate parameter index beyond the parameter vector")
    return grad


def num_threads() -> int:
    return int(lib().or_num_threads())
