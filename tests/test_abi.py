"""The C ABI library loads and exports every entry point include/qsim.h
declares; the Python binding marshals gates without a GPU.  No compute call is
made here (there may be no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_quant_ph_0201042_gb300 as qs
from paper_quant_ph_0201042_gb300 import build as qbuild
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    return qbuild.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["qs_alloc", "qs_wrap", "qs_free", "qs_set_stream", "qs_init_basis",
                     "qs_apply_1q", "qs_apply_ctrl", "qs_apply_mctrl", "qs_apply_swap",
                     "qs_apply_circuit", "qs_prob", "qs_prob_qubit", "qs_expect", "qs_inner",
                     "qs_norm", "qs_copy_out", "qs_copy_in", "qs_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = declared_functions() - {"qs_last_error"}
    assert names <= set(qs._SIGS), names - set(qs._SIGS)


def test_last_error_is_callable_without_gpu(libpath):
    L = qs.lib()
    assert isinstance(L.qs_last_error(), bytes)


def test_argument_errors_without_gpu(libpath):
    # validation happens before any CUDA call
    L = qs.lib()
    h = ctypes.c_void_p()
    assert L.qs_alloc(0, qs.QS_C64, ctypes.byref(h)) == 2          # QS_ERANGE
    assert L.qs_alloc(41, qs.QS_C64, ctypes.byref(h)) == 2
    assert L.qs_alloc(5, 7, ctypes.byref(h)) == 1                   # QS_EINVAL
    assert L.qs_wrap(None, 5, qs.QS_C64, ctypes.byref(h)) == 1
    assert L.qs_wrap(ctypes.c_void_p(8), 5, qs.QS_C64, ctypes.byref(h)) == 1   # misaligned
    assert b"aligned" in L.qs_last_error()
    bad = qs.gates_to_abi([W.Gate("X", 2, controls={2: 1})])
    p = ctypes.c_void_p()
    assert L.qs_plan_create(4, qs.QS_C64, bad, 1, None, ctypes.byref(p)) == 1
    assert b"control" in L.qs_last_error()
    bad = qs.gates_to_abi([W.Gate("H", 4)])
    assert L.qs_plan_create(4, qs.QS_C64, bad, 1, None, ctypes.byref(p)) == 1
    bad = qs.gates_to_abi([W.Gate("SWAP", 1, target2=1)])
    assert L.qs_plan_create(4, qs.QS_C64, bad, 1, None, ctypes.byref(p)) == 1


def test_new_entry_points_validate_without_gpu(libpath):
    L = qs.lib()
    buf = ctypes.create_string_buffer(16)
    assert L.qs_copy_out_async(None, buf, 16) == 1                  # QS_EINVAL
    assert L.qs_sync(None) == 1
    need = ctypes.c_size_t()
    g = qs.gates_to_abi([W.Gate("H", 0)])
    assert L.qs_adjoint_describe(0, qs.QS_C64, g, 1, None, 0, ctypes.byref(need)) == 2     # QS_ERANGE
    assert L.qs_adjoint_describe(41, qs.QS_C64, g, 1, None, 0, ctypes.byref(need)) == 2
    assert L.qs_adjoint_describe(4, 9, g, 1, None, 0, ctypes.byref(need)) == 1             # bad dtype
    assert L.qs_adjoint_describe(4, qs.QS_C64, None, 1, None, 0, ctypes.byref(need)) == 1
    bad = qs.gates_to_abi([W.Gate("H", 4)])                                                 # target out of range
    assert L.qs_adjoint_describe(4, qs.QS_C64, bad, 1, None, 0, ctypes.byref(need)) != 0
    # a parameter on a gate kind without angles
    bad = qs.gates_to_abi([W.Gate("H", 1, param=0)])
    assert L.qs_adjoint_describe(4, qs.QS_C64, bad, 1, None, 0, ctypes.byref(need)) == 6   # QS_EUNSUPPORTED
    # an empty circuit describes itself as nothing, a truncated buffer stays NUL-terminated
    assert L.qs_adjoint_describe(8, qs.QS_C64, None, 0, None, 0, ctypes.byref(need)) == 0 and need.value == 1
    text = qs.adjoint_describe(8, "c64", W.ansatz_circuit(8, 1, seed=2)[0])
    small = ctypes.create_string_buffer(10)
    assert L.qs_adjoint_describe(8, qs.QS_C64, qs.gates_to_abi(W.ansatz_circuit(8, 1, seed=2)[0]), 23, small, 10,
                                 None) == 0
    assert small.value.decode() == text[:9]


def test_plans_build_without_gpu(libpath):
    # planning is host-only: a fused plan of the 30-qubit random circuit
    gates = W.random_circuit(30, 2, seed=1)
    p = qs.Plan(30, "c64", gates)
    assert p.n_gates == len(gates)
    assert 1 <= p.launches < len(gates)
    u = qs.Plan(30, "c64", gates, fuse=False)
    assert u.launches == len(gates)
    q = qs.Plan(10, "c128", W.qft_circuit(10))
    assert q.launches >= 1


def test_gate_struct_layout():
    arr = qs.gates_to_abi([W.Gate("UP1", 3, controls={1: 1, 5: 0}, angles=(0.25,), param=7)])
    g = arr[0]
    assert g.kind == 5 and g.t == 3 and g.param == 7
    assert g.ctrl_mask == (1 << 1) | (1 << 5) and g.ctrl_val == 1 << 1
    assert g.theta[0] == 0.25


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without libqsim.so every entry point raises
    monkeypatch.setattr(qs, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(qs, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        qs.lib()
    with pytest.raises(RuntimeError, match="not built|no CUDA device"):
        qs.State(4, "c64")


def test_plans_schedule_fewer_transposes_than_program_order(libpath):
    # the list scheduler keeps a pass's ops within their commutation freedom
    # and needs fewer transposes than program order would
    import re
    d = qs.Plan(28, "c64", W.random_circuit(28, 40, seed=20260515)).describe()
    xp = sum(int(v) for v in re.findall(r"xpose=(\d+)", d))
    passes = len(re.findall(r"^pass ", d, flags=re.M))
    assert passes > 0 and xp < 1.6 * passes, (xp, passes)


def test_norm_noalloc_rejects_bad_arguments_without_launching(libpath):
    # every check runs on the host before any CUDA call, so fake device
    # pointers are safe here: nothing is dereferenced or launched
    L = qs.lib()
    ok_state, ok_out = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 21)
    assert L.qs_norm_noalloc(ok_state, 0, qs.QS_C64, ok_out, None) == 2            # QS_ERANGE: n < 1
    assert L.qs_norm_noalloc(ok_state, 33, qs.QS_C128, ok_out, None) == 2          # QS_ERANGE: n > 32
    assert L.qs_norm_noalloc(None, 10, qs.QS_C64, ok_out, None) == 1               # QS_EINVAL: NULL state
    assert L.qs_norm_noalloc(ok_state, 10, qs.QS_C64, None, None) == 1             # QS_EINVAL: NULL result
    assert L.qs_norm_noalloc(ok_state, 10, 7, ok_out, None) == 1                   # QS_EINVAL: bad dtype
    # misaligned pointers: a complex128 state needs 16 bytes, complex64 8, the result 8
    assert L.qs_norm_noalloc(ctypes.c_void_p((1 << 20) + 8), 10, qs.QS_C128, ok_out, None) == 1
    assert b"16-byte" in L.qs_last_error()
    assert L.qs_norm_noalloc(ctypes.c_void_p((1 << 20) + 4), 10, qs.QS_C64, ok_out, None) == 1
    assert b"8-byte" in L.qs_last_error()
    assert L.qs_norm_noalloc(ok_state, 10, qs.QS_C64, ctypes.c_void_p((1 << 21) + 4), None) == 1
    assert b"dev_out" in L.qs_last_error()
