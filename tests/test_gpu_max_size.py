"""The largest registers one GB300 holds, and allocation failure.

A 34-qubit complex64 register is 128 GiB (the part has 284 GiB); the fused
passes, the FFT and the reductions use 64-bit indices throughout.  The oracle
cannot run at this size, so the checks are properties that hold at any size:
a circuit followed by its inverse returns |0...0>, the norm stays 1, and the
QFT of a basis state has the closed-form amplitudes of Sec. 2.3.2.
"""
import ctypes
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_quant_ph_0201042_gb300 as qs  # noqa: E402
from paper_quant_ph_0201042_gb300 import build as qbuild  # noqa: E402

qbuild.build()

N_MAX = 34


def inverse(gates):
    out = []
    for g in reversed(gates):
        if g.kind == "MATRIX":
            out.append(W.Gate("MATRIX", g.target, controls=dict(g.controls), matrix=np.conj(g.matrix).T))
        else:
            out.append(g)      # X, C-NOT and SWAP are their own inverses
    return out


def test_n34_circuit_and_inverse():
    free, _ = torch.cuda.mem_get_info()
    if free < (140 << 30):
        pytest.skip("needs 140 GiB of free device memory")
    n = N_MAX
    gates = W.random_circuit(n, 3, seed=34)
    s = qs.State(n, "c64").init_basis(0)
    s.apply_circuit(gates)
    assert abs(s.norm() - 1) < 1e-4
    p1 = [s.prob_qubit(q) for q in (0, n // 2, n - 1)]
    assert all(0.0 < p < 1.0 for p in p1)
    s.apply_circuit(inverse(gates))
    assert abs(s.prob(0) - 1) < 1e-4
    # QFT of a basis state: sampled amplitudes against the closed form, then back
    x = W.basis_index(3434, n)
    s.init_basis(x).qft()
    ys = np.concatenate([np.arange(16), W.rng(6).integers(0, 1 << n, size=1000)]).astype(np.int64)
    got = s.tensor[torch.from_numpy(ys).to(s.tensor.device)].cpu().numpy().astype(np.complex128)
    e = (x * ys.astype(object)) % (1 << n)
    want = np.array([complex(math.cos(2 * math.pi * v / (1 << n)), math.sin(2 * math.pi * v / (1 << n)))
                     for v in e]) * 2.0 ** (-n / 2)
    assert np.max(np.abs(got - want)) * 2.0 ** (n / 2) < 2e-5
    s.qft(inverse=True)
    assert abs(s.prob(x) - 1) < 1e-4
    s.close()
    del s
    torch.cuda.empty_cache()


def test_allocation_failure_is_an_error_status():
    # 2^39 complex64 amplitudes (4 TiB) cannot be allocated: QS_ENOMEM, no fault
    h = ctypes.c_void_p()
    st = qs.lib().qs_alloc(39, 1, ctypes.byref(h))
    assert st == 3, st
    assert b"alloc" in qs.lib().qs_last_error().lower()
    # above QS_MAX_QUBITS: QS_ERANGE before any allocation
    st = qs.lib().qs_alloc(41, 1, ctypes.byref(h))
    assert st == 2, st
    # the device still works
    t = qs.State(10, "c64").init_basis(5)
    assert abs(t.prob(5) - 1) < 1e-12
