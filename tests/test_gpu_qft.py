"""The QFT as a black-box operator (qs_qft, the FFT of Sec. 2.3.2) against the
oracle's plain double sum, and at full size against the closed form of a
basis state and its own inverse.

Tolerances (||psi_gpu - psi_oracle||_2 of unit vectors): 1e-12 for the
complex128 state; 2e-6 * sqrt(L) for the complex64 state (each radix-2 stage
adds a rounding of relative size ~2^-24 to every amplitude, twiddles come
from double-precision tables rounded once).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _util import random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_quant_ph_0201042_gb300 as qs  # noqa: E402
from paper_quant_ph_0201042_gb300 import build as qbuild  # noqa: E402

qbuild.build()


def tol(dtype, L):
    return 1e-12 if dtype == "c128" else 2e-6 * math.sqrt(L)


# (n, q0, L): one CTA in shared memory (n below a tile), a low pass only, high
# and low passes, sub-registers at the top, middle and bottom of the index,
# L = 1 (a Hadamard), ranges starting on bits 0..7
CASES = [(1, 0, 1), (3, 0, 3), (5, 1, 3), (8, 2, 4), (11, 0, 11), (12, 0, 12), (12, 3, 7),
         (13, 0, 13), (13, 12, 1), (13, 0, 1), (14, 0, 14), (14, 5, 6), (15, 0, 15), (15, 1, 10),
         (15, 2, 13), (16, 9, 4), (17, 3, 8), (17, 0, 5), (18, 0, 9), (18, 9, 9), (19, 4, 15),
         (14, 11, 3), (15, 11, 2), (16, 11, 5), (16, 10, 5)]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,q0,L", CASES)
def test_qft_matches_oracle(dtype, n, q0, L):
    r = W.rng(9000 + 64 * n + 8 * q0 + L)
    psi = random_state(r, n)
    if dtype == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    for inverse in (False, True):
        want = oracle.qft(psi, q0, L, inverse=inverse)
        s = qs.State(n, dtype).from_numpy(psi)
        s.qft(q0, L, inverse=inverse)
        got = s.to_numpy().astype(np.complex128)
        e = float(np.linalg.norm(got - want))
        assert e < tol(dtype, L), (inverse, e)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_qft_equals_fused_circuit(dtype):
    # the black box against the library's own QFT circuit (Sec. 2.3.2) at a
    # size the oracle's double sum cannot reach quickly
    n = 20
    psi = random_state(W.rng(77), n)
    a = qs.State(n, dtype).from_numpy(psi).qft()
    b = qs.State(n, dtype).from_numpy(psi).apply_circuit(W.qft_circuit(n))
    d = (a.tensor.to(torch.complex128) - b.tensor.to(torch.complex128)).abs().pow(2).sum().sqrt().item()
    assert d < (1e-11 if dtype == "c128" else 5e-5), d


def test_qft_edge_cases():
    s = qs.State(6, "c128").init_basis(5)
    for q0, L in ((0, 0), (-1, 2), (4, 3), (0, 7)):
        with pytest.raises(qs.QsimError):
            s.qft(q0, L)
    # L = 1 on any qubit is the Hadamard gate
    psi = random_state(W.rng(4), 6)
    for q in range(6):
        a = qs.State(6, "c128").from_numpy(psi).qft(q, 1).to_numpy()
        b = oracle.run(6, [W.Gate("H", q)], psi=psi)
        assert np.linalg.norm(a - b) < 1e-14


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_qft_n30_full_size(dtype):
    # the paper's largest register (n = 30): QFT of a basis state |x> has
    # amplitudes 2^-15 e^{2 pi i x y / 2^30}; sampled outputs against that
    # closed form, then the inverse transform returns |x>
    n = 30
    x = W.basis_index(30030, n)
    s = qs.State(n, dtype).init_basis(x)
    s.qft()
    ys = np.concatenate([np.arange(64), W.rng(5).integers(0, 1 << n, size=4000), [(1 << n) - 1]]).astype(np.int64)
    got = s.tensor[torch.from_numpy(ys).to(s.tensor.device)].cpu().numpy().astype(np.complex128)
    e = (x * ys.astype(object)) % (1 << n)
    want = np.array([complex(math.cos(2 * math.pi * v / (1 << n)), math.sin(2 * math.pi * v / (1 << n)))
                     for v in e]) * 2.0 ** -15
    rel = np.max(np.abs(got - want)) / 2.0 ** -15
    assert rel < (1e-12 if dtype == "c128" else 1e-5), rel
    s.qft(inverse=True)
    assert abs(s.prob(x) - 1) < (1e-12 if dtype == "c128" else 1e-5)
    assert abs(s.norm() - 1) < (1e-12 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,eps", [(12, 1e-2), (16, 1e-3)])
def test_approximate_qft_circuit(dtype, n, eps):
    # the approximate QFT of Sec. 2.3.2 (phase shifts with k > ceil(log2(n /
    # eps)) left out) through the fused planner, against the oracle's gate by
    # gate run of the same circuit, and within the dropped gates' bound of the
    # exact transform (the black box)
    mk = W.approx_qft_max_k(n, eps)
    approx = W.qft_circuit(n, max_k=mk)
    assert len(approx) < len(W.qft_circuit(n))
    psi = random_state(W.rng(4200 + n), n)
    if dtype == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    want = oracle.run(n, approx, psi=psi)
    got = qs.State(n, dtype).from_numpy(psi).apply_circuit(approx).to_numpy().astype(np.complex128)
    assert np.linalg.norm(got - want) < (1e-12 if dtype == "c128" else 1e-5)
    exact = qs.State(n, dtype).from_numpy(psi).qft().to_numpy().astype(np.complex128)
    dropped = sum(1 for j in range(n) for k in range(mk + 1, n - j + 1))
    bound = sum(2 * math.pi / (1 << k) for j in range(n) for k in range(mk + 1, n - j + 1))
    assert dropped > 0 and np.linalg.norm(got - exact) <= bound + 1e-5
