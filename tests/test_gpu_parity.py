"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (||psi_gpu - psi_oracle||_2): 1e-12 for the complex128 state and
1e-5 for the complex64 state at depth <= 500, the bounds the workloads fix;
longer circuits state their own bound in the test.  Reductions accumulate in
double precision on both sides.

Fused complex128 passes run in double-single arithmetic by default (each
double split into two floats, 48 significant bits, error-free products and
sums); the tests run them and the double-precision passes ("f64") against the
same bounds.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _util import random_gate, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_quant_ph_0201042_gb300 as qs  # noqa: E402
from paper_quant_ph_0201042_gb300 import build as qbuild  # noqa: E402
from paper_quant_ph_0201042_gb300 import paper  # noqa: E402

qbuild.build()

TOL = {"c128": 1e-12, "c64": 1e-5}
DTYPES = ["c128", "c64"]


def gpu_run(n, gates, dtype, fuse=True, x0=0, psi=None, max_ops=0, arith="default"):
    s = qs.State(n, dtype)
    if psi is not None:
        s.from_numpy(psi)
    else:
        s.init_basis(x0)
    s.apply_circuit(gates, fuse=fuse, max_ops=max_ops, arith=arith)
    out = s.to_numpy().astype(np.complex128)
    s.close()
    return out


def err(a, b):
    return float(np.linalg.norm(a - b))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_unfused_gates_every_kind(dtype, n):
    r = W.rng(1000 + n)
    gates = [random_gate(r, n) for _ in range(60)]
    psi = random_state(r, n)
    want = oracle.run(n, gates, psi=psi)
    s = qs.State(n, dtype).from_numpy(psi)
    for g in gates:
        s.apply_gate(g)
    got = s.to_numpy().astype(np.complex128)
    assert err(got, want) < TOL[dtype]


@pytest.mark.parametrize("arith", ["default", "f64"])
@pytest.mark.parametrize("n", [2, 7, 12])
def test_unfused_circuit_complex128_arithmetic(arith, n):
    # the per-gate sweeps of a complex128 state in double-single (default) and
    # in double-precision instructions, every gate kind, against the oracle
    r = W.rng(3000 + n)
    gates = [random_gate(r, n) for _ in range(80)]
    psi = random_state(r, n)
    want = oracle.run(n, gates, psi=psi)
    assert err(gpu_run(n, gates, "c128", fuse=False, psi=psi, arith=arith), want) < TOL["c128"]


@pytest.mark.parametrize("dtype", DTYPES)
def test_entry_points(dtype):
    n = 9
    r = W.rng(77)
    psi = random_state(r, n)
    s = qs.State(n, dtype).from_numpy(psi)
    ref = psi.copy()
    U = W.haar_su2(r)
    for q in [0, 4, 8]:
        s.apply_1q(q, U)
        ref = oracle.run(n, [W.Gate("MATRIX", q, matrix=U)], psi=ref)
    s.apply_ctrl(2, 7, U)
    ref = oracle.run(n, [W.Gate("MATRIX", 7, controls={2: 1}, matrix=U)], psi=ref)
    s.apply_ctrl(8, 0, U)
    ref = oracle.run(n, [W.Gate("MATRIX", 0, controls={8: 1}, matrix=U)], psi=ref)
    s.apply_mctrl((1 << 1) | (1 << 3) | (1 << 6), 1 << 3, 5, U)
    ref = oracle.run(n, [W.Gate("MATRIX", 5, controls={1: 0, 3: 1, 6: 0}, matrix=U)], psi=ref)
    s.apply_swap(1, 8)
    ref = oracle.run(n, [W.Gate("SWAP", 1, target2=8)], psi=ref)
    assert err(s.to_numpy().astype(np.complex128), ref) < TOL[dtype]


# (dtype, arithmetic of the fused complex128 passes)
VARIANTS = [("c128", "ds"), ("c128", "f64"), ("c64", "default")]


@pytest.mark.parametrize("dtype,arith", VARIANTS)
@pytest.mark.parametrize("n", [9, 10, 11, 12, 13, 14, 16, 17])
def test_fused_random_circuits(dtype, arith, n):
    r = W.rng(2000 + n)
    for trial in range(3):
        gates = [random_gate(r, n) for _ in range(150)]
        psi = random_state(r, n)
        want = oracle.run(n, gates, psi=psi)
        got = gpu_run(n, gates, dtype, fuse=True, psi=psi, arith=arith)
        assert err(got, want) < TOL[dtype], trial


@pytest.mark.parametrize("dtype,arith", VARIANTS)
@pytest.mark.parametrize("max_ops", [4, 7, 16])
def test_fused_small_passes(dtype, arith, max_ops):
    # many short passes, transposes at pass edges
    n = 13
    r = W.rng(31 + max_ops)
    gates = [random_gate(r, n, max_ctrl=2) for _ in range(120)]
    psi = random_state(r, n)
    want = oracle.run(n, gates, psi=psi)
    got = gpu_run(n, gates, dtype, fuse=True, psi=psi, max_ops=max_ops, arith=arith)
    assert err(got, want) < TOL[dtype]


@pytest.mark.parametrize("dtype,arith", VARIANTS)
def test_fused_high_qubit_only_and_lane_only(dtype, arith):
    n = 15
    r = W.rng(5)
    psi = random_state(r, n)
    high = [W.Gate("MATRIX", q, matrix=W.haar_su2(r)) for q in range(0, 10)] * 3
    lane = [W.Gate("MATRIX", q, matrix=W.haar_su2(r)) for q in range(10, 15)] * 3
    for gates in (high, lane, high + lane + high):
        want = oracle.run(n, gates, psi=psi)
        assert err(gpu_run(n, gates, dtype, psi=psi, arith=arith), want) < TOL[dtype]


@pytest.mark.parametrize("dtype,arith", VARIANTS)
def test_fused_every_gate_class(dtype, arith):
    # every kind with controls inside and outside the tile, Hadamard
    # butterflies (an odd count, so the folded factor is not a power of two),
    # diagonal gates with an exact-1 entry, SWAPs; a random state so that no
    # amplitude is zero
    n = 14
    r = W.rng(606)
    psi = random_state(r, n)
    gates = [random_gate(r, n, max_ctrl=2) for _ in range(200)]
    gates += [W.Gate("H", q) for q in (0, 3, 9, 12, 13)]
    gates += [W.Gate("UP1", q, angles=(0.3 * q,), controls={(q + 5) % n: 1}) for q in range(n)]
    want = oracle.run(n, gates, psi=psi)
    assert err(gpu_run(n, gates, dtype, psi=psi, arith=arith), want) < TOL[dtype]


def test_qft_n10_closed_form():
    # the QFT workload: a seeded basis state |x>, x uniform in [0, 1024), complex128
    n = 10
    x = W.basis_index(20260101, n)
    e = np.zeros(1 << n, dtype=complex)
    e[x] = 1
    closed = np.fft.ifft(e) * math.sqrt(1 << n)
    want = oracle.run(n, W.qft_circuit(n), x0=x)
    for fuse in (True, False):
        got = gpu_run(n, W.qft_circuit(n), "c128", fuse=fuse, x0=x)
        assert err(got, want) < 1e-12
        assert err(got, closed) < 1e-12
    got = gpu_run(n, W.qft_circuit(n), "c64", x0=x)
    assert err(got, closed) < 1e-5


@pytest.mark.parametrize("dtype", DTYPES)
def test_reductions(dtype):
    n = 12
    r = W.rng(9)
    psi = random_state(r, n)
    phi = random_state(r, n)
    if dtype == "c64":   # both sides reduce the same single-precision inputs
        psi = psi.astype(np.complex64).astype(np.complex128)
        phi = phi.astype(np.complex64).astype(np.complex128)
    a = qs.State(n, dtype).from_numpy(psi)
    b = qs.State(n, dtype).from_numpy(phi)
    assert abs(a.norm() - oracle.norm2(psi)) < 1e-12
    for idx in [0, 1, 777, (1 << n) - 1]:
        assert abs(a.prob(idx) - oracle.prob(psi, idx)) < 1e-15
    for q in range(n):
        assert abs(a.prob_qubit(q) - oracle.prob_qubit(psi, q)) < 1e-12
    for _ in range(12):
        p = "".join(r.choice(list("IXYZ"), size=n))
        assert abs(a.expect(p) - oracle.expect_pauli(psi, p)) < 1e-12, p
    # flips on the lowest and the highest index bit, an odd and an even number
    # of Y factors (the pair terms add to a real or to an imaginary part)
    for p in ["X" + "I" * (n - 1), "I" * (n - 1) + "Y", "Y" + "Z" * (n - 1), "XY" + "I" * (n - 2), "YY" + "Z" * (n - 2)]:
        assert abs(a.expect(p) - oracle.expect_pauli(psi, p)) < 1e-12, p
    assert abs(a.inner(b) - oracle.inner(psi, phi)) < 1e-12
    a.renormalize()
    assert abs(a.norm() - 1) < (1e-14 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("dtype", DTYPES)
def test_grover_n12_full_state(dtype):
    n = 12
    k = W.basis_index(4242, n)
    it = W.grover_iterations(n)
    gates = W.grover_circuit(n, k, it)
    want = oracle.run(n, gates)
    got = gpu_run(n, gates, dtype)
    assert err(got, want) < (1e-11 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype", DTYPES)
def test_grover_n24_success_probability(dtype):
    # the Grover workload: n = 24, floor(pi/4 sqrt(2^24)) = 3216 iterations; success
    # probability against sin^2((2k+1) theta), sin theta = 2^-12
    n = 24
    k = W.basis_index(24, n)
    it = W.grover_iterations(n)
    assert it == 3216
    # complex64: a double-precision renormalisation every 256 iterations
    search = paper.GroverSearch(n, k, it, dtype)
    s = search.run(qs.State(n, dtype))
    th = math.asin(2.0 ** (-n / 2))
    want = math.sin((2 * it + 1) * th) ** 2
    assert want == search.closed_form()
    p = s.prob(k)
    tol = 1e-9 if dtype == "c128" else 1e-5
    assert abs(p - want) < tol, (p, want)
    assert p <= 1 + 1e-7
    assert abs(s.norm() - 1) < (1e-9 if dtype == "c128" else 1e-5)


def test_grover_n24_complex64_drifts_without_renormalisation():
    # the same search as one plan, no renormalisation: the norm drifts by
    # the accumulated single-precision rounding, which the renormalising run
    # above removes
    n = 24
    k = W.basis_index(24, n)
    it = W.grover_iterations(n)
    s = paper.GroverSearch(n, k, it, "c64", renorm_every=0).run(qs.State(n, "c64"))
    drift = abs(s.norm() - 1)
    assert 1e-7 < drift < 1e-3, drift


@pytest.mark.parametrize("dtype,arith", VARIANTS)
def test_random_circuit_n20_oracle(dtype, arith):
    # the 40-layer random circuit of the throughput workload at n = 20
    n = 20
    gates = W.random_circuit(n, 40, seed=7)
    want = oracle.run(n, gates)
    got = gpu_run(n, gates, dtype, arith=arith)
    assert err(got, want) < TOL[dtype]


@pytest.fixture(scope="module")
def oracle_n26():
    # the throughput workload's generator at n = 26, 10 layers (390 gates):
    # the largest register the oracle runs in test time (1 GiB complex128)
    n = 26
    gates = W.random_circuit(n, 10, seed=11)
    return n, gates, oracle.run(n, gates)


@pytest.mark.parametrize("dtype,arith", VARIANTS)
def test_random_circuit_n26_oracle(oracle_n26, dtype, arith):
    n, gates, want = oracle_n26
    got = gpu_run(n, gates, dtype, arith=arith)
    assert err(got, want) < TOL[dtype]


def test_random_circuit_n30_full_size():
    # the throughput workload at full size, in the benchmark's launch
    # configuration; the oracle cannot run it in test time, so: the complex64
    # state against the complex128 state, norms, and the inverse circuit
    n = 30
    gates = W.random_circuit(n, 40, seed=1)
    p64 = qs.Plan(n, "c64", gates)
    s64 = qs.State(n, "c64").init_basis(0)
    p64.execute(s64)
    assert abs(s64.norm() - 1) < 1e-4
    s128 = qs.State(n, "c128").init_basis(0)
    qs.Plan(n, "c128", gates).execute(s128)
    assert abs(s128.norm() - 1) < 1e-11
    d = (s64.tensor.to(torch.complex128) - s128.tensor).abs().pow(2).sum().sqrt().item()
    assert d < 1e-5, d
    del s64
    # U^dagger U |0> = |0>
    inv = []
    for g in reversed(gates):
        if g.kind == "MATRIX":
            inv.append(W.Gate("MATRIX", g.target, matrix=np.conj(g.matrix).T))
        else:
            inv.append(g)
    qs.Plan(n, "c128", inv).execute(s128)
    assert abs(s128.prob(0) - 1) < 1e-10


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_qft_n30_closed_form_sampled(dtype):
    # the fused passes at the throughput workload's size (n = 30, the bench's
    # launch configuration: the default fused plan) on a circuit with a
    # closed form: the QFT circuit of a basis state |x>, whose output
    # amplitudes are 2^{-n/2} e^{2 pi i x y / 2^n}, checked on sampled y
    n = 30
    x = W.basis_index(30030, n)
    s = qs.State(n, dtype).init_basis(x)
    qs.Plan(n, dtype, W.qft_circuit(n)).execute(s)
    r = W.rng(17)
    ys = np.concatenate([[0, 1, (1 << n) - 1], r.integers(0, 1 << n, size=61)]).astype(np.int64)
    got = s.tensor[torch.from_numpy(ys).to("cuda")].cpu().numpy().astype(np.complex128)
    ph = ((x * ys) % (1 << n)).astype(np.float64) / float(1 << n)
    want = np.exp(2j * np.pi * ph) / math.sqrt(1 << n)
    # relative error of each sampled amplitude, held to the state bound (480
    # gates, depth <= 500); with the error spread evenly over the amplitudes
    # this is the relative 2-norm error
    tol = 1e-12 if dtype == "c128" else 1e-5
    assert np.max(np.abs(got - want)) * math.sqrt(1 << n) < tol, np.max(np.abs(got - want))
    assert abs(s.norm() - 1) < (1e-12 if dtype == "c128" else 1e-5)


def test_alu_peak_probe():
    f32, f64 = qs.alu_peak("f32"), qs.alu_peak("f64")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # lane FMAs per second: at most 128 (single) per SM per clock at 2.1 GHz,
    # and at least half of that at a 1 GHz clock (the probe warms the clock up)
    assert sms * 64 * 1e9 < f32 < sms * 128 * 2.2e9
    assert 1e10 < f64 < f32


def test_edge_cases():
    s = qs.State(4, "c128").init_basis(3)
    with pytest.raises(qs.QsimError):
        s.init_basis(16)
    with pytest.raises(qs.QsimError):
        s.apply_gate(W.Gate("H", 4))
    with pytest.raises(qs.QsimError):
        s.apply_ctrl(1, 1, np.eye(2))
    with pytest.raises(qs.QsimError):
        s.expect("XX")
    s.apply_circuit([])                      # empty circuit: no-op
    v = s.to_numpy()
    assert v[3] == 1 and np.count_nonzero(v) == 1
    # the torch tensor is the state
    assert torch.equal(s.tensor.cpu(), torch.from_numpy(v))
    # a gate with every other qubit as control touches one pair
    n = 16
    psi = random_state(W.rng(3), n)
    g = W.phase_flip(n, 12345)
    want = oracle.run(n, [g], psi=psi)
    t = qs.State(n, "c128").from_numpy(psi).apply_gate(g)
    assert err(t.to_numpy(), want) < 1e-14
    assert err(gpu_run(n, [g], "c128", psi=psi), want) < 1e-14


def test_wrapped_state_follows_torch_stream():
    n = 12
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = qs.State(n, "c64")
        s.init_basis(0).apply_circuit(W.hadamard_layer(n))
        p = s.prob(5)
    assert abs(p - 2.0 ** -n) < 1e-9
