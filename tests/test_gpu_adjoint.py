"""Adjoint gradients (qs_adjoint_grad) against the oracle's parameter-shift
rule (FP64) at n = 10, and at the full 26-qubit size against central finite
differences of the complex128 GPU forward pass at sampled angles."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_quant_ph_0201042_gb300 as qs  # noqa: E402
from paper_quant_ph_0201042_gb300 import build as qbuild  # noqa: E402

qbuild.build()

GTOL = {"c128": 1e-9, "c64": 2e-4}


def perturbed(params, sigma, seed):
    return params + sigma * W.rng(seed).standard_normal(params.size)


@pytest.mark.parametrize("fuse", [True, False])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ansatz_n10_pauli_against_parameter_shift(dtype, fuse):
    # the gradient workload at the oracle's size: 25 layers of RY, RZ and a
    # C-NOT ladder on 10 qubits (500 angles), observable <Z_0>
    n = 10
    gates, params = W.ansatz_circuit(n, 25, seed=4)
    pauli = "Z" + "I" * (n - 1)
    work = qs.State(n, dtype)
    val, grad = qs.adjoint_grad(work, gates, params, pauli=pauli, fuse=fuse)
    want_val = oracle.cost(n, gates, params, pauli=pauli)
    want = oracle.gradient(n, gates, params, pauli=pauli, method="shift")
    assert abs(val - want_val) < GTOL[dtype]
    assert np.max(np.abs(grad - want)) < GTOL[dtype], np.max(np.abs(grad - want))
    fd = oracle.gradient(n, gates, params, pauli=pauli, method="fd", h=1e-4)
    assert np.max(np.abs(grad - fd)) < GTOL[dtype] + 1e-7


@pytest.mark.parametrize("fuse", [True, False])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ansatz_n10_fidelity_to_noiseless_output(dtype, fuse):
    # the fidelity to the noiseless output, differentiated with respect to
    # every (deviated) angle: d/dx F(theta + x) = dF/dtheta at theta + x
    n = 10
    gates, params = W.ansatz_circuit(n, 25, seed=5)
    ideal = oracle.run(n, gates)
    x = perturbed(params, 0.05, 6)
    ref = qs.State(n, dtype).from_numpy(ideal)
    work = qs.State(n, dtype)
    val, grad = qs.adjoint_grad(work, gates, x, ref=ref, fuse=fuse)
    want_val = oracle.cost(n, gates, x, ref=ideal)
    want = oracle.gradient(n, gates, x, ref=ideal, method="shift")
    assert abs(val - want_val) < GTOL[dtype]
    assert np.max(np.abs(grad - want)) < GTOL[dtype], np.max(np.abs(grad - want))


def test_urp1_and_controlled_parameters():
    # the paper's synthesis U_R(theta) U_P1(phi) (two angles per gate),
    # controlled phase shifts, and a parameter shared by two gates of the same
    # shift class (a U_R gate reusing the first U_R angle)
    n = 6
    r = W.rng(8)
    gates = []
    k = 0
    for layer in range(3):
        for q in range(n):
            gates.append(W.Gate("URP1", q, angles=(0.0, 0.0), param=k))
            k += 2
        for q in range(n - 1):
            gates.append(W.Gate("UP1", q + 1, controls={q: 1}, angles=(0.0,), param=k))
            k += 1
    gates.append(W.Gate("UR", 3, angles=(0.0,), param=0))
    params = r.uniform(-math.pi, math.pi, size=k)
    pauli = "XZYIZX"
    want = oracle.gradient(n, gates, params, pauli=pauli, method="shift")
    assert np.max(np.abs(want)) > 1e-2
    for dtype in ("c128", "c64"):
        for fuse in (True, False):
            work = qs.State(n, dtype)
            val, grad = qs.adjoint_grad(work, gates, params, pauli=pauli, fuse=fuse)
            assert np.max(np.abs(grad - want)) < GTOL[dtype], (dtype, fuse)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [13, 14])
def test_fused_sweep_every_gate_kind(dtype, n):
    # several tiles: parameterised gates of every differentiable kind with
    # controls inside and outside the tile, diagonal gates on outer bits,
    # SWAPs and C-NOTs, two gates sharing a parameter; fused and per-step
    # sweeps against the oracle's parameter-shift rule
    r = W.rng(300 + n)
    kinds = ["RY", "RZ", "UR", "UP1", "UP2", "URP1"]
    gates, k = W.hadamard_layer(n), 0
    for layer in range(4):
        for q in range(n):
            kind = kinds[int(r.integers(len(kinds)))]
            ctr = {}
            if r.random() < 0.3:
                c = int(r.choice([x for x in range(n) if x != q]))
                ctr[c] = int(r.integers(2))
            na = 2 if kind == "URP1" else 1
            gates.append(W.Gate(kind, q, controls=ctr, angles=(0.0,) * na, param=k))
            k += na
        for q in range(0, n - 1, 2):
            gates.append(W.Gate("X", q + 1, controls={q: 1}))
        a, b = (int(v) for v in r.choice(n, size=2, replace=False))
        gates.append(W.Gate("SWAP", a, target2=b))
    g0 = gates[n]                                               # a second gate on the first gate's parameter(s)
    gates.append(W.Gate(g0.kind, (g0.target + 3) % n, angles=g0.angles, param=g0.param))
    params = r.uniform(-math.pi, math.pi, size=k)
    pauli = "".join(r.choice(list("IXYZ"), size=n))
    want = oracle.gradient(n, gates, params, pauli=pauli, method="shift")
    want_val = oracle.cost(n, gates, params, pauli=pauli)
    assert np.max(np.abs(want)) > 1e-3
    for fuse in (True, False):
        work = qs.State(n, dtype)
        val, grad = qs.adjoint_grad(work, gates, params, pauli=pauli, fuse=fuse)
        assert abs(val - want_val) < GTOL[dtype], fuse
        assert np.max(np.abs(grad - want)) < GTOL[dtype] * 4, (fuse, np.max(np.abs(grad - want)))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fused_sweep_runs_of_one_target(dtype):
    # steps grouped on one target bit: several C-NOTs in a row on it with
    # controls on lane, warp and outer bits (they fold into the run's load),
    # diagonals controlled by the run's own bit, diagonals on outer bits and
    # on other tile bits, real and complex rotations, all against the
    # oracle's parameter-shift rule
    n = 15
    r = W.rng(1515)
    gates, k = W.hadamard_layer(n), 0
    for t in (0, 4, 6, 9, 13):
        others = [x for x in range(n) if x != t]
        block = []
        for _ in range(3):
            c = int(r.choice(others))
            block.append(W.Gate("X", t, controls={c: int(r.integers(2))}))
        for kind in ("RZ", "UP1", "RY", "UR", "URP1"):
            na = 2 if kind == "URP1" else 1
            ctr = {int(r.choice(others)): int(r.integers(2))} if r.random() < 0.5 else {}
            block.append(W.Gate(kind, t, controls=ctr, angles=(0.0,) * na, param=k))
            k += na
        d = int(r.choice(others))
        block.append(W.Gate("RZ", d, controls={t: 1}, angles=(0.0,), param=k))      # controlled by the run's bit
        k += 1
        block.append(W.Gate("UP1", int(r.choice(others)), angles=(0.0,), param=k))  # another bit, uncontrolled
        k += 1
        gates += block
        gates.append(W.Gate("X", (t + 1) % n, controls={t: 1}))
    params = r.uniform(-math.pi, math.pi, size=k)
    # <Z_t> for each block's target: together they reach most parameters
    seen = np.zeros(k)
    for t in (0, 4, 6, 9, 13):
        pauli = "".join("Z" if q == t else "I" for q in range(n))
        want = oracle.gradient(n, gates, params, pauli=pauli, method="shift")
        want_val = oracle.cost(n, gates, params, pauli=pauli)
        seen = np.maximum(seen, np.abs(want))
        for fuse in (True, False):
            val, grad = qs.adjoint_grad(qs.State(n, dtype), gates, params, pauli=pauli, fuse=fuse)
            assert abs(val - want_val) < GTOL[dtype], (t, fuse)
            assert np.max(np.abs(grad - want)) < GTOL[dtype] * 4, (t, fuse, np.max(np.abs(grad - want)))
    assert np.sum(seen > 1e-3) > 25


def test_autograd_function_matches():
    n = 8
    gates, params = W.ansatz_circuit(n, 4, seed=12)
    work = qs.State(n, "c128")
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    E = qs.AdjointExpectation.apply(p, work, gates, "Z" + "I" * (n - 1), None)
    (2.0 * E).backward()
    want = oracle.gradient(n, gates, params, pauli="Z" + "I" * (n - 1), method="shift")
    assert np.max(np.abs(p.grad.numpy() - 2.0 * want)) < 1e-9


def test_adjoint_n26_full_size():
    # the gradient workload at full size: n = 26, 25 layers (1300 angles),
    # complex64 state; observables <Z_0> and the fidelity to the noiseless
    # output at deviated angles.  Sampled components are checked against the
    # parameter-shift rule and central finite differences (h = 1e-4) of the
    # complex128 GPU forward pass.
    n = 26
    gates, params = W.ansatz_circuit(n, 25, seed=2026)
    x = perturbed(params, 0.02, 7)
    pauli = "Z" + "I" * (n - 1)
    work = qs.State(n, "c64")
    ref64 = qs.State(n, "c64").init_basis(0).apply_circuit(gates)      # noiseless output
    zval, zgrad = qs.adjoint_grad(work, gates, x, pauli=pauli)
    fval, fgrad = qs.adjoint_grad(work, gates, x, ref=ref64)
    assert zgrad.size == 1300 and fgrad.size == 1300
    ref_np = ref64.to_numpy()
    del work, ref64
    torch.cuda.empty_cache()
    s128 = qs.State(n, "c128")
    r128 = qs.State(n, "c128").from_numpy(ref_np.astype(np.complex128))

    def run(pv):
        g2 = [W.Gate(g.kind, g.target, angles=(float(pv[g.param]),), param=g.param) if g.param >= 0 else g
              for g in gates]
        s128.init_basis(0).apply_circuit(g2)

    def Z(pv):
        run(pv)
        return s128.expect(pauli)

    def F(pv):
        run(pv)
        return abs(r128.inner(s128)) ** 2

    assert abs(zval - Z(x)) < 1e-5
    assert abs(fval - F(x)) < 1e-5
    assert 0.5 < fval < 0.999
    rs = W.rng(99)
    for k in sorted(set([0, 1299, 650] + [int(v) for v in rs.integers(0, 1300, size=2)])):
        for fn, grad, tol in ((F, fgrad, 2e-4), (Z, zgrad, 2e-5)):
            pp, pm = x.copy(), x.copy()
            pp[k] += 1e-4
            pm[k] -= 1e-4
            fd = (fn(pp) - fn(pm)) / 2e-4
            pp[k] = x[k] + math.pi / 2
            pm[k] = x[k] - math.pi / 2
            shift = (fn(pp) - fn(pm)) / 2
            assert abs(fd - shift) < 1e-6, (k, fd, shift)
            assert abs(grad[k] - shift) < tol, (k, grad[k], shift)


def test_no_parameters_and_unused_parameters():
    # a circuit without parameters: the value only; parameters no gate uses
    # get a zero derivative
    n = 12
    gates = W.random_circuit(n, 2, seed=3)
    work = qs.State(n, "c64")
    val, grad = qs.adjoint_grad(work, gates, np.zeros(0), pauli="Z" * n)
    assert grad.size == 0
    assert abs(val - oracle.cost(n, gates, np.zeros(0), pauli="Z" * n)) < 1e-5
    g2, p2 = W.ansatz_circuit(n, 2, seed=4)
    params = np.concatenate([p2, [0.3, -0.7]])            # two trailing unused parameters
    for fuse in (True, False):
        val, grad = qs.adjoint_grad(qs.State(n, "c128"), g2, params, pauli="Z" + "I" * (n - 1), fuse=fuse)
        assert grad.size == params.size and grad[-1] == 0.0 and grad[-2] == 0.0
        want = oracle.gradient(n, g2, params, pauli="Z" + "I" * (n - 1), method="shift")
        assert np.max(np.abs(grad - want)) < 1e-9
