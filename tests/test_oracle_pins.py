"""Pins of the CPU oracle against things other than itself (no GPU needed).

Every check here takes its expected value from an independent route: dense
Kronecker-product matrices built with numpy/scipy, matrix exponentials of the
gate generators, numpy's FFT, scipy's Hadamard matrix, Grover's closed form,
curand's host Philox generator, the one-qubit density-matrix recursions of the
paper (Sec. 4.3.1), and finite differences.
"""
import ctypes
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as sst

import oracle
import workloads as W
from _util import random_gate, random_state

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def test_pauli_algebra_of_test_matrices():
    # the test's own Pauli matrices satisfy XY = iZ, YZ = iX, ZX = iY
    assert np.allclose(PX @ PY, 1j * PZ)
    assert np.allclose(PY @ PZ, 1j * PX)
    assert np.allclose(PZ @ PX, 1j * PY)


def expected_2x2(g):
    """2x2 matrix of a gate by an independent route (matrix exponentials)."""
    a = g.angles
    if g.kind == "MATRIX":
        return np.asarray(g.matrix)
    if g.kind == "H":
        return sla.hadamard(2).astype(complex) / math.sqrt(2)
    if g.kind == "X":
        return PX
    if g.kind == "Y":
        return PY
    if g.kind == "Z":
        return PZ
    if g.kind == "UP1":
        return sla.expm(1j * a[0] * P1)
    if g.kind == "UP2":
        return sla.expm(1j * a[0] * P0)
    if g.kind == "UR":
        return sla.expm(-1j * a[0] * PY)       # [[cos, -sin], [sin, cos]]
    if g.kind == "URP1":
        return sla.expm(-1j * a[0] * PY) @ sla.expm(1j * a[1] * P1)
    if g.kind == "RY":
        return sla.expm(-0.5j * a[0] * PY)
    if g.kind == "RZ":
        return sla.expm(-0.5j * a[0] * PZ)
    raise KeyError(g.kind)


def kron_list(ops):
    out = np.array([[1.0 + 0j]])
    for o in ops:
        out = np.kron(out, o)
    return out


def dense_operator(n, g):
    """2^n x 2^n matrix of a gate: Kronecker products with qubit 0 as the
    leftmost (most significant) factor; controls as projectors."""
    if g.kind == "SWAP":
        def pair(P):
            ops = [I2] * n
            ops[g.target] = P
            ops[g.target2] = P
            return kron_list(ops)
        S = 0.5 * (np.eye(1 << n) + pair(PX) + pair(PY) + pair(PZ))
        U_big, id_big = S, np.eye(1 << n)
    else:
        U = expected_2x2(g)
        ops = [I2] * n
        ops[g.target] = U
        U_big = kron_list(ops)
        id_big = np.eye(1 << n)
    if not g.controls:
        return U_big
    proj = [I2] * n
    for q, v in g.controls.items():
        proj[q] = P1 if v else P0
    Pm = kron_list(proj)
    return Pm @ U_big + (id_big - Pm)


@pytest.mark.parametrize("kind", ["H", "X", "Y", "Z", "UP1", "UP2", "UR", "URP1", "RY", "RZ", "MATRIX"])
def test_gate_matrices_match_generators(kind):
    r = W.rng(11)
    for _ in range(5):
        angles = tuple(r.uniform(-math.pi, math.pi, size=W.KINDS[kind]))
        m = W.haar_su2(r) if kind == "MATRIX" else None
        g = W.Gate(kind, 0, angles=angles, matrix=m)
        assert np.allclose(oracle.gate_matrix(g), expected_2x2(g), atol=1e-14, rtol=0)


def test_paper_synthesis_of_h_and_not():
    # Sec. 3.2: H = U_R(pi/4) U_P1(pi), NOT = U_R(pi/2) U_P1(pi)
    h = oracle.gate_matrix(W.Gate("URP1", 0, angles=(math.pi / 4, math.pi)))
    x = oracle.gate_matrix(W.Gate("URP1", 0, angles=(math.pi / 2, math.pi)))
    assert np.allclose(h, sla.hadamard(2) / math.sqrt(2), atol=1e-15)
    assert np.allclose(x, PX, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_gates_equal_dense_kronecker_products(n):
    r = W.rng(100 + n)
    for _ in range(25):
        g = random_gate(r, n)
        psi = random_state(r, n)
        got = oracle.run(n, [g], psi=psi)
        want = dense_operator(n, g) @ psi
        assert np.max(np.abs(got - want)) < 1e-13, g


def test_circuit_equals_product_of_dense_operators():
    n = 6
    r = W.rng(7)
    gates = [random_gate(r, n) for _ in range(40)]
    psi = random_state(r, n)
    want = psi.copy()
    for g in gates:
        want = dense_operator(n, g) @ want
    got = oracle.run(n, gates, psi=psi)
    assert np.max(np.abs(got - want)) < 1e-12


def test_invalid_gates_rejected():
    with pytest.raises(ValueError):
        oracle.run(3, [W.Gate("H", 3)])
    with pytest.raises(ValueError):
        oracle.run(3, [W.Gate("X", 1, controls={1: 1})])
    with pytest.raises(ValueError):
        oracle.run(3, [W.Gate("SWAP", 1, target2=1)])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_qft_closed_form(n):
    # Sec. 2.3.2: QFT|x> = 2^{-n/2} sum_y e^{2 pi i x y / 2^n} |y>, which is
    # numpy's inverse DFT of the basis vector times sqrt(2^n)
    N = 1 << n
    for x in sorted({0, 1, N - 1, W.basis_index(1234 + n, n)}):
        got = oracle.run(n, W.qft_circuit(n), x0=x)
        e = np.zeros(N, dtype=complex)
        e[x] = 1
        want = np.fft.ifft(e) * math.sqrt(N)
        assert np.linalg.norm(got - want) < 1e-12


def test_qft_gate_count_n10():
    g = W.qft_circuit(10)
    assert sum(1 for x in g if x.kind == "H") == 10
    assert sum(1 for x in g if x.kind == "UP1") == 45
    assert sum(1 for x in g if x.kind == "SWAP") == 5


def dft_matrix(L, inverse=False):
    """2^{-L/2} w^{xy} built from numpy's FFT of the identity columns."""
    M = 1 << L
    eye = np.eye(M, dtype=complex)
    return (np.fft.fft(eye, axis=0) if inverse else np.fft.ifft(eye, axis=0) * M) / math.sqrt(M)


@pytest.mark.parametrize("n", [1, 2, 4, 7, 10])
def test_qft_black_box_whole_register(n):
    # the QFT as a black box (Sec. 2.3.2) on random vectors against numpy's
    # inverse FFT times 2^{n/2}, and against the oracle's own gate-by-gate
    # QFT circuit; the inverse undoes it
    r = W.rng(600 + n)
    psi = random_state(r, n)
    got = oracle.qft(psi)
    assert np.linalg.norm(got - np.fft.ifft(psi) * math.sqrt(1 << n)) < 1e-12
    assert np.linalg.norm(got - oracle.run(n, W.qft_circuit(n), psi=psi)) < 1e-12
    back = oracle.qft(got, inverse=True)
    assert np.linalg.norm(back - psi) < 1e-12
    assert np.linalg.norm(oracle.qft(psi, inverse=True) - np.fft.fft(psi) / math.sqrt(1 << n)) < 1e-12


@pytest.mark.parametrize("n,q0,L", [(3, 0, 1), (4, 1, 2), (6, 2, 3), (7, 0, 4), (7, 3, 4), (8, 5, 3)])
def test_qft_black_box_sub_register(n, q0, L):
    # QFT of qubits q0..q0+L-1 = I_{2^q0} (x) F_{2^L} (x) I_{2^{n-q0-L}} with
    # qubit 0 the most significant (Kronecker order = qubit order), and the
    # same sub-register circuit applied gate by gate
    r = W.rng(700 + 16 * n + q0)
    psi = random_state(r, n)
    for inv in (False, True):
        Umat = np.kron(np.kron(np.eye(1 << q0), dft_matrix(L, inv)), np.eye(1 << (n - q0 - L)))
        assert np.linalg.norm(oracle.qft(psi, q0, L, inverse=inv) - Umat @ psi) < 1e-12
    assert np.linalg.norm(oracle.qft(psi, q0, L) - oracle.run(n, W.qft_circuit(n, q0, L), psi=psi)) < 1e-12


def test_qft_black_box_rejects_bad_ranges():
    psi = random_state(W.rng(1), 4)
    for q0, L in ((0, 0), (3, 2), (-1, 2)):
        with pytest.raises(ValueError):
            oracle.qft(psi, q0, L)


@pytest.mark.parametrize("L,eps", [(8, 1e-2), (12, 1e-3)])
def test_approximate_qft_error_bound(L, eps):
    # the approximate QFT (Sec. 2.3.2) drops the phase shifts of index
    # k > max_k; every dropped gate differs from the identity by
    # |e^{i 2 pi / 2^k} - 1| <= 2 pi / 2^k, so the operator-norm error is at
    # most the sum of those; checked against the exact transform on random
    # states, and the gate count is O(L log(L / eps))
    mk = W.approx_qft_max_k(L, eps)
    full, approx = W.qft_circuit(L), W.qft_circuit(L, max_k=mk)
    dropped = [g for g in full if g.kind == "UP1" and g.angles[0] < 2 * math.pi / (1 << mk) - 1e-15]
    assert len(full) - len(approx) == len(dropped)
    bound = sum(2 * math.pi / (1 << round(math.log2(2 * math.pi / g.angles[0]))) for g in dropped)
    assert sum(1 for g in approx if g.kind == "UP1") <= L * mk
    r = W.rng(800 + L)
    for _ in range(3):
        psi = random_state(r, L)
        e = np.linalg.norm(oracle.run(L, approx, psi=psi) - oracle.qft(psi))
        assert 0 < e <= bound + 1e-12


@pytest.mark.parametrize("n", [1, 3, 6, 8])
def test_hadamard_transform(n):
    # Sec. 2.3.1: H_n|x> = 2^{-n/2} sum_y (-1)^{x.y}|y>; scipy's Sylvester
    # Hadamard matrix has entries (-1)^{popcount(x & y)}
    N = 1 << n
    Hm = sla.hadamard(N) / math.sqrt(N)
    r = W.rng(n)
    for x in [0, N - 1, int(r.integers(N))]:
        got = oracle.run(n, W.hadamard_layer(n), x0=x)
        assert np.max(np.abs(got - Hm[:, x])) < 1e-13


def test_hadamard_uniform_magnitudes_n14():
    n = 14
    got = oracle.run(n, W.hadamard_layer(n), x0=12345)
    assert np.max(np.abs(np.abs(got) ** 2 - 2.0 ** -n)) < 1e-16


def grover_closed_form(n, k, j):
    N = 1 << n
    th = math.asin(1 / math.sqrt(N))
    v = np.full(N, math.cos((2 * j + 1) * th) / math.sqrt(N - 1), dtype=complex)
    v[k] = math.sin((2 * j + 1) * th)
    return v * (-1) ** j


@pytest.mark.parametrize("n", [2, 4, 7])
def test_grover_closed_form_state(n):
    k = W.basis_index(55 + n, n)
    for j in range(0, W.grover_iterations(n) + 2):
        got = oracle.run(n, W.grover_circuit(n, k, j))
        assert np.linalg.norm(got - grover_closed_form(n, k, j)) < 1e-12


def test_grover_success_probability_n10():
    n, k = 10, 777
    it = W.grover_iterations(n)
    got = oracle.run(n, W.grover_circuit(n, k, it))
    th = math.asin(2 ** (-n / 2))
    assert abs(oracle.prob(got, k) - math.sin((2 * it + 1) * th) ** 2) < 1e-12


def test_norm_preserved_random_circuit():
    n = 10
    psi = oracle.run(n, W.random_circuit(n, 6, seed=3))
    assert abs(oracle.norm2(psi) - 1) < 1e-13


def test_reductions_against_numpy():
    n = 7
    r = W.rng(5)
    psi = random_state(r, n)
    phi = random_state(r, n)
    assert abs(oracle.norm2(psi) - np.vdot(psi, psi).real) < 1e-14
    assert abs(oracle.inner(psi, phi) - np.vdot(psi, phi)) < 1e-14
    for q in range(n):
        p1 = np.sum(np.abs(psi.reshape([2] * n)) ** 2, axis=tuple(a for a in range(n) if a != q))[1]
        assert abs(oracle.prob_qubit(psi, q) - p1) < 1e-14
    for _ in range(10):
        s = "".join(r.choice(list("IXYZ"), size=n))
        P = kron_list([{"I": I2, "X": PX, "Y": PY, "Z": PZ}[c] for c in s])
        assert abs(oracle.expect_pauli(psi, s) - np.vdot(psi, P @ psi).real) < 1e-13
    for idx in [0, 5, 127]:
        assert abs(oracle.prob(psi, idx) - abs(psi[idx]) ** 2) < 1e-16


def test_measurement_rule():
    # Sec. 2.2.3: smallest i with r < sum_{j<=i} |alpha_j|^2
    n = 6
    r = W.rng(8)
    psi = random_state(r, n)
    cdf = np.cumsum(np.abs(psi) ** 2)
    for u in r.uniform(0, 0.999, size=200):
        assert oracle.measure(psi, u) == int(np.searchsorted(cdf, u, side="right"))
    # zero-probability amplitudes are never an outcome; r at or beyond the
    # rounded total gives the last index with non-zero probability
    phi = psi.copy()
    phi[5] = 0
    phi[-3:] = 0
    phi /= np.linalg.norm(phi)
    cdf = np.cumsum(np.abs(phi) ** 2)
    for u in np.concatenate([r.uniform(0, 0.999, size=200), [cdf[4], cdf[-1], 0.9999999999999999]]):
        got = oracle.measure(phi, u)
        if u < cdf[-1]:
            assert got == int(np.searchsorted(cdf, u, side="right"))
        else:
            assert got == (1 << n) - 4
        assert abs(phi[got]) > 0


# ---------------------------------------------------------------------------
# Philox4x32-10 against curand's host generator (an independent implementation)
# ---------------------------------------------------------------------------

def _curand_host_words(seed, count):
    try:
        cr = ctypes.CDLL("libcurand.so")
    except OSError:
        try:
            cr = ctypes.CDLL("/usr/local/cuda/lib64/libcurand.so")
        except OSError:
            pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("curand host generator unavailable")
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2 ** 64 - 1])
def test_philox_matches_curand_host_generator(seed):
    # curand's host Philox4_32_10 emits block k = Philox(counter (0, 0, k, 0),
    # key (seed low word, seed high word))
    words = _curand_host_words(seed, 4 * 512)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in list(range(0, 512, 7)) + [511]:
        assert list(oracle.philox((0, 0, k, 0), key)) == list(words[4 * k:4 * k + 4])


def test_gaussian_draws_are_standard_normal():
    g = np.array([oracle.gauss(99, t, s, a) for t in range(40) for s in range(50) for a in range(2)])
    assert sst.kstest(g, "norm").pvalue > 1e-3
    assert abs(g.mean()) < 0.1 and abs(g.std() - 1) < 0.05


def test_flip_threshold():
    assert oracle.flip_threshold(0.0) == 0
    assert oracle.flip_threshold(1e-3) == 4294967
    assert oracle.flip_threshold(0.5) == 2 ** 31


# ---------------------------------------------------------------------------
# Noisy trajectories against the paper's error-model closed forms (Sec. 4.3.1)
# ---------------------------------------------------------------------------

def test_noiseless_trajectory_equals_circuit():
    n = 5
    gates = W.noisy_synthesis(W.qft_circuit(n))
    psi, st = oracle.run_trajectory(n, gates, 0.0, 0.0, seed=1, traj=3, x0=9)
    assert np.linalg.norm(psi - oracle.run(n, W.qft_circuit(n), x0=9)) < 1e-13
    assert list(st) == [0, 0, 0, 0]


def _ht_zero_term(n, k, p, sigma, mode, every, n_traj, seed):
    gates = W.noisy_synthesis(W.hadamard_layer(n) * k)
    vals = []
    nflips = 0
    for t in range(n_traj):
        psi, st = oracle.run_trajectory(n, gates, p, sigma, seed, t, 0, mode=mode, every=every)
        vals.append(abs(psi[0]) ** 2)
        nflips += int(st[0] + st[1] + st[2])
    v = np.array(vals)
    return v.mean(), v.std() / math.sqrt(n_traj), nflips


def test_trajectories_flip_noise_closed_form():
    # X or Z flip with probability p/2 each after every gate step, on every
    # qubit: Bloch x and z components shrink by (1 - p) per step and H swaps
    # them, so the |0><0| term after k (even) Hadamard transforms of n qubits
    # is ((1 + (1 - p)^{n k}) / 2)^n
    n, k, p = 3, 4, 0.02
    mean, se, nflips = _ht_zero_term(n, k, p, 0.0, oracle.NOISE_FLIPS, 1, 4000, 21)
    want = ((1 + (1 - p) ** (n * k)) / 2) ** n
    assert abs(mean - want) < 4 * se + 1e-3
    expect_flips = 4000 * n * k * n * p
    assert abs(nflips - expect_flips) < 5 * math.sqrt(expect_flips)


def test_trajectories_depolarizing_closed_form_paper():
    # Sec. 4.3.1: depolarizing channel once per Hadamard transform gives
    # ((1 + (1 - 4p/3)^k) / 2)^n for even k
    n, k, p = 3, 6, 0.05
    mean, se, _ = _ht_zero_term(n, k, p, 0.0, oracle.NOISE_DEPOLARIZING, n, 4000, 22)
    want = ((1 + (1 - 4 * p / 3) ** k) / 2) ** n
    assert abs(mean - want) < 4 * se + 1e-3


def test_trajectories_operational_error_closed_form_paper():
    # Sec. 4.3.1: H(x, y) = U_R(pi/4 + x) U_P1(pi + y) with x, y ~ N(0, sigma^2)
    # gives ((1 + exp(-9 sigma^2 k / 4)) / 2)^n for even k
    n, k, sigma = 3, 10, 0.1
    mean, se, _ = _ht_zero_term(n, k, 0.0, sigma, oracle.NOISE_FLIPS, 1, 3000, 23)
    want = ((1 + math.exp(-9 * sigma ** 2 * k / 4)) / 2) ** n
    assert abs(mean - want) < 4 * se + 1e-3


def test_operational_closed_form_matches_quadrature():
    # the paper's one-qubit formula against a Gauss-Hermite quadrature of the
    # density-matrix recursion rho_{k+1} = E[H(x,y) rho_k H(x,y)^*]
    from numpy.polynomial.hermite_e import hermegauss
    sigma = 0.05
    xs, ws = hermegauss(30)
    ws = ws / ws.sum()
    rho = P0.copy()
    for k in range(1, 21):
        new = np.zeros((2, 2), complex)
        for x, wx in zip(xs, ws):
            Rx = sla.expm(-1j * (math.pi / 4 + sigma * x) * PY)
            for y, wy in zip(xs, ws):
                Hxy = Rx @ sla.expm(1j * (math.pi + sigma * y) * P1)
                new += wx * wy * Hxy @ rho @ Hxy.conj().T
        rho = new
        if k % 2 == 0:
            assert abs(rho[0, 0].real - (1 + math.exp(-9 * sigma ** 2 * k / 4)) / 2) < 1e-12


def test_trajectory_gate_flags():
    # per-gate flags: flips only after the last gate of each Hadamard layer is
    # the same draw sequence as every = n (bit for bit); no deviation on any
    # gate is the sigma = 0 trajectory; a noiseless preparation leaves the
    # prepared state exact
    n, k = 4, 6
    gates = W.noisy_synthesis(W.hadamard_layer(n) * k)
    fl = [0 if (s + 1) % n == 0 else oracle.NO_FLIPS for s in range(len(gates))]
    for t in range(20):
        a = oracle.run_trajectory(n, gates, 0.05, 0.02, 7, t, 0, mode=oracle.NOISE_DEPOLARIZING, every=n)
        b = oracle.run_trajectory(n, gates, 0.05, 0.02, 7, t, 0, mode=oracle.NOISE_DEPOLARIZING, flags=fl)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        c = oracle.run_trajectory(n, gates, 0.0, 0.3, 7, t, 0, flags=[oracle.NO_DEVIATION] * len(gates))
        assert np.linalg.norm(c[0] - oracle.run(n, gates)) < 1e-13
    prep = W.noisy_synthesis(W.hadamard_layer(n))
    d = oracle.run_trajectory(n, prep, 0.5, 0.3, 7, 0, 0, flags=[3] * n)
    assert np.allclose(d[0], np.full(1 << n, 2 ** (-n / 2))) and list(d[1]) == [0, 0, 0, 0]


def test_trajectory_draws_are_deterministic():
    n = 4
    gates = W.noisy_synthesis(W.qft_circuit(n))
    a = oracle.run_trajectory(n, gates, 0.05, 0.01, seed=5, traj=17, x0=3)
    b = oracle.run_trajectory(n, gates, 0.05, 0.01, seed=5, traj=17, x0=3)
    c = oracle.run_trajectory(n, gates, 0.05, 0.01, seed=5, traj=18, x0=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[1], c[1]) or not np.array_equal(a[0], c[0])


# ---------------------------------------------------------------------------
# Gradients
# ---------------------------------------------------------------------------

def test_gradient_controlled_rotation_and_shared_parameter_closed_forms():
    # controlled RY(t) with the control in |+>: <Z_target> = (1 + cos t) / 2,
    # derivative -sin(t) / 2 (generator eigenvalues {-1/2, 0, 1/2}: the
    # four-term rule); RY(t) twice on one qubit is RY(2t): <Z> = cos 2t,
    # derivative -2 sin 2t (the occurrences' derivatives add)
    for t in [-2.5, -0.4, 0.9, 2.2]:
        gates = [W.Gate("H", 0), W.Gate("RY", 1, controls={0: 1}, angles=(t,), param=0)]
        for method in ("shift", "fd"):
            g = oracle.gradient(2, gates, np.array([t]), pauli="IZ", method=method, h=1e-5)
            assert abs(g[0] + math.sin(t) / 2) < (1e-13 if method == "shift" else 1e-9)
        gates = [W.Gate("RY", 0, angles=(t,), param=0), W.Gate("RY", 0, angles=(t,), param=0)]
        g = oracle.gradient(1, gates, np.array([t]), pauli="Z", method="shift")
        assert abs(g[0] + 2 * math.sin(2 * t)) < 1e-13
        # controlled U_R(t) with control |+>: <Z> = (1 + cos 2t) / 2
        gates = [W.Gate("H", 0), W.Gate("UR", 1, controls={0: 1}, angles=(t,), param=0)]
        g = oracle.gradient(2, gates, np.array([t]), pauli="IZ", method="shift")
        assert abs(g[0] + math.sin(2 * t)) < 1e-13


def test_gradient_closed_forms_one_qubit():
    # RY(t)|0>: <Z> = cos t;  U_R(t)|0>: <Z> = cos 2t
    for t in [-2.0, -0.3, 0.7, 2.9]:
        g = oracle.gradient(1, [W.Gate("RY", 0, angles=(t,), param=0)], np.array([t]), pauli="Z")
        assert abs(g[0] + math.sin(t)) < 1e-13
        g = oracle.gradient(1, [W.Gate("UR", 0, angles=(t,), param=0)], np.array([t]), pauli="Z")
        assert abs(g[0] + 2 * math.sin(2 * t)) < 1e-13


@pytest.mark.parametrize("obs", ["pauli", "fidelity"])
def test_parameter_shift_matches_finite_differences(obs):
    n = 5
    gates, params = W.ansatz_circuit(n, 2, seed=9)
    ref = None
    pauli = None
    if obs == "pauli":
        pauli = "Z" + "I" * (n - 1)
    else:
        ref = oracle.run(n, W.random_circuit(n, 2, seed=10))
    gs = oracle.gradient(n, gates, params, pauli=pauli, ref=ref, method="shift")
    gf = oracle.gradient(n, gates, params, pauli=pauli, ref=ref, method="fd", h=1e-4)
    assert np.max(np.abs(gs - gf)) < 1e-7
    assert np.max(np.abs(gs)) > 1e-3
