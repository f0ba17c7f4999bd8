"""GPU parity of the batched noisy trajectories (qs_run_trajectories) against
the oracle's one-at-a-time replay, plus the paper's error-model closed forms.

Flip decisions are integer (Philox word < floor(p 2^32)), so the flip counts
and the event fingerprint must match the oracle bit for bit; metrics agree to
the state precision (the Gaussian deviations use each side's libm).
"""
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

MTOL = {"c128": 1e-10, "c64": 2e-5}


def oracle_metric(n, gates, p, sigma, seed, traj, x0, metric, target, mode=0, every=1):
    psi, st = oracle.run_trajectory(n, gates, p, sigma, seed, traj, x0, mode=mode, every=every)
    if metric == "prob":
        return abs(psi[target]) ** 2, st
    ideal = oracle.run(n, gates, x0=x0)
    return abs(oracle.inner(ideal, psi)) ** 2, st


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noiseless_trajectories(dtype):
    n = 8
    r = W.rng(3)
    x0 = r.integers(0, 1 << n, size=16, dtype=np.uint64)
    g_qft = {"n": n, "gates": W.noisy_synthesis(W.qft_circuit(n)), "x0": x0, "first": 0}
    k = 77
    it = W.grover_iterations(n)
    g_gr = {"n": n, "gates": W.noisy_synthesis(W.grover_circuit(n, k, it)), "x0": np.zeros(8, np.uint64),
            "first": 16, "metric": "prob", "target": k}
    met, st = qs.run_trajectories([g_qft, g_gr], 0.0, 0.0, seed=1, dtype=dtype)
    assert np.all(st == 0)
    assert np.max(np.abs(met[:16] - 1.0)) < MTOL[dtype] * 10
    th = math.asin(2 ** (-n / 2))
    assert np.max(np.abs(met[16:] - math.sin((2 * it + 1) * th) ** 2)) < MTOL[dtype] * 10


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", [oracle.NOISE_FLIPS, oracle.NOISE_DEPOLARIZING])
def test_trajectories_match_oracle_replay(dtype, mode):
    n = 7
    seed = 0xC0FFEE1234
    gates = W.noisy_synthesis(W.qft_circuit(n))
    r = W.rng(11)
    x0 = r.integers(0, 1 << n, size=24, dtype=np.uint64)
    k = 5
    it = 4
    ggates = W.noisy_synthesis(W.grover_circuit(n, k, it))
    groups = [{"n": n, "gates": gates, "x0": x0, "first": 100},
              {"n": n, "gates": ggates, "x0": np.zeros(12, np.uint64), "first": 500, "metric": "prob", "target": k}]
    p, sigma = 0.02, 0.05
    met, st = qs.run_trajectories(groups, p, sigma, seed, dtype=dtype, mode=mode)
    flips = 0
    for i in range(24):
        m, s = oracle_metric(n, gates, p, sigma, seed, 100 + i, int(x0[i]), "fidelity", 0, mode=mode)
        assert list(s) == [int(v) for v in st[i]], i
        assert abs(m - met[i]) < MTOL[dtype], (i, m, met[i])
        flips += int(s[0] + s[1] + s[2])
    for i in range(12):
        m, s = oracle_metric(n, ggates, p, sigma, seed, 500 + i, 0, "prob", k, mode=mode)
        assert list(s) == [int(v) for v in st[24 + i]], i
        assert abs(m - met[24 + i]) < MTOL[dtype], (i, m, met[24 + i])
    assert flips > 10     # the noise is really exercised


def test_every_granularity_matches_oracle():
    n = 5
    gates = W.noisy_synthesis(W.hadamard_layer(n) * 6)
    x0 = np.zeros(16, np.uint64)
    met, st = qs.run_trajectories([{"n": n, "gates": gates, "x0": x0, "first": 0, "metric": "prob", "target": 0}],
                                  0.05, 0.02, seed=9, dtype="c128", mode=oracle.NOISE_DEPOLARIZING, every=n)
    for i in range(16):
        psi, s = oracle.run_trajectory(n, gates, 0.05, 0.02, 9, i, 0, mode=oracle.NOISE_DEPOLARIZING, every=n)
        assert list(s) == [int(v) for v in st[i]]
        assert abs(abs(psi[0]) ** 2 - met[i]) < 1e-10


def test_paper_depolarizing_closed_form():
    # Sec. 4.3.1: the |0><0| term after k (even) Hadamard transforms of n
    # qubits with the depolarizing channel once per transform is
    # ((1 + (1 - 4p/3)^k) / 2)^n
    n, k, p = 6, 20, 0.01
    T = 8192
    gates = W.noisy_synthesis(W.hadamard_layer(n) * k)
    met, _ = qs.run_trajectories([{"n": n, "gates": gates, "x0": np.zeros(T, np.uint64), "first": 0,
                                   "metric": "prob", "target": 0}], p, 0.0, seed=2024, dtype="c64",
                                 mode=qs.NOISE_DEPOLARIZING, every=n, with_stats=False)
    want = ((1 + (1 - 4 * p / 3) ** k) / 2) ** n
    se = met.std() / math.sqrt(T)
    assert abs(met.mean() - want) < 4 * se + 1e-3, (met.mean(), want)


def test_paper_operational_closed_form():
    # Sec. 4.3.1: H(x, y) = U_R(pi/4 + x) U_P1(pi + y), x, y ~ N(0, sigma^2):
    # ((1 + exp(-9 sigma^2 k / 4)) / 2)^n for even k
    n, k, sigma = 6, 20, 0.08
    T = 8192
    gates = W.noisy_synthesis(W.hadamard_layer(n) * k)
    met, _ = qs.run_trajectories([{"n": n, "gates": gates, "x0": np.zeros(T, np.uint64), "first": 0,
                                   "metric": "prob", "target": 0}], 0.0, sigma, seed=77, dtype="c64",
                                 with_stats=False)
    want = ((1 + math.exp(-9 * sigma ** 2 * k / 4)) / 2) ** n
    se = met.std() / math.sqrt(T)
    assert abs(met.mean() - want) < 4 * se + 1e-3, (met.mean(), want)


def test_batch_4096_mixed_widths():
    # the batched-trajectory workload: 4096 trajectories of 12, 16 and 20
    # qubits in ratio 2:1:1, QFT on seeded basis states at every width and
    # Grover at 12/16; sigma = 1e-2, p = 1e-3; complex64 state
    batch = W.trajectory_batch(4096, ((12, 2), (16, 1), (20, 1)), (12, 16), seed=31337)
    groups = qs.batch_groups(batch)
    seed = 0x5EED5EED
    met, st = qs.run_trajectories(groups, 1e-3, 1e-2, seed, dtype="c64")
    assert met.size == 4096
    assert np.all((met >= -1e-6) & (met <= 1 + 1e-5))
    # replay sampled trajectories of every group on the oracle
    for k, g in enumerate(groups):
        n = g["n"]
        picks = [0, len(g["x0"]) - 1] if n < 20 else [0]
        for i in picks:
            t = g["first"] + i
            m, s = oracle_metric(n, g["gates"], 1e-3, 1e-2, seed, t, int(g["x0"][i]),
                                 g.get("metric", "fidelity"), g.get("target", 0))
            assert list(s) == [int(v) for v in st[t]], (k, i)
            assert abs(m - met[t]) < 5e-4, (k, i, m, met[t])


@pytest.mark.parametrize("mode,p,sigma", [(qs.NOISE_DEPOLARIZING, 1e-3, 0.0), (qs.NOISE_FLIPS, 0.0, 0.03)])
def test_paper_ht_experiment_n20(mode, p, sigma):
    # the paper's experiment (Sec. 4.3.1) at its size: a 20-qubit register in
    # |0...0>, the Hadamard transform applied k times (even), decoherence once
    # per transform (depolarizing) or deviated H angles, averaged over runs;
    # the |0><0| term against the paper's closed forms
    n, k, T = 20, 10, 1024
    gates = W.noisy_synthesis(W.hadamard_layer(n) * k)
    met, _ = qs.run_trajectories([{"n": n, "gates": gates, "x0": np.zeros(T, np.uint64), "first": 0,
                                   "metric": "prob", "target": 0}], p, sigma, seed=1000 + k, dtype="c64",
                                 mode=mode, every=n, with_stats=False)
    if p > 0:
        want = ((1 + (1 - 4 * p / 3) ** k) / 2) ** n
    else:
        want = ((1 + math.exp(-9 * sigma ** 2 * k / 4)) / 2) ** n
    se = met.std() / math.sqrt(T)
    assert abs(met.mean() - want) < 4 * se + 2e-3, (met.mean(), want, se)


@pytest.mark.parametrize("mode", [qs.NOISE_FLIPS, qs.NOISE_DEPOLARIZING])
@pytest.mark.parametrize("max_ops", [0, 6, 60])
def test_fused_trajectories_match_plain_and_oracle(mode, max_ops):
    # the fused path (Pauli frame folded into the gates) against the plain
    # path (flips applied to the states) and the oracle's replay
    n = 11
    seed = 0xABCDEF
    r = W.rng(21)
    x0 = r.integers(0, 1 << n, size=20, dtype=np.uint64)
    k = 333
    groups = [{"n": n, "gates": W.noisy_synthesis(W.qft_circuit(n)), "x0": x0, "first": 0},
              {"n": n, "gates": W.noisy_synthesis(W.grover_circuit(n, k, 6)), "x0": np.zeros(10, np.uint64),
               "first": 20, "metric": "prob", "target": k}]
    p, sigma = 0.01, 0.03
    mf, sf = qs.run_trajectories(groups, p, sigma, seed, dtype="c64", mode=mode, fuse=True, max_ops=max_ops)
    mp, sp = qs.run_trajectories(groups, p, sigma, seed, dtype="c64", mode=mode, fuse=False)
    assert np.array_equal(sf, sp)
    assert np.max(np.abs(mf - mp)) < 2e-5
    assert int(sf[:, :3].sum()) > 20
    for i in (0, 7, 19):
        m, s = oracle_metric(n, groups[0]["gates"], p, sigma, seed, i, int(x0[i]), "fidelity", 0, mode=mode)
        assert list(s) == [int(v) for v in sf[i]]
        assert abs(m - mf[i]) < 2e-5
    for i in (20, 29):
        m, s = oracle_metric(n, groups[1]["gates"], p, sigma, seed, i, 0, "prob", k, mode=mode)
        assert list(s) == [int(v) for v in sf[i]]
        assert abs(m - mf[i]) < 2e-5


@pytest.mark.parametrize("n", [8, 11])
@pytest.mark.parametrize("fuse", [True, False])
def test_gate_flags_period_finding_qft(n, fuse):
    # the QFT experiment of Sec. 5.2 at a size the oracle replays: noiseless
    # preparation of a periodic register, deviated angles on every QFT gate,
    # flips after the phase shifts R_d only; flags change no counter, so the
    # flip events match the oracle bit for bit
    gates, flags = W.period_finding_qft(n, 3, 5)
    assert len(flags) == len(gates)
    x0 = np.zeros(12, np.uint64)
    p, sigma, seed = 0.01, 0.02, 0xF1A65
    mode = qs.NOISE_DEPOLARIZING
    groups = [{"n": n, "gates": gates, "x0": x0, "first": 40, "flags": flags}]
    met, st = qs.run_trajectories(groups, p, sigma, seed, dtype="c64", mode=mode, fuse=fuse)
    flips = 0
    for i in range(12):
        psi, s = oracle.run_trajectory(n, gates, p, sigma, seed, 40 + i, 0, mode=mode, flags=flags)
        ideal = oracle.run(n, gates)
        assert list(s) == [int(v) for v in st[i]], i
        assert abs(abs(oracle.inner(ideal, psi)) ** 2 - met[i]) < 2e-5, i
        flips += int(s[0] + s[1] + s[2])
    assert flips > 5
    # a noiseless run with the flags is the exact periodic-state QFT: 2^r peaks
    m0, s0 = qs.run_trajectories(groups, 0.0, 0.0, seed, dtype="c64", fuse=fuse)
    assert np.all(s0 == 0) and np.max(np.abs(m0 - 1)) < 1e-5


def test_empty_and_degenerate_groups():
    # a group without trajectories contributes nothing; a group without gates
    # keeps every trajectory at its basis state (fidelity 1, probability of x0
    # 1) and draws no flips (flips follow gate steps)
    n = 11
    x0 = np.array([3, 5, 7], np.uint64)
    groups = [{"n": n, "gates": W.noisy_synthesis(W.qft_circuit(n)), "x0": np.zeros(0, np.uint64), "first": 0},
              {"n": n, "gates": [], "x0": x0, "first": 10},
              {"n": n, "gates": [], "x0": x0, "first": 20, "metric": "prob", "target": 5}]
    for fuse in (True, False):
        met, st = qs.run_trajectories(groups, 0.5, 0.1, seed=3, dtype="c64", fuse=fuse)
        assert met.size == 6
        assert np.max(np.abs(met[:3] - 1)) < 1e-6
        assert np.allclose(met[3:], [0.0, 1.0, 0.0], atol=1e-6)
        assert np.all(st == 0)
