"""The fused adjoint sweep's host-side plan (qs_adjoint_describe), checked on
the CPU without a GPU: every reverse step is scheduled exactly once; within a
run every non-diagonal step targets one of the run's (at most three) bits, and
the leading steps a run folds into its load are exchanges on its bits; non-diagonal targets lie in the pass's
tile; and the scheduled order of U^dagger factors, applied to a random state,
gives the same vector as the program's reverse order (the reordering only
moves steps past steps they commute with)."""
import math
import re

import numpy as np
import pytest

import paper_quant_ph_0201042_gb300 as qs
from paper_quant_ph_0201042_gb300 import build as qbuild
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def libpath():
    return qbuild.build()


def parse(text):
    steps, passes = {}, []
    for line in text.splitlines():
        if line.startswith("step "):
            m = re.match(r"step (\d+) cls=(\w+) bit=(\d+) cmask=([0-9a-f]+) cval=([0-9a-f]+) u=(.*)$", line)
            u = [float(x) for x in m.group(6).split(",")]
            steps[int(m.group(1))] = {
                "cls": m.group(2), "bit": int(m.group(3)), "cmask": int(m.group(4), 16), "cval": int(m.group(5), 16),
                "u": np.array([complex(u[2 * k], u[2 * k + 1]) for k in range(4)]).reshape(2, 2)}
        elif line.startswith("pass "):
            tile = [int(x) for x in line.split("tile=")[1].split(",")]
            passes.append({"tile": tile, "runs": []})
        elif line.startswith("run "):
            m = re.match(r"run bit=(-?\d+) bit2=(-?\d+) bit3=(-?\d+) pre=(\d+) steps=(.*)$", line)
            passes[-1]["runs"].append({"bit": int(m.group(1)), "bit2": int(m.group(2)), "bit3": int(m.group(3)),
                                       "pre": int(m.group(4)), "steps": [int(x) for x in m.group(5).split(",") if x]})
    return steps, passes


def apply_dagger(psi, st):
    """psi <- U^dagger psi on the pairs of st's target bit whose controls hold."""
    n_amp = psi.size
    i = np.arange(n_amp, dtype=np.int64)
    b = 1 << st["bit"]
    sel = ((i & b) == 0) & ((i & st["cmask"]) == st["cval"])
    i0 = i[sel]
    i1 = i0 | b
    ud = np.conj(st["u"]).T
    x, y = psi[i0].copy(), psi[i1].copy()
    psi[i0] = ud[0, 0] * x + ud[0, 1] * y
    psi[i1] = ud[1, 0] * x + ud[1, 1] * y


def mixed_circuit(n, seed):
    r = W.rng(seed)
    kinds = ["RY", "RZ", "UR", "UP1", "UP2", "URP1", "H", "X"]
    gates, k = [], 0
    for layer in range(5):
        for q in range(n):
            kind = kinds[int(r.integers(len(kinds)))]
            ctr = {}
            if r.random() < 0.35:
                c = int(r.choice([x for x in range(n) if x != q]))
                ctr[c] = int(r.integers(2))
            if kind in ("H", "X"):
                gates.append(W.Gate(kind, q, controls=ctr))
                continue
            na = 2 if kind == "URP1" else 1
            ang = tuple(float(v) for v in r.uniform(-math.pi, math.pi, size=na))
            gates.append(W.Gate(kind, q, controls=ctr, angles=ang, param=k))
            k += na
        for q in range(layer % 2, n - 1, 2):
            gates.append(W.Gate("X", q + 1, controls={q: 1}))
        a, b = (int(v) for v in r.choice(n, size=2, replace=False))
        gates.append(W.Gate("SWAP", a, target2=b))
    return gates


def check_plan(n, dtype, gates, seed):
    steps, passes = parse(qs.adjoint_describe(n, dtype, gates))
    K = min(n, 12 if dtype == "c64" else 11)
    order = []
    for p in passes:
        assert len(p["tile"]) == K and p["tile"][:5] == [0, 1, 2, 3, 4] and p["tile"] == sorted(p["tile"])
        for run in p["runs"]:
            assert 0 <= run["pre"] <= len(run["steps"])
            for pos, j in enumerate(run["steps"]):
                st = steps[j]
                bits = (run["bit"], run["bit2"], run["bit3"])
                if pos < run["pre"]:
                    assert st["cls"] == "x" and st["bit"] in bits, (j, run)
                if st["cls"] != "diag":
                    assert st["bit"] in bits, (j, run)
                    assert st["bit"] in p["tile"], (j, p["tile"])
                    assert not (st["cmask"] >> st["bit"]) & 1
            if run["bit"] == -1:
                assert all(steps[j]["cls"] == "diag" for j in run["steps"])
            order += run["steps"]
    assert sorted(order) == list(range(len(steps)))
    r = W.rng(seed)
    psi0 = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
    a, b = psi0.copy(), psi0.copy()
    for j in reversed(range(len(steps))):
        apply_dagger(a, steps[j])
    for j in order:
        apply_dagger(b, steps[j])
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(psi0))
    return steps, passes


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [11, 13, 14])
def test_mixed_circuit_plan_is_a_valid_reordering(n, dtype):
    check_plan(n, dtype, mixed_circuit(n, 40 + n), 7 + n)


def test_ansatz_runs_group_three_targets():
    # the gradient workload's layer reversed: C-NOT(q-1, q), RZ(q), RY(q) share
    # target q, and a run takes up to three such targets, so it holds about
    # nine steps
    n = 13
    gates, _ = W.ansatz_circuit(n, 3, seed=5)
    steps, passes = check_plan(n, "c64", gates, 3)
    runs = [run for p in passes for run in p["runs"]]
    assert len(runs) <= len(steps) // 6, (len(runs), len(steps))
    assert sum(1 for run in runs if run["bit3"] >= 0) >= 0.6 * len(runs)


@pytest.mark.parametrize("n", [5, 10])
def test_small_registers_have_no_fused_plan(n):
    # the fused sweep needs a tile of one octet per thread (2^11 amplitudes)
    gates, _ = W.ansatz_circuit(n, 2, seed=1)
    steps, passes = parse(qs.adjoint_describe(n, "c64", gates))
    assert len(steps) == len(gates) and passes == []
