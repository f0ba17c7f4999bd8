"""The fused planner's op order (qs_plan_describe), checked on the CPU without
a GPU: every planned op (a SWAP as three C-NOTs) runs exactly once, and the
passes' execution order, applied to a random state, gives the same vector as
program order.  The list scheduler moves an op ahead only past ops it
commutes with; this checks that on circuits with controls inside and outside
the tile, diagonal gates, many-controlled gates and SWAPs."""
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
    ops, order = {}, []
    for line in text.splitlines():
        if line.startswith("op "):
            m = re.match(r"op (\d+) bit=(\d+) cmask=([0-9a-f]+) cval=([0-9a-f]+) u=(.*)$", line)
            u = [float(x) for x in m.group(5).split(",")]
            ops[int(m.group(1))] = (int(m.group(2)), int(m.group(3), 16), int(m.group(4), 16),
                                    np.array([complex(u[2 * k], u[2 * k + 1]) for k in range(4)]).reshape(2, 2))
        elif line.startswith("  order="):
            order += [int(x) for x in line.split("=")[1].split(",") if x]
    return ops, order


def apply(psi, op):
    bit, cmask, cval, u = op
    i = np.arange(psi.size, dtype=np.int64)
    b = 1 << bit
    i0 = i[((i & b) == 0) & ((i & cmask) == cval)]
    i1 = i0 | b
    x, y = psi[i0].copy(), psi[i1].copy()
    psi[i0] = u[0, 0] * x + u[0, 1] * y
    psi[i1] = u[1, 0] * x + u[1, 1] * y


def mixed_circuit(n, seed):
    r = W.rng(seed)
    kinds = ["MATRIX", "H", "X", "Y", "Z", "RY", "RZ", "UR", "UP1", "UP2", "URP1"]
    gates = []
    for layer in range(6):
        for q in range(n):
            kind = kinds[int(r.integers(len(kinds)))]
            ctr = {}
            nc = int(r.choice([0, 0, 1, 2]))
            for c in r.choice([x for x in range(n) if x != q], size=nc, replace=False):
                ctr[int(c)] = int(r.integers(2))
            if kind == "MATRIX":
                gates.append(W.Gate("MATRIX", q, controls=ctr, matrix=W.haar_su2(r)))
            elif kind in ("H", "X", "Y", "Z"):
                gates.append(W.Gate(kind, q, controls=ctr))
            else:
                na = 2 if kind == "URP1" else 1
                gates.append(W.Gate(kind, q, controls=ctr,
                                    angles=tuple(float(v) for v in r.uniform(-math.pi, math.pi, size=na))))
        perm = r.permutation(n)
        for k in range(n // 2):
            gates.append(W.Gate("X", int(perm[2 * k + 1]), controls={int(perm[2 * k]): 1}))
        a, b = (int(v) for v in r.choice(n, size=2, replace=False))
        sw_ctr = {int(r.choice([x for x in range(n) if x not in (a, b)])): 1} if layer % 2 else {}
        gates.append(W.Gate("SWAP", a, target2=b, controls=sw_ctr))
    return gates


def check(n, dtype, gates, seed):
    ops, order = parse(qs.Plan(n, dtype, gates).describe())
    assert sorted(order) == list(range(len(ops)))
    r = W.rng(seed)
    psi0 = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
    a, b = psi0.copy(), psi0.copy()
    for k in range(len(ops)):
        apply(a, ops[k])
    for k in order:
        apply(b, ops[k])
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(psi0))
    return ops, order


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [12, 14, 16])
def test_mixed_circuit_order_is_a_valid_reordering(n, dtype):
    check(n, dtype, mixed_circuit(n, 100 + n), n)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_random_circuit_and_qft_orders(dtype):
    ops, order = check(15, dtype, W.random_circuit(15, 6, seed=15), 1)
    assert order != sorted(order)          # the scheduler did move ops
    check(14, dtype, W.qft_circuit(14), 2)
    check(13, dtype, W.grover_circuit(13, 1234, 3), 3)
