"""Random gate and state generators used by several test files (seeded)."""
import math

import numpy as np

import workloads as W

ALL_KINDS = ["MATRIX", "H", "X", "Y", "Z", "UP1", "UP2", "UR", "URP1", "RY", "RZ"]


def random_gate(r, n, allow_swap=True, kinds=None, max_ctrl=3):
    kinds = list(kinds or ALL_KINDS)
    if allow_swap and n >= 2 and "SWAP" not in kinds:
        kinds.append("SWAP")
    kind = kinds[r.integers(len(kinds))]
    t = int(r.integers(n))
    t2 = -1
    busy = {t}
    if kind == "SWAP":
        t2 = int(r.choice([q for q in range(n) if q != t]))
        busy.add(t2)
    free = [q for q in range(n) if q not in busy]
    nc = int(r.integers(0, min(max_ctrl, len(free)) + 1))
    ctr = {}
    for q in r.permutation(free)[:nc]:
        ctr[int(q)] = int(r.integers(2))
    angles = tuple(float(x) for x in r.uniform(-math.pi, math.pi, size=W.KINDS[kind]))
    m = W.haar_su2(r) * np.exp(1j * r.uniform(0, 2 * math.pi)) if kind == "MATRIX" else None
    return W.Gate(kind, t, target2=t2, controls=ctr, angles=angles, matrix=m)


def random_state(r, n):
    v = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
    return v / np.linalg.norm(v)
