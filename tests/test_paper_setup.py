"""CPU checks of the inputs of the paper's experiments (no GPU): the period of
Shor's step for N = 187, x = 23 and the periodic register the QFT step acts on."""
import math

import numpy as np

import oracle
import workloads as W
from paper_quant_ph_0201042_gb300 import paper


def test_period_of_23_mod_187():
    # 187 = 11 * 17; 23 = 1 (mod 11) and 23 = 6 (mod 17) with ord_17(6) = 16
    assert paper.multiplicative_order(23, 187) == 16
    assert pow(23, 16, 187) == 1 and all(pow(23, r, 187) != 1 for r in range(1, 16))


def test_period_finding_register_and_its_transform():
    # the prepared register is 2^{-(n-r)/2} sum_j |offset + j 2^r>; its QFT has
    # 2^r peaks of magnitude 2^{-r/2} at multiples of 2^{n-r} with phases
    # e^{2 pi i offset y / 2^n} (Sec. 2.3.2 applied to a periodic state)
    n, r, off = 8, 3, 5
    gates, flags = W.period_finding_qft(n, r, off)
    n_prep = sum(1 for f in flags if f == (W.NO_DEVIATION | W.NO_FLIPS))
    prep = oracle.run(n, gates[:n_prep])
    want = np.zeros(1 << n, complex)
    want[off::1 << r] = 2 ** (-(n - r) / 2)
    assert np.linalg.norm(prep - want) < 1e-13
    out = oracle.run(n, gates)
    y = np.arange(0, 1 << n, 1 << (n - r))
    peaks = 2 ** (-r / 2) * np.exp(2j * math.pi * off * y / (1 << n))
    full = np.zeros(1 << n, complex)
    full[y] = peaks
    assert np.linalg.norm(out - full) < 1e-12
    # decoherence only after the controlled phase shifts of the QFT
    rd = [g for g, f in zip(gates, flags) if f == 0]
    assert all(g.kind == "UP1" and g.controls for g in rd) and len(rd) == n * (n - 1) // 2
