"""Measurement gate (qs_measure, Sec. 2.2.3) against the oracle's sequential
cumulative-sum rule on the same amplitudes.  Where r lies within rounding of
a cumulative boundary both neighbouring outcomes are correct; such shots are
checked for validity, all others must match exactly."""
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


def check_outcomes(psi, r, got, exact_sample=None):
    p = np.abs(psi) ** 2
    cdf = np.cumsum(p)
    lo = np.concatenate([[0.0], cdf[:-1]])
    idx = range(len(r)) if exact_sample is None else exact_sample
    for k in idx:
        u = r[k]
        g = int(got[k])
        assert p[g] > 0, (k, g)
        near = np.min(np.abs(cdf - u)) < 1e-12
        want = oracle.measure(psi, u)
        if not near:
            assert g == want, (k, u, g, want)
        else:
            assert lo[g] - 1e-12 <= u < cdf[g] + 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 3, 12, 17])
def test_measure_matches_oracle(dtype, n):
    r = W.rng(40 + n)
    psi = random_state(r, n)
    if n >= 3:
        psi[[1, 2]] = 0          # zero-probability outcomes must never appear
        psi /= np.linalg.norm(psi)
    s = qs.State(n, dtype).from_numpy(psi)
    held = s.to_numpy().astype(np.complex128)   # the amplitudes the GPU holds
    u = r.uniform(0, 1, size=3000)
    got = s.measure(u)
    check_outcomes(held, u, got, exact_sample=range(0, 3000, 7) if n >= 17 else None)


def test_measure_statistics_and_edges():
    n = 20
    st = qs.State(n, "c128").init_basis(0).apply_circuit(W.random_circuit(n, 3, seed=5))
    psi = st.to_numpy()
    p = np.abs(psi) ** 2
    u = W.rng(3).uniform(0, 1, size=1 << 20)
    got = st.measure(u)
    counts = np.bincount(got.astype(np.int64), minlength=1 << n)
    # coarse-grained chi-square over 256 groups of outcomes
    cg = counts.reshape(256, -1).sum(1)
    pg = p.reshape(256, -1).sum(1) * u.size
    chi2 = np.sum((cg - pg) ** 2 / pg)
    assert chi2 < 256 + 6 * np.sqrt(2 * 256), chi2
    # r just below 1 gives the last outcome with non-zero probability
    last = int(np.nonzero(p)[0][-1])
    assert int(st.measure([0.9999999999999999])[0]) in (last, oracle.measure(psi, 0.9999999999999999))
    with pytest.raises(qs.QsimError):
        st.measure([1.0])
    assert st.measure([]).size == 0


def test_measure_basis_state():
    st = qs.State(24, "c64").init_basis(12345)
    assert np.all(st.measure(W.rng(1).uniform(0, 1, size=1000)) == 12345)
