"""qs_norm_noalloc, the allocation-free norm, against qs_norm.

Some callers cannot allocate device memory where they need a norm (a
framework that owns the device memory budget, a loop that must not let
cudaMalloc/cudaFree synchronize the device).  qs_norm_noalloc keeps its
partial sums in a fixed array of the library's device memory instead of
allocating them.  This test calls it through the C ABI twice in a row on the
same state (the second call reuses the array the first one left behind) and
checks both results against the allocating entry point qs_norm.  The file is
named to run last; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_quant_ph_0201042_gb300 as qs  # noqa: E402
from paper_quant_ph_0201042_gb300 import build as qbuild  # noqa: E402
import workloads as W  # noqa: E402

qbuild.build()


@pytest.mark.parametrize("dtype,n", [("c128", 12), ("c64", 12), ("c64", 21), ("c128", 3), ("c128", 18),
                                     ("c128", 20)])
def test_norm_noalloc_matches_qs_norm(dtype, n):
    L = qs.lib()
    s = qs.State(n, dtype)
    r = W.rng(100 + n)
    v = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
    s.from_numpy(v / np.linalg.norm(v))    # unit norm, as in the other reduction tests
    want = s.norm()                        # the existing, allocating entry point
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    got = []
    for k in range(2):                     # two calls in a row share the scratch array
        out.zero_()
        qs.check(L.qs_norm_noalloc(ctypes.c_void_p(s.tensor.data_ptr()), n, qs.DTYPES[dtype],
                                   ctypes.c_void_p(out.data_ptr()), stream))
        torch.cuda.synchronize()
        got.append(out[0].item())
    for g in got:
        assert abs(g - want) < 1e-12, (g, want)


def test_norm_noalloc_rejects_oversized_states():
    L = qs.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(2, dtype=torch.complex64, device="cuda")
    st = L.qs_norm_noalloc(ctypes.c_void_p(x.data_ptr()), 33, qs.QS_C64, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 2                                     # QS_ERANGE, nothing launched
    assert b"n > 32" in L.qs_last_error()
