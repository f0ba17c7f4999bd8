"""The partitioned register's device side on one GPU: qs_shard_pack /
qs_shard_unpack and every rank's localized gates run by the library's
kernels, the ranks' slices held as separate states on the same GPU and the
exchanges done rank pair by rank pair from the host (the transport between
GPUs is the caller's; nothing here waits on another rank's kernel).  The
gathered state, put back in logical qubit order, is compared with the CPU
oracle's run of the whole register."""
import ctypes

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
from paper_quant_ph_0201042_gb300 import shard as S  # noqa: E402

qbuild.build()
TOL = {"c128": 1e-12, "c64": 1e-5}


def test_pack_unpack_round_trip():
    n = 13
    psi = random_state(W.rng(1), n)
    for dtype in ("c128", "c64"):
        s = qs.State(n, dtype).from_numpy(psi)
        want = s.to_numpy()
        for q in (0, 4, 7, 12):
            for v in (0, 1):
                buf = torch.empty(1 << (n - 1), dtype=s.tensor.dtype, device="cuda")
                qs.check(qs.lib().qs_shard_pack(s.handle, q, v, ctypes.c_void_p(buf.data_ptr())))
                ref = want.reshape(1 << q, 2, -1)[:, v, :].reshape(-1)
                assert np.array_equal(buf.cpu().numpy(), ref)
                buf.zero_()
                qs.check(qs.lib().qs_shard_unpack(s.handle, q, v, ctypes.c_void_p(buf.data_ptr())))
                got = s.to_numpy().reshape(1 << q, 2, -1)
                assert not np.any(got[:, v, :]) and np.array_equal(got[:, 1 - v, :],
                                                                    want.reshape(1 << q, 2, -1)[:, 1 - v, :])
                s.from_numpy(want)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("g", [1, 2])
def test_ranks_on_one_gpu_match_the_whole_register(dtype, g):
    n = 14
    r = W.rng(50 + g)
    gates = [random_gate(r, n, max_ctrl=2) for _ in range(100)] + W.random_circuit(n, 4, seed=g)
    psi = random_state(W.rng(2), n)
    plan = S.ShardPlan(n, g, gates)
    assert plan.exchanges > 0
    R, nl = 1 << g, n - g
    st = [qs.State(nl, dtype).from_numpy(psi[k << nl:(k + 1) << nl]) for k in range(R)]
    opts = qs._opts(True)
    for seg in plan.segments:
        if seg[0] == "local":
            for k in range(R):
                arr, m = plan.localize(seg[1], seg[2], k)
                if m:
                    qs.check(qs.lib().qs_apply_circuit(st[k].handle, arr, m, ctypes.byref(opts)))
        else:
            bufs = []
            for k in range(R):
                peer, q, v = plan.exchange_roles(seg[1], seg[2], k)
                b = torch.empty(1 << (nl - 1), dtype=st[k].tensor.dtype, device="cuda")
                qs.check(qs.lib().qs_shard_pack(st[k].handle, q, v, ctypes.c_void_p(b.data_ptr())))
                bufs.append((peer, q, v, b))
            for k in range(R):
                peer, q, v, _ = bufs[k]
                qs.check(qs.lib().qs_shard_unpack(st[k].handle, q, v, ctypes.c_void_p(bufs[peer][3].data_ptr())))
    torch.cuda.synchronize()
    phys = np.concatenate([s.to_numpy().astype(np.complex128) for s in st])
    got = np.transpose(phys.reshape([2] * n), axes=plan.final_pos).reshape(-1)
    want = oracle.run(n, gates, psi=psi)
    assert float(np.linalg.norm(got - want)) < TOL[dtype]
    assert abs(sum(s.norm() for s in st) - 1) < TOL[dtype]
