"""The partitioned register (qs_shard_plan / qs_shard_localize and the
executor in paper_quant_ph_0201042_gb300/shard.py), on the CPU.

The paper's block decomposition (Sec. 2.2.1) spread over 2^g ranks: qubits
0 .. g-1 name the rank, rank r holds the amplitudes whose top g bits equal r.
Here the local gates of every rank run in the CPU oracle (the test's engine),
the exchanges move half slices between ranks, and the gathered state, put
back in logical qubit order, is compared with the oracle's run of the whole
circuit on the whole register.  Exchanges only move data and a rank applies
the same gate to the same amplitude pairs as the whole-register run, so the
results agree to the last bits.  The multi-rank tests run world-size 2 and 4
gloo process groups.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from paper_quant_ph_0201042_gb300 import build as qbuild  # noqa: E402
from paper_quant_ph_0201042_gb300 import shard as S  # noqa: E402
from _util import random_gate, random_state  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


def to_logical(phys, n, final_pos):
    """Physical-order vector -> logical order: logical qubit q is physical
    qubit final_pos[q] (qubit 0 the most significant index bit)."""
    return np.transpose(phys.reshape([2] * n), axes=final_pos).reshape(-1)


def mixed_circuit(n, seed, m=120):
    r = W.rng(seed)
    gates = [random_gate(r, n, max_ctrl=2) for _ in range(m)]
    # gates on the top qubits of every kind, controls on them, diagonals on them
    gates += [W.Gate("MATRIX", 0, matrix=W.haar_su2(r)), W.Gate("H", 1, controls={0: 1}),
              W.Gate("RZ", 0, angles=(0.7,)), W.Gate("UP1", 1, angles=(0.3,), controls={5: 1, 0: 0}),
              W.Gate("SWAP", 0, target2=n - 1), W.Gate("SWAP", 1, target2=3, controls={2: 1})]
    gates += W.random_circuit(n, 3, seed=seed)
    return gates


@pytest.mark.parametrize("g", [1, 2, 3])
def test_plan_on_the_whole_register(g):
    # the physical list run on the whole register (an exchange is a SWAP of a
    # global and a local qubit there) is the circuit up to the final qubit order
    n = 10
    gates = mixed_circuit(n, 40 + g)
    plan = S.ShardPlan(n, g, gates)
    phys = S.abi_to_gates(plan.phys, plan.m)
    assert plan.exchanges > 0
    for x in phys:
        if x.kind == "SWAP":
            assert x.target < g <= x.target2 and not x.controls       # only exchanges remain
        elif x.target < g:
            assert x.kind in ("RZ", "UP1", "UP2", "Z") or (x.kind == "MATRIX" and abs(x.matrix[0, 1]) == 0
                                                           and abs(x.matrix[1, 0]) == 0)
    psi = random_state(W.rng(7), n)
    got = to_logical(oracle.run(n, phys, psi=psi), n, plan.final_pos)
    want = oracle.run(n, gates, psi=psi)
    assert np.max(np.abs(got - want)) < 1e-13


def run_ranks_in_one_process(n, g, gates, psi):
    """Every rank's part of the schedule, in one process: localized gates on
    each slice (oracle), exchanges as numpy half-slice swaps."""
    plan = S.ShardPlan(n, g, gates)
    R = 1 << g
    nl = n - g
    sl = [psi[r << nl:(r + 1) << nl].copy() for r in range(R)]
    for seg in plan.segments:
        if seg[0] == "local":
            for r in range(R):
                arr, m = plan.localize(seg[1], seg[2], r)
                if m:
                    sl[r] = oracle.run(nl, S.abi_to_gates(arr, m), psi=sl[r])
        else:
            sent = {}
            for r in range(R):
                peer, q, v = plan.exchange_roles(seg[1], seg[2], r)
                sent[r] = (peer, q, v, half(sl[r], nl, q, v).copy())
            for r in range(R):
                peer, q, v, _ = sent[r]
                set_half(sl[r], nl, q, v, sent[peer][3])
    return to_logical(np.concatenate(sl), n, plan.final_pos), plan


def half(v, nl, q, val):
    return v.reshape(1 << q, 2, -1)[:, val, :].reshape(-1)


def set_half(v, nl, q, val, data):
    v.reshape(1 << q, 2, -1)[:, val, :] = data.reshape(1 << q, -1)


@pytest.mark.parametrize("g", [1, 2, 3])
def test_ranks_exchange_half_slices(g):
    n = 10
    gates = mixed_circuit(n, 70 + g)
    psi = random_state(W.rng(8), n)
    got, plan = run_ranks_in_one_process(n, g, gates, psi)
    want = oracle.run(n, gates, psi=psi)
    assert np.max(np.abs(got - want)) < 1e-13
    # the throughput workload's layers: every layer touches the global qubits
    gates = W.random_circuit(n, 6, seed=11)
    got, plan = run_ranks_in_one_process(n, g, gates, psi)
    assert np.max(np.abs(got - oracle.run(n, gates, psi=psi))) < 1e-13
    assert plan.exchanges <= 2 * 6 * g        # about one exchange per global qubit per layer


def test_localize_drops_and_scales():
    # rank bits decide global controls; a diagonal on a global qubit becomes
    # this rank's entry on the slice
    n, g = 6, 2
    gates = [W.Gate("X", 3, controls={0: 1}), W.Gate("UP1", 1, angles=(0.5,)), W.Gate("Z", 0, controls={4: 1})]
    plan = S.ShardPlan(n, g, gates)
    assert plan.exchanges == 0
    per_rank = {}
    for r in range(4):
        arr, m = plan.localize(0, plan.m, r)
        per_rank[r] = S.abi_to_gates(arr, m)
    # rank 0 (bits 00): X dropped, UP1 entry 1 dropped, Z entry 1 dropped
    assert per_rank[0] == []
    # rank 3 (bits 11): X on local qubit 1; e^{0.5 i} on the slice; -1 where local qubit 2 is 1
    k3 = per_rank[3]
    assert [x.kind for x in k3] == ["X", "MATRIX", "MATRIX"]
    assert k3[0].target == 1 and not k3[0].controls
    assert np.allclose(np.diag(k3[1].matrix), [np.exp(0.5j)] * 2)
    assert k3[2].controls == {2: 1} and np.allclose(np.diag(k3[2].matrix), [-1, -1])


def test_plan_rejects_bad_input():
    from paper_quant_ph_0201042_gb300 import QsimError
    with pytest.raises(QsimError):
        S.ShardPlan(4, 3, [W.Gate("H", 0)])            # fewer than two local qubits
    with pytest.raises(QsimError):
        S.ShardPlan(4, 1, [W.Gate("H", 4)])            # qubit out of range


# ---------------------------------------------------------------------------
# gloo process groups: one process per rank, exchanges by send/receive
# ---------------------------------------------------------------------------

class NumpyShard:
    """The test's engine: one rank's slice as a numpy vector, gates by the
    oracle, half slices as CPU tensors."""

    def __init__(self, plan, vec):
        self.plan = plan
        self.nl = plan.n - plan.g
        self.v = vec.copy()
        self.device = "cpu"

    def apply(self, arr, m):
        self.v = oracle.run(self.nl, S.abi_to_gates(arr, m), psi=self.v)

    def pack(self, q, val):
        return torch.from_numpy(half(self.v, self.nl, q, val).copy())

    def unpack(self, q, val, buf):
        set_half(self.v, self.nl, q, val, buf.numpy())

    def norm(self):
        return float(np.vdot(self.v, self.v).real)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, seed, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = world.bit_length() - 1
        gates = mixed_circuit(n, seed)
        psi = random_state(W.rng(seed + 1), n)
        plan = S.ShardPlan(n, g, gates)
        nl = n - g
        eng = NumpyShard(plan, psi[rank << nl:(rank + 1) << nl])
        S.run(plan, eng, rank, dist)
        nrm = S.global_norm(eng, dist)
        parts = [torch.zeros(1 << nl, 2, dtype=torch.float64) for _ in range(world)] if rank == 0 else None
        dist.gather(torch.view_as_real(torch.from_numpy(eng.v)), parts, dst=0)
        if rank == 0:
            got = to_logical(np.concatenate([torch.view_as_complex(p).numpy() for p in parts]), n, plan.final_pos)
            want = oracle.run(n, gates, psi=psi)
            out["err"] = float(np.max(np.abs(got - want)))
            out["norm"] = nrm
            out["exchanges"] = plan.exchanges
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_match_the_whole_register(world):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, 10, 900 + world, out), nprocs=world, join=True)
    assert out["exchanges"] > 0
    assert out["err"] < 1e-13
    assert abs(out["norm"] - 1.0) < 1e-13
