"""A register partitioned over 2^g ranks, one GPU each.

The paper splits the overall matrix of a gate into independent blocks
M_k = S_k phi_k and hands groups of blocks to processors (Sec. 2.2.1).  Over
several GPUs the same split is a partition of the amplitude index: qubits
0 .. g-1 (the most significant index bits, "global" qubits) name the rank,
and rank r holds the 2^(n-g) amplitudes whose top g bits equal r as an
(n-g)-qubit state.  The library plans the circuit for that partition
(qs_shard_plan): gates on local qubits run unchanged on every rank, controls
on global qubits and diagonal gates on global qubits become per-rank
predicates and scalars (qs_shard_localize), and a non-diagonal gate on a
global qubit is preceded by an exchange that swaps the global qubit with a
local one: each rank sends half of its slice to the partner rank that differs
in that bit and receives the partner's half in its place (qs_shard_pack /
qs_shard_unpack around a send/receive).  Reductions end in one
double-precision all-reduce.

This module is the host-side executor: ShardPlan holds the plan, run()
walks it on one rank with an engine (GpuShard: the library's kernels on the
rank's GPU, transport by torch.distributed, NCCL between GPUs) and a process
group.  Argument marshalling and scheduling only: every gate, pack and unpack
runs in the library.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np

from . import (KIND_CODES, QsGate, State, _opts, check, gates_to_abi, lib)

_KIND_NAMES = {v: k for k, v in KIND_CODES.items()}


def abi_to_gates(arr, m: int) -> list:
    """Gate descriptions (workloads.Gate) of m qs_gate entries, the inverse of
    gates_to_abi."""
    import workloads as W
    out = []
    for k in range(m):
        c = arr[k]
        kind = _KIND_NAMES[c.kind]
        ctr = {q: (c.ctrl_val >> q) & 1 for q in range(64) if (c.ctrl_mask >> q) & 1}
        na = W.KINDS[kind]
        mat = None
        if kind == "MATRIX":
            mat = np.array([complex(c.u[j].re, c.u[j].im) for j in range(4)]).reshape(2, 2)
        out.append(W.Gate(kind, c.t, target2=c.t2 if kind == "SWAP" else -1, controls=ctr,
                          angles=tuple(c.theta[j] for j in range(na)), matrix=mat, param=c.param))
    return out


class ShardPlan:
    """qs_shard_plan of `gates` for n qubits over 2^g ranks.

    segments: a list of ("local", start, stop) stretches of the physical gate
    list and ("exchange", t, t2) qubit swaps (t global, t2 local).
    final_pos[q]: the physical qubit of logical qubit q after the circuit."""

    def __init__(self, n: int, g: int, gates: Sequence):
        self.n, self.g = n, g
        src = gates_to_abi(gates)
        need = ctypes.c_size_t()
        check(lib().qs_shard_plan(n, g, src, len(gates), None, 0, ctypes.byref(need), None))
        self.phys = (QsGate * max(1, need.value))()
        fp = (ctypes.c_int32 * n)()
        cnt = ctypes.c_size_t()
        check(lib().qs_shard_plan(n, g, src, len(gates), self.phys, need.value, ctypes.byref(cnt), fp))
        self.m = cnt.value
        self.final_pos = [int(fp[q]) for q in range(n)]
        self.segments: List[Tuple] = []
        start = 0
        for k in range(self.m):
            c = self.phys[k]
            if c.kind == KIND_CODES["SWAP"] and c.t < g:
                if k > start:
                    self.segments.append(("local", start, k))
                self.segments.append(("exchange", c.t, c.t2))
                start = k + 1
        if self.m > start:
            self.segments.append(("local", start, self.m))
        self.exchanges = sum(1 for s in self.segments if s[0] == "exchange")

    def localize(self, start: int, stop: int, rank: int):
        """(qs_gate array, count): rank's gates on its slice for phys[start:stop]."""
        m = stop - start
        seg = (QsGate * max(1, m)).from_buffer(self.phys, start * ctypes.sizeof(QsGate))
        need = ctypes.c_size_t()
        check(lib().qs_shard_localize(self.n, self.g, rank, seg, m, None, 0, ctypes.byref(need)))
        out = (QsGate * max(1, need.value))()
        cnt = ctypes.c_size_t()
        check(lib().qs_shard_localize(self.n, self.g, rank, seg, m, out, need.value, ctypes.byref(cnt)))
        return out, cnt.value

    def exchange_roles(self, t: int, t2: int, rank: int) -> Tuple[int, int, int]:
        """(partner rank, local qubit, half to send and receive) of exchange
        SWAP(t, t2) on `rank`: the rank's bit b of global qubit t selects the
        partner rank ^ (1 << (g-1-t)) and the half whose local qubit t2-g
        equals 1-b."""
        sh = self.g - 1 - t
        b = (rank >> sh) & 1
        return rank ^ (1 << sh), t2 - self.g, 1 - b


def run(plan: ShardPlan, engine, rank: int, dist) -> None:
    """Walks the plan on one rank: local stretches through engine.apply,
    exchanges through engine.pack / engine.unpack and one send/receive with
    the partner over the process group `dist` (torch.distributed)."""
    import torch
    for seg in plan.segments:
        if seg[0] == "local":
            arr, m = plan.localize(seg[1], seg[2], rank)
            if m:
                engine.apply(arr, m)
        else:
            peer, q, v = plan.exchange_roles(seg[1], seg[2], rank)
            send = engine.pack(q, v)
            recv = torch.empty_like(send)
            # moved as (re, im) pairs of reals: every backend carries those
            ops = [dist.P2POp(dist.isend, torch.view_as_real(send), peer),
                   dist.P2POp(dist.irecv, torch.view_as_real(recv), peer)]
            for req in dist.batch_isend_irecv(ops):
                req.wait()
            engine.unpack(q, v, recv)


def global_norm(engine, dist) -> float:
    """sum_i |alpha_i|^2 over all ranks: each rank's double-precision partial
    sum, then one all-reduce."""
    import torch
    t = torch.tensor([engine.norm()], dtype=torch.float64, device=engine.device)
    dist.all_reduce(t)
    return float(t.item())


class GpuShard:
    """One rank's slice of the register on its GPU: an (n-g)-qubit State run
    by the library's kernels; half slices move through device buffers."""

    def __init__(self, plan: ShardPlan, dtype: str = "c128"):
        import torch
        self.plan = plan
        self.state = State(plan.n - plan.g, dtype)
        self.device = self.state.tensor.device
        self._opts = _opts(True)
        self._torch = torch

    def apply(self, arr, m: int) -> None:
        check(lib().qs_apply_circuit(self.state.handle, arr, m, ctypes.byref(self._opts)))

    def pack(self, q: int, v: int):
        buf = self._torch.empty(1 << (self.state.n - 1), dtype=self.state.tensor.dtype, device=self.device)
        check(lib().qs_shard_pack(self.state.handle, q, v, ctypes.c_void_p(buf.data_ptr())))
        self._torch.cuda.current_stream().synchronize()
        return buf

    def unpack(self, q: int, v: int, buf) -> None:
        check(lib().qs_shard_unpack(self.state.handle, q, v, ctypes.c_void_p(buf.data_ptr())))

    def norm(self) -> float:
        return self.state.norm()
