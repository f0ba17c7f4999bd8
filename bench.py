"""Throughput benchmark of the random-circuit workload: n = 30 qubits, 40 layers
of Haar-random SU(2) gates on every qubit followed by C-NOTs on 15 random
disjoint pairs (1800 gates), complex128 state (16 GiB, the paper's double
precision) by default.

One step = one simulation of the whole circuit from |0...0>: qs_init_basis
followed by the fused circuit plan (every gate of the circuit).  The
complex128 passes compute in double-single arithmetic (the library's default
for complex128; --arith f64 selects double-precision instructions).  Prints
one JSON line (see --help).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype c128|c64]
                  [--arith default|f64] [--no-fuse] [--impl ours|reference]

--impl reference times the CPU oracle (complex128, plain row-by-row gate
application) on the host cores, on a bounded sample of the same workload.
Under torchrun each rank runs an independent replica of the workload (its own
seed); no data crosses ranks; value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

N_QUBITS = 30
LAYERS = 40
SEED = 20260515


def amp_updates(n, gates):
    """Amplitudes changed by each gate's definition: 2^n for a single-qubit
    gate, 2^(n - #controls) for a controlled one."""
    tot = 0
    for g in gates:
        if g.kind == "SWAP":
            tot += 1 << (n - len(g.controls))
        else:
            tot += 1 << (n - len(g.controls))
    return tot


def workload_config(args, n_ranks):
    n = args.n
    # the workload only (the arithmetic each arm uses is in the line's "arith")
    kind = "complex64" if args.dtype == "c64" else "complex128"
    return {
        "workload": "random circuit n=%d, %d layers (Haar SU(2) on every qubit + C-NOTs on %d disjoint pairs), %s state"
                    % (n, LAYERS, n // 2, kind),
        "n_qubits": n, "layers": LAYERS, "gates": LAYERS * (n + n // 2),
        "state_bytes": (8 if args.dtype == "c64" else 16) << n,
        "fused": not args.no_fuse,
        "l2": ("state (%d MiB) larger than L2 (129 MB); no flush needed" % (((8 if args.dtype == "c64" else 16) << n) >> 20)
               if ((8 if args.dtype == "c64" else 16) << n) > (129 << 20) else
               "state (%d MiB) fits L2 (129 MB): a profiling size, not the workload" % (((8 if args.dtype == "c64" else 16) << n) >> 20)),
        "parallelism": "replicas%d" % n_ranks,
    }


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def max_over_ranks(x, dist):
    """The maximum of a per-rank float over all ranks (identity without a
    process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_per_step_rank, units_per_step_rank, world, dist):
    """(ms_per_step, value): the slowest rank's time and the units all ranks
    processed per second (every rank runs the same amount of work)."""
    ms = max_over_ranks(ms_per_step_rank, dist)
    return ms, world * units_per_step_rank / (ms / 1e3)


def cpu_baseline(dtype, budget_s=20.0, n=None):
    """The oracle (complex128, row-by-row, OpenMP over rows) on the host cores,
    on a bounded prefix of the same circuit.  n = 30 when the host has room
    for the state and its out-of-place copy (2 x 16 GiB), else n = 26."""
    import oracle
    try:
        with open("/proc/meminfo") as f:
            avail = int([l for l in f if l.startswith("MemAvailable")][0].split()[1]) * 1024
    except Exception:
        avail = 0
    if n is None:
        n = N_QUBITS if avail > 48 * (1 << 30) else 26
    gates = W.random_circuit(n, LAYERS, seed=SEED)
    psi = oracle.basis(n, 0)
    done, upd = 0, 0
    t0 = time.perf_counter()
    for g in gates:
        psi = oracle.run(n, [g], psi=psi)
        done += 1
        upd += amp_updates(n, [g])
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    del psi
    return {"value": upd / dt, "unit": "amp-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "first %d of %d gates of the workload at n=%d (complex128, OpenMP rows), %.1f s"
                      % (done, len(gates), n, dt),
            "sample_seconds": dt, "full_step_updates": amp_updates(n, gates)}


def run_reference(args, rank, world):
    """--impl reference: the oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    steps = []
    base = None
    for k in range(args.warmup + args.steps):
        b = cpu_baseline(args.dtype, budget_s=args.ref_budget, n=None if args.n == N_QUBITS else args.n)
        if k >= args.warmup:
            steps.append(b)
        base = b
    val = statistics.median([s["value"] for s in steps])
    line = {
        "impl": "reference", "metric": "amp-updates/s", "value": val, "unit": "amp-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        # each timed step is a bounded sample of the workload; ms_per_step is
        # one full step at the measured rate
        "ms_per_step": base["full_step_updates"] / val * 1e3,
        "sample_ms_per_step": statistics.median([s["sample_seconds"] for s in steps]) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": workload_config(args, world),
        "arith": "FP64 (the CPU oracle: plain row-by-row gate application, OpenMP over rows)",
        "cpu_baseline": {"value": val, "unit": "amp-updates/s", "cores": base["cores"],
                         "kind": "oracle", "sample": base["sample"]},
        "e2e": {"value": val, "unit": "amp-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time(torch, fn, reps=1):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# FP32 instructions per changed amplitude of the double-single arithmetic of
# the complex128 fused pass (qs_ds.cuh): a general 2x2 gate makes two
# four-term dot products per amplitude (re, im) of 43 instructions each (four
# exact products with their low-order terms, three TwoSums, the low-order
# sum and a FastTwoSum)
DS_INSTR_GENERAL = 86
# DRAM bytes (read + write) of one complex128 double-single pass at n = 26,
# from one ncu capture of k_fused_ds (2.0866 GB against 2.147 GB algorithmic);
# a pass moves every amplitude once, so a launch at n scales by 2^(n-26)
DS_TRAFFIC_N26 = 2.0866e9
# the same for the complex64 pass k_fused_c64 (1013.5 MB per n = 26 launch)
C64_TRAFFIC_N26 = 1013.5e6


def general_gates(gates):
    return sum(1 for g in gates if g.kind == "MATRIX")


def rooflines(args, n, gates, kern_ms_step, launches_step, sm_mhz, sms, peaks):
    """Roofline views of the dominant kernel from its per-launch device time.
    hbm: one read and one write of the state per pass (fused) or of the
    touched amplitudes per gate (unfused); alu: the arithmetic of the general
    gates (the C-NOTs move no data in the fused passes)."""
    amp_bytes = 8 if args.dtype == "c64" else 16
    hbm_peak, hbm_src = measured_peaks()
    if args.no_fuse:
        bytes_step = sum(2 * amp_bytes * (1 << (n - len(g.controls))) for g in gates)
    else:
        bytes_step = launches_step * 2 * (amp_bytes << n)
    t = kern_ms_step / 1e3
    views = {"hbm": {"achieved": bytes_step / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": bytes_step / t / 1e9 / hbm_peak, "peak_source": hbm_src + " copy bandwidth"}}
    ngen = general_gates(gates)
    issue_peak = sms * 128 * sm_mhz * 1e6          # FP32 lanes x SM clock (instructions/s)
    fp64_flops = ngen * 16 * (1 << n)              # 8 double multiply-adds per amplitude
    ds = args.dtype == "c128" and args.arith != "f64"
    if ds:
        instr = ngen * DS_INSTR_GENERAL * (1 << n)
        views["alu"] = {"achieved": instr / t / 1e12, "peak": issue_peak / 1e12, "unit": "T FP32 instr/s",
                        "frac": instr / t / issue_peak,
                        "peak_source": "%d SMs x 128 FP32 lanes x %.0f MHz (measured SM clock)" % (sms, sm_mhz),
                        "peak_measured_ffma": peaks["f32"] / 1e12,
                        "work": "%d FP32 instructions per amplitude per general gate (double-single)"
                                % DS_INSTR_GENERAL}
        views["fp64_equivalent"] = {"achieved": fp64_flops / t / 1e12, "unit": "TFLOP/s (FP64 flops of the gates)",
                                    "fp64_pipe_peak_measured": 2 * peaks["f64"] / 1e12,
                                    "ratio_to_fp64_pipe": fp64_flops / t / (2 * peaks["f64"])}
    elif args.dtype == "c128":
        views["alu"] = {"achieved": fp64_flops / t / 1e12, "peak": 2 * peaks["f64"] / 1e12, "unit": "TFLOP/s",
                        "frac": fp64_flops / t / (2 * peaks["f64"]),
                        "peak_source": "measured FP64 FMA rate (qs_alu_peak) x 2 flops"}
    else:
        flops = ngen * 16 * (1 << n)
        peak = sms * 128 * 2 * sm_mhz * 1e6
        views["alu"] = {"achieved": flops / t / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                        "frac": flops / t / peak,
                        "peak_source": "%d SMs x 128 FP32 lanes x 2 flops x %.0f MHz (measured SM clock)" % (sms, sm_mhz),
                        "peak_measured_ffma": 2 * peaks["f32"] / 1e12}
    t_hbm = bytes_step / (hbm_peak * 1e9)
    t_alu = views["alu"]["achieved"] * t / views["alu"]["peak"] if "peak" in views["alu"] else 0.0
    bound = "alu" if t_alu > t_hbm else "hbm"
    main = views[bound]
    if args.no_fuse:
        traffic, kern = None, "k_pair_ds" if ds else "k_pair"
    elif ds:
        traffic, kern = DS_TRAFFIC_N26 * (1 << (n - 26)), "k_fused_ds"
    elif args.dtype == "c64":
        traffic, kern = C64_TRAFFIC_N26 * (1 << (n - 26)), "k_fused_c64"
    else:
        traffic, kern = None, "k_fused<double,4>"
    return {"bound": bound, "achieved": main["achieved"], "peak": main["peak"], "unit": main["unit"],
            "frac": main["frac"], "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": kern,
            "peak_source": main["peak_source"], "views": views}


def e2e_pipelined(torch, qs, state, n, dtype, garr, n_gates, opts, k, dist, local):
    """k end-to-end steps through the public C ABI, alternating between two
    states on two streams: each step initialises its state, applies the
    circuit (gate list copied in from host memory) and enqueues the copy of the
    whole result to its own pinned host buffer (qs_copy_out_async), so that a
    step's copy runs while the next step computes.  The timed region ends when
    both streams are idle, i.e. after the last copy."""
    import ctypes
    L = qs.lib()
    cdt = torch.complex64 if dtype == "c64" else torch.complex128
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    other = qs.State(n, dtype, stream=streams[1])
    old_stream = state.stream
    qs.check(L.qs_set_stream(state.handle, ctypes.c_void_p(streams[0].cuda_stream)))
    try:
        hosts = [torch.empty(1 << n, dtype=cdt, pin_memory=True) for _ in range(2)]
        bufs = [h.numpy() for h in hosts]
        sts = [state, other]

        def step(i):
            st, b = sts[i % 2], bufs[i % 2]
            qs.check(L.qs_init_basis(st.handle, 0))
            qs.check(L.qs_apply_circuit(st.handle, garr, n_gates, ctypes.byref(opts)))
            qs.check(L.qs_copy_out_async(st.handle, b.ctypes.data_as(ctypes.c_void_p), b.nbytes))

        def drain():
            for st in sts:
                qs.check(L.qs_sync(st.handle))

        step(0)
        step(1)
        drain()
        if dist:
            dist.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        t0 = time.perf_counter()
        for i in range(k):
            step(i)
        drain()
        dt = max_over_ranks((time.perf_counter() - t0) / k, dist)
        clocks = sampler.stop()
        return {"ms_per_step": dt * 1e3, "steps": k, "pipelined": True, "states": 2, "streams": 2,
                "clocks": clocks, "host_buffers_pinned": all(bool(h.is_pinned()) for h in hosts),
                "note": "every step copies its gate list in and its whole state out inside the timed region; "
                        "a step's copy-out overlaps the next step's passes, and the two independent circuits "
                        "overlap each other's pass tails, so this can come out below the single-stream "
                        "device-timed step"}
    finally:
        # both streams idle before the second state goes and the first moves back
        L.qs_sync(other.handle)
        L.qs_sync(state.handle)
        qs.check(L.qs_set_stream(state.handle, ctypes.c_void_p(old_stream.cuda_stream)))
        other.close()


def _release(torch):
    release = getattr(torch._C, "_host_emptyCache", None)
    if release is not None:
        release()
    torch.cuda.empty_cache()


def secondary(args, torch, qs, state128, peaks, sms, sm_mhz):
    """The other measurements the metric and the workloads name, each on its
    own workload: the complex64 state at n = 30 (same circuit) and its
    distance to the complex128 result, double-precision instructions against
    double-single at n = 28, the unfused per-gate path, the FFT QFT, the
    adjoint gradient against measured finite differences and parameter
    shifts, the 4096-trajectory batch, and Grover n = 24."""
    import ctypes
    from paper_quant_ph_0201042_gb300 import paper
    out = {}
    n = args.n
    gates = W.random_circuit(n, LAYERS, seed=SEED)
    upd = amp_updates(n, gates)
    ngen = general_gates(gates)
    hbm_peak = measured_peaks()[0]

    # complex64 state, same circuit: throughput, roofline, distance to complex128
    p64 = qs.Plan(n, "c64", gates)
    s64 = qs.State(n, "c64")
    step64 = lambda: (s64.init_basis(0), p64.execute(s64))
    step64()
    ms64 = _time(torch, step64, reps=3)
    p64.set_timing(True)
    p64.timing()
    step64()
    kms, kn = p64.timing()
    p64.set_timing(False)
    flops = ngen * 16 * (1 << n)
    fpk = sms * 128 * 2 * sm_mhz * 1e6
    c64 = {"value": upd / (ms64 / 1e3), "unit": "amp-updates/s", "ms_per_step": ms64, "passes": p64.launches,
           "roofline": {"bound": "alu", "kernel": "k_fused_c64", "achieved": flops / (kms / 1e3) / 1e12,
                        "peak": fpk / 1e12, "unit": "TFLOP/s", "frac": flops / (kms / 1e3) / fpk,
                        "hbm_gbs": kn * 2 * (8 << n) / (kms / 1e3) / 1e9,
                        "hbm_frac": kn * 2 * (8 << n) / (kms / 1e3) / 1e9 / hbm_peak,
                        "traffic": C64_TRAFFIC_N26 * (1 << (n - 26))}}
    if state128 is not None:
        d = (s64.tensor.to(torch.complex128) - state128.tensor).abs().pow(2).sum().sqrt().item()
        c64["state_error_vs_c128"] = d
    out["c64"] = c64

    # double-precision reductions (norm, Pauli expectation, inner product) at
    # n = 30: bytes read per call against HBM; per-thread float-pair
    # accumulation, double precision across threads
    red = {}
    zstr, xstr = "Z" * n, "X" + "Z" * (n - 1)
    for dt_name, st, B in (("c64", s64, 8), ("c128", state128, 16)):
        if st is None:
            continue
        other = qs.State(n, dt_name).init_basis(0)
        r = {}
        for name, fn, nbytes in (("norm", lambda: st.norm(), B << n),
                                 ("expect_Z", lambda: st.expect(zstr), B << n),
                                 ("expect_XZ", lambda: st.expect(xstr), B << n),
                                 ("inner", lambda: st.inner(other), 2 * (B << n))):
            fn()
            ms = _time(torch, fn, reps=5)
            r[name] = {"ms": ms, "hbm_gbs": nbytes / (ms / 1e3) / 1e9,
                       "frac_of_measured_hbm": nbytes / (ms / 1e3) / 1e9 / hbm_peak}
        r["fp64_pipe_ms_if_two_dfma_per_amplitude"] = (2 << n) / peaks["f64"] * 1e3
        red[dt_name] = r
        other.close()
    out["reductions_n30"] = red
    s64.close()
    del p64
    _release(torch)

    # double-precision instructions against double-single, n = 28 (the n = 30
    # step with doubles takes about 18 s): time and the distance of the states
    nd = 28
    gd = W.random_circuit(nd, LAYERS, seed=SEED)
    res = {}
    sts = {}
    for ar in ("f64", "default"):
        pl = qs.Plan(nd, "c128", gd, arith=ar)
        st = qs.State(nd, "c128")
        run = lambda: (st.init_basis(0), pl.execute(st))
        run()
        ms = _time(torch, run)
        res[ar] = {"ms": ms, "passes": pl.launches, "value": amp_updates(nd, gd) / (ms / 1e3)}
        sts[ar] = st
        del pl
    dd = (sts["f64"].tensor - sts["default"].tensor).abs().pow(2).sum().sqrt().item()
    out["c128_f64_vs_double_single_n28"] = {
        "workload": "random circuit n=28, 40 layers, complex128", "f64_instructions": res["f64"],
        "double_single": res["default"], "speedup": res["f64"]["ms"] / res["default"]["ms"],
        "fp64_peak_measured_tflops": 2 * peaks["f64"] / 1e12,
        "f64_fraction_of_fp64_pipe": general_gates(gd) * 16 * (1 << nd) / (res["f64"]["ms"] / 1e3)
                                     / (2 * peaks["f64"]),
        "state_distance": dd}
    for st in sts.values():
        st.close()
    _release(torch)

    # unfused per-gate path (one pair sweep per gate, the paper's evolution
    # step as written) on the first two layers of the n = 30 circuit: every
    # gate reads and writes the amplitudes it touches once, so the HBM
    # fraction is the figure of merit
    pre = gates[:2 * (n + n // 2)]
    unf = {}
    for name, dt_u, ar_u, B in (("c128_double_single", "c128", "default", 16), ("c128_f64", "c128", "f64", 16),
                                ("c64", "c64", "default", 8)):
        if dt_u == "c128" and state128 is None:
            continue
        su = state128 if dt_u == "c128" else qs.State(n, "c64")
        pu = qs.Plan(n, dt_u, pre, fuse=False, arith=ar_u)
        run = lambda: pu.execute(su)
        run()
        ms = _time(torch, run, reps=2 if name != "c128_f64" else 1)
        ub = sum(2 * B * (1 << (n - len(g.controls))) for g in pre)
        unf[name] = {"ms": ms, "gates_per_s": len(pre) / (ms / 1e3),
                     "amp_updates_per_s": amp_updates(n, pre) / (ms / 1e3),
                     "hbm_gbs": ub / (ms / 1e3) / 1e9, "hbm_frac": ub / (ms / 1e3) / 1e9 / hbm_peak}
        del pu
        if su is not state128:
            su.close()
        _release(torch)
    if unf:
        unf["workload"] = ("first 2 of the 40 layers of the n=%d random circuit (%d gates), one pair-sweep launch "
                           "per gate; bytes = one read and one write of the amplitudes each gate touches" % (n, len(pre)))
        unf["arith"] = {"c128_double_single": "double-single (the default for complex128)",
                        "c128_f64": "double-precision instructions (FP64-pipe bound on this part)",
                        "c64": "FP32 instructions"}
        out["unfused_n30"] = unf

    # the QFT black box (FFT, Sec. 2.3.2), complex64 n = 30: 4 transform
    # passes and a bit-reversal pass, each one read + one write
    sq = qs.State(n, "c64").init_basis(12345)
    sq.qft()
    t = _time(torch, lambda: sq.qft(), reps=3)
    nbytes = 5 * 2 * (8 << n)
    out["qft_fft_c64"] = {"workload": "QFT of all %d qubits by the FFT (qs_qft), complex64" % n, "ms": t,
                          "hbm_gbs_5_passes": nbytes / (t / 1e3) / 1e9,
                          "frac_of_measured_hbm": nbytes / (t / 1e3) / 1e9 / hbm_peak}
    sq.close()
    _release(torch)

    # adjoint gradient at n = 26 (complex64) against measured finite
    # differences and parameter shifts on a few angles, and the plain per-step
    # sweep with double instructions on a complex128 state
    na = 26
    agates, aparams = W.ansatz_circuit(na, 25, seed=2026)
    pauli = "Z" + "I" * (na - 1)
    work = qs.State(na, "c64")
    qs.adjoint_grad(work, agates, aparams, pauli=pauli)
    t_adj = _time(torch, lambda: qs.adjoint_grad(work, agates, aparams, pauli=pauli), reps=3)
    pf = qs.Plan(na, "c64", agates)
    fwd = lambda: (work.init_basis(0), pf.execute(work), work.expect(pauli))
    fwd()
    t_fwd = _time(torch, fwd, reps=3)

    def energy(prm):
        gs = [W.Gate(g.kind, g.target, controls=g.controls,
                     angles=((float(prm[g.param]),) if g.param >= 0 else g.angles), param=g.param)
              for g in agates]
        work.init_basis(0).apply_circuit(gs)
        return work.expect(pauli)

    sample = [0, 333, 777, 1299]
    t0 = time.perf_counter()
    for k in sample:                    # central differences, h = 1e-4
        for sgn in (1, -1):
            prm = aparams.copy()
            prm[k] += sgn * 1e-4
            energy(prm)
    t_fd = (time.perf_counter() - t0) / len(sample)
    t0 = time.perf_counter()
    for k in sample:                    # parameter shift: E(t + pi/2) - E(t - pi/2), over 2
        for sgn in (1, -1):
            prm = aparams.copy()
            prm[k] += sgn * math.pi / 2
            energy(prm)
    t_ps = (time.perf_counter() - t0) / len(sample)
    n_par = aparams.size
    work.close()
    del pf
    _release(torch)
    w128 = qs.State(na, "c128")
    t0 = time.perf_counter()
    qs.adjoint_grad(w128, agates, aparams, pauli=pauli, fuse=False)
    t_plain = time.perf_counter() - t0
    w128.close()
    _release(torch)
    out["adjoint"] = {
        "workload": "ansatz n=26, 25 layers of RY/RZ + C-NOT ladder, 1300 angles, complex64, <Z_0>",
        "adjoint_ms": t_adj, "forward_ms": t_fwd, "adjoint_over_forward": t_adj / t_fwd,
        "finite_diff_ms_per_angle_measured": t_fd * 1e3, "finite_diff_ms_all_angles": t_fd * 1e3 * n_par,
        "parameter_shift_ms_per_angle_measured": t_ps * 1e3, "parameter_shift_ms_all_angles": t_ps * 1e3 * n_par,
        "speedup_vs_finite_diff": t_fd * 1e3 * n_par / t_adj,
        "speedup_vs_parameter_shift": t_ps * 1e3 * n_par / t_adj,
        "sample": "finite differences and parameter shifts timed end to end (circuit from host gates, forward "
                  "passes, <Z_0>) on angles %s, 2 runs each, then x %d angles" % (sample, n_par),
        "plain_fp64_per_step_sweep_ms": t_plain * 1e3,
        "speedup_vs_plain_fp64": t_plain * 1e3 / t_adj,
        "plain_fp64_note": "qs_adjoint_grad_ex with no_fusion = 1 on a complex128 state: one sweep of both "
                           "vectors per step, double-precision instructions"}

    # batched noisy trajectories
    batch = W.trajectory_batch(4096, ((12, 2), (16, 1), (20, 1)), (12, 16), seed=31337)
    groups = qs.batch_groups(batch)
    qs.run_trajectories(groups, 1e-3, 1e-2, 7, dtype="c64", with_stats=False)
    t0 = time.perf_counter()
    met, _ = qs.run_trajectories(groups, 1e-3, 1e-2, 7, dtype="c64", with_stats=False)
    dt = time.perf_counter() - t0
    hist, _ = np.histogram(met, bins=10, range=(0.0, 1.0))
    method_upd, echo_upd = 0, 0
    for g in groups:
        m = len(g["x0"])
        per = amp_updates(g["n"], g["gates"])
        method_upd += m * per
        if g.get("metric", "fidelity") == "fidelity":
            echo_upd += m * per      # the noiseless inverse circuit that measures the fidelity
    _release(torch)
    t0 = time.perf_counter()
    qs.run_trajectories(groups, 1e-3, 1e-2, 7, dtype="c128", with_stats=False, fuse=False)
    t_plain = time.perf_counter() - t0
    _release(torch)
    out["trajectories"] = {"workload": "4096 trajectories, 12/16/20 qubits 2:1:1, QFT + Grover(12,16), "
                                       "sigma=1e-2, p=1e-3, complex64",
                           "seconds": dt, "trajectories_per_s": len(met) / dt,
                           "amp_updates_per_s": method_upd / dt,
                           "amp_updates_note": "the circuits' own gates; the fidelity echo (the inverse noiseless "
                                               "circuit of the QFT groups, %.3g updates) is overhead and not counted"
                                               % echo_upd,
                           "echo_share_of_updates": echo_upd / (method_upd + echo_upd),
                           "histogram_0_1_10bins": hist.tolist(), "mean_metric": float(met.mean()),
                           "plain_fp64_seconds": t_plain, "speedup_vs_plain_fp64": t_plain / dt,
                           "plain_fp64_note": "qs_run_trajectories with no_fusion = 1 on complex128: one launch "
                                              "per gate step, flips applied to the states, double instructions"}

    # Grover search, n = 24, floor(pi/4 sqrt(2^24)) = 3216 iterations;
    # success probability against sin^2((2j+1) theta), sin theta = 2^-12;
    # complex64 renormalised in double precision every 256 iterations
    gn = 24
    gk = W.basis_index(24, gn)
    git = W.grover_iterations(gn)
    gro = {}
    for dt_name, B in (("c64", 8), ("c128", 16)):
        search = paper.GroverSearch(gn, gk, git, dt_name)
        gs = qs.State(gn, dt_name)
        run = lambda: search.run(gs)
        run()
        ms = _time(torch, run)
        p_succ = gs.prob(gk)
        want = search.closed_form()
        gro[dt_name] = {"ms": ms, "gates_per_s": search.n_gates / (ms / 1e3), "passes": search.launches,
                        "renormalised_every": 256 if search.renorm else None,
                        "hbm_gbs": search.launches * 2.0 * (B << gn) / (ms / 1e3) / 1e9,
                        "success_probability": p_succ, "closed_form": want, "error": abs(p_succ - want)}
        gro[dt_name]["frac_of_measured_hbm"] = gro[dt_name]["hbm_gbs"] / hbm_peak
        gs.close()
        del search
        _release(torch)
    gro["workload"] = "Grover n=24, %d iterations (2 H layers and 2 one-amplitude phase flips per iteration)" % git
    out["grover_n24"] = gro
    return out


def paper_tables(torch, qs):
    """The paper's tables and figures (Sec. 4.2, 4.3, 5.2) on this GPU:
    timings of the HT, the QFT circuit and the FFT black box, and the Monte
    Carlo error experiments (Table hod, Figs. 20d/20o, Table qft16od)."""
    from paper_quant_ph_0201042_gb300 import paper
    out = {"table_qft": paper.table_qft(), "table_qft_c64": paper.table_qft(dtype="c64"),
           "table_ht": paper.table_ht()}
    torch.cuda.empty_cache()
    out["table_qft16od"] = paper.table_qft16()
    out["table_hod"] = paper.table_hod()
    out["fig20"] = paper.fig20()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c128")
    ap.add_argument("--arith", choices=["default", "f64"], default="default",
                    help="complex128 fused passes: double-single (default) or double-precision instructions")
    ap.add_argument("--no-fuse", action="store_true")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the complex64, adjoint, trajectory and Grover measurements")
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--paper-tables", action="store_true",
                    help="run the paper's tables (QFT circuit vs FFT, HT, Table hod, Figs. 20d/20o, "
                         "Table qft16od) and exit")
    ap.add_argument("--qubits", "--n", dest="n", type=int, default=N_QUBITS,
                    help="qubits (profiling of smaller cases; the workload is n=30)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    torch.cuda.set_device(local)
    import paper_quant_ph_0201042_gb300 as qs
    from paper_quant_ph_0201042_gb300 import build as qbuild
    qbuild.build()

    if args.paper_tables:
        if rank == 0:
            print(json.dumps({"paper_tables": paper_tables(torch, qs)}), flush=True)
        return

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = {"f32": qs.alu_peak("f32"), "f64": qs.alu_peak("f64")}
    n = args.n
    gates = W.random_circuit(n, LAYERS, seed=SEED + rank)
    upd = amp_updates(n, gates)
    arith = args.arith if args.dtype == "c128" else "default"
    plan = qs.Plan(n, args.dtype, gates, fuse=not args.no_fuse, arith=arith)
    state = qs.State(n, args.dtype)

    def step():
        state.init_basis(0)
        plan.execute(state)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: device events on the launching stream; no per-launch
    # events inside it
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    ms_per_step, value = aggregate(ev0.elapsed_time(ev1) / args.steps, upd, world, dist)

    # roofline of the dominant kernel: a separate pass of steps with a CUDA
    # event pair around every launch, on the launching stream
    roof_steps = 2
    plan.set_timing(True)
    plan.timing()
    for _ in range(roof_steps):
        step()
    kern_ms, kern_n = plan.timing()
    plan.set_timing(False)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    roof = rooflines(args, n, gates, kern_ms / roof_steps, kern_n / roof_steps, sm_mhz, sms, peaks)
    roof.update({"launches_timed": kern_n, "steps_timed": roof_steps,
                 "kernel_ms_per_launch": kern_ms / max(1, kern_n), "kernel_ms_per_step": kern_ms / roof_steps,
                 "timing": "per-launch CUDA events in a separate pass of %d steps after the timed region"
                           % roof_steps})

    dtype_name = {"c64": "f32", "c128": "f64"}[args.dtype]
    line = {
        "metric": "amp-updates/s", "value": value, "unit": "amp-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_name,
        "arith": ("double-single: each double split into two floats (48 significant bits), gates by "
                  "error-free products and sums on the FP32 pipe; state, copies and reductions in FP64; "
                  "parity vs the FP64 oracle <= 1e-12"
                  if (args.dtype == "c128" and arith != "f64") else
                  ("FP64 instructions" if args.dtype == "c128" else "FP32 instructions, FP64 reductions")),
        "data": "synthetic", "config": workload_config(args, world),
        "gates_per_s": world * len(gates) / (ms_per_step / 1e3),
        "hbm_gbs_algorithmic": world * roof["views"]["hbm"]["achieved"] * roof["kernel_ms_per_step"] / ms_per_step,
        "passes_per_step": plan.launches,
        "roofline": roof,
        "peaks_measured": {"fp32_fma_per_s": peaks["f32"], "fp64_fma_per_s": peaks["f64"], "sms": sms},
        "gpu_launches": args.steps * (plan.launches + 1),
        "clocks": clocks,
    }

    # end to end through the public API with host buffers: the gate list goes
    # in from host memory (qs_apply_circuit copies, plans and launches), the
    # final state comes back to pinned host memory (qs_copy_out)
    if not args.no_e2e:
        import ctypes
        host = torch.empty(1 << n, dtype=torch.complex64 if args.dtype == "c64" else torch.complex128,
                           pin_memory=True)
        hbuf = host.numpy()
        garr = qs.gates_to_abi(gates)
        opts = qs._opts(not args.no_fuse, 0, arith)

        def e2e_step():
            qs.check(qs.lib().qs_init_basis(state.handle, 0))
            qs.check(qs.lib().qs_apply_circuit(state.handle, garr, len(gates), ctypes.byref(opts)))
            qs.check(qs.lib().qs_copy_out(state.handle, hbuf.ctypes.data_as(ctypes.c_void_p), hbuf.nbytes))

        e2e_step()
        if dist:
            dist.barrier()
        k = max(1, min(args.steps, 3))
        esampler = ClockSampler(local)
        esampler.start()
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(k):
            ts = time.perf_counter()
            e2e_step()          # ends with the synchronous copy-out
            step_ms.append((time.perf_counter() - ts) * 1e3)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / k, dist)
        eclocks = esampler.stop()
        # the device-to-host copy alone (what the host link adds to the step)
        t1 = time.perf_counter()
        qs.check(qs.lib().qs_copy_out(state.handle, hbuf.ctypes.data_as(ctypes.c_void_p), hbuf.nbytes))
        tc = time.perf_counter() - t1
        line["e2e"] = {"value": world * upd / dt, "unit": "amp-updates/s",
                       "h2d_bytes_per_step": ctypes.sizeof(garr), "d2h_bytes_per_step": hbuf.nbytes,
                       "ms_per_step": dt * 1e3, "steps": k, "step_ms": [round(v, 2) for v in step_ms],
                       "clocks": eclocks,
                       "d2h_copy_ms": tc * 1e3, "d2h_gbs": hbuf.nbytes / tc / 1e9,
                       "host_buffer_pinned": bool(host.is_pinned())}
        del host
        _release(torch)
        # pipelined: the same steps on two states and two streams, each step's
        # copy-out overlapping the next step's passes; the serial figures stay
        # beside it
        try:
            pipe = e2e_pipelined(torch, qs, state, n, args.dtype, garr, len(gates), opts,
                                 max(3, min(args.steps, 4)), dist, local)
        except (RuntimeError, MemoryError) as exc:
            pipe = None
            line["e2e"]["pipelined_unavailable"] = str(exc).splitlines()[0][:200] if str(exc) else type(exc).__name__
        _release(torch)
        if pipe is not None:
            serial = line["e2e"]
            line["e2e"] = {"value": world * upd / (pipe["ms_per_step"] / 1e3), "unit": "amp-updates/s",
                           "h2d_bytes_per_step": serial["h2d_bytes_per_step"],
                           "d2h_bytes_per_step": serial["d2h_bytes_per_step"], **pipe,
                           "serial": {k2: serial[k2] for k2 in ("value", "ms_per_step", "steps", "step_ms", "clocks",
                                                                "d2h_copy_ms", "d2h_gbs", "host_buffer_pinned")}}

    if not args.no_secondary and rank == 0 and n == N_QUBITS:
        step()   # the headline state for the complex64 distance
        line["secondary"] = secondary(args, torch, qs, state if args.dtype == "c128" else None, peaks, sms,
                                      sm_mhz)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        state.close()
        del state
        _release(torch)
        cb = cpu_baseline(args.dtype)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
