"""Throughput benchmark of the random-circuit workload: n = 30 qubits, 40 layers
of Haar-random SU(2) gates on every qubit followed by C-NOTs on 15 random
disjoint pairs (1800 gates), complex64 state (8 GiB) by default.

One step = one simulation of the whole circuit from |0...0>: qs_init_basis
followed by the fused circuit plan (every gate of the circuit).  Prints one
JSON line (see --help).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype c64|c128]
                  [--no-fuse] [--impl ours|reference]

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
    return {
        "workload": "random circuit n=%d, %d layers (Haar SU(2) on every qubit + C-NOTs on %d disjoint pairs), %s state"
                    % (n, LAYERS, n // 2, "complex64" if args.dtype == "c64" else "complex128"),
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


def secondary(args, torch, qs, state64):
    """The other measurements the metric names, each on its own workload:
    the complex128 state at n = 30 (same circuit), the adjoint gradient
    against finite differences at n = 26 (25 layers, 1300 angles), and the
    4096-trajectory noisy batch."""
    out = {}
    n = args.n
    gates = W.random_circuit(n, LAYERS, seed=SEED)
    upd = amp_updates(n, gates)
    # the QFT black box (FFT, Sec. 2.3.2) on the same complex64 register:
    # 4 transform passes and a bit-reversal pass, each one read + one write
    if state64 is not None:
        state64.qft()
        t = _time(torch, lambda: state64.qft(), reps=3)
        nbytes = 5 * 2 * (8 << n)
        out["qft_fft_c64"] = {"workload": "QFT of all %d qubits by the FFT (qs_qft), complex64" % n,
                              "ms": t, "hbm_gbs_5_passes": nbytes / (t / 1e3) / 1e9,
                              "frac_of_measured_hbm": nbytes / (t / 1e3) / 1e9 / measured_peaks()[0]}
    # complex128: one warm-up, one timed step (FP64-ALU bound)
    if state64 is not None:
        state64.close()
    torch.cuda.empty_cache()
    p128 = qs.Plan(n, "c128", gates)
    s128 = qs.State(n, "c128")
    step = lambda: (s128.init_basis(0), p128.execute(s128))
    step()
    p128.set_timing(True)
    p128.timing()
    ms = _time(torch, step)
    kms, kn = p128.timing()
    flops = sum(16 * (1 << n) for g in gates if g.kind == "MATRIX")
    out["c128"] = {"value": upd / (ms / 1e3), "unit": "amp-updates/s", "ms_per_step": ms,
                   "passes": p128.launches,
                   "roofline": {"bound": "alu", "achieved": flops / (kms / 1e3) / 1e12, "peak": 1.25,
                                "unit": "TFLOP/s", "frac": flops / (kms / 1e3) / 1e12 / 1.25,
                                "peak_source": "nominal FP64 1.25 TFLOP/s", "kernel": "k_fused<double,4>"}}
    s128.close()
    del p128
    torch.cuda.empty_cache()
    # adjoint gradient at n = 26 vs finite differences / parameter shift
    na = 26
    agates, aparams = W.ansatz_circuit(na, 25, seed=2026)
    work = qs.State(na, "c64")
    pauli = "Z" + "I" * (na - 1)
    qs.adjoint_grad(work, agates, aparams, pauli=pauli)
    t_adj = _time(torch, lambda: qs.adjoint_grad(work, agates, aparams, pauli=pauli))
    pf = qs.Plan(na, "c64", agates)
    fwd = lambda: (work.init_basis(0), pf.execute(work), work.expect(pauli))
    fwd()
    t_fwd = _time(torch, fwd, reps=3)
    n_par = aparams.size
    out["adjoint"] = {"workload": "ansatz n=26, 25 layers of RY/RZ + C-NOT ladder, 1300 angles, complex64, <Z_0>",
                      "adjoint_ms": t_adj, "forward_ms": t_fwd,
                      "finite_diff_ms_estimate": 2 * n_par * t_fwd,
                      "speedup_vs_finite_diff": 2 * n_par * t_fwd / t_adj,
                      "speedup_vs_parameter_shift": 2 * n_par * t_fwd / t_adj,
                      "note": "finite differences and the parameter-shift rule both take 2 forward passes per "
                              "angle; their cost is 2 x 1300 x the measured forward time"}
    work.close()
    del pf
    torch.cuda.empty_cache()
    # batched noisy trajectories
    batch = W.trajectory_batch(4096, ((12, 2), (16, 1), (20, 1)), (12, 16), seed=31337)
    groups = qs.batch_groups(batch)
    qs.run_trajectories(groups, 1e-3, 1e-2, 7, dtype="c64", with_stats=False)
    t0 = time.perf_counter()
    met, _ = qs.run_trajectories(groups, 1e-3, 1e-2, 7, dtype="c64", with_stats=False)
    dt = time.perf_counter() - t0
    hist, edges = np.histogram(met, bins=10, range=(0.0, 1.0))
    tupd = 0
    for g in groups:
        m = len(g["x0"])
        per = amp_updates(g["n"], g["gates"]) * (2 if g.get("metric", "fidelity") == "fidelity" else 1)
        tupd += m * per
    out["trajectories"] = {"workload": "4096 trajectories, 12/16/20 qubits 2:1:1, QFT + Grover(12,16), "
                                       "sigma=1e-2, p=1e-3, complex64",
                           "seconds": dt, "trajectories_per_s": len(met) / dt,
                           "amp_updates_per_s": tupd / dt,
                           "histogram_0_1_10bins": hist.tolist(), "mean_metric": float(met.mean())}

    # Grover search, n = 24, floor(pi/4 sqrt(2^24)) = 3216 iterations, as one
    # plan; success probability against sin^2((2j+1) theta), sin theta = 2^-12
    gn = 24
    gk = W.basis_index(24, gn)
    git = W.grover_iterations(gn)
    ggates = W.grover_circuit(gn, gk, git)
    want = math.sin((2 * git + 1) * math.asin(2.0 ** (-gn / 2))) ** 2
    gro = {"workload": "Grover n=24, %d iterations (%d gates: 2 H layers and 2 one-amplitude phase flips "
                       "per iteration)" % (git, len(ggates))}
    for dt_name, B in (("c64", 8), ("c128", 16)):
        gs = qs.State(gn, dt_name)
        gp = qs.Plan(gn, dt_name, ggates)
        run = lambda: (gs.init_basis(0), gp.execute(gs))
        run()
        ms = _time(torch, run)
        p_succ = gs.prob(gk)
        gro[dt_name] = {"ms": ms, "gates_per_s": len(ggates) / (ms / 1e3), "passes": gp.launches,
                        "hbm_gbs": gp.launches * 2.0 * (B << gn) / (ms / 1e3) / 1e9,
                        "success_probability": p_succ, "closed_form": want, "error": abs(p_succ - want)}
        gro[dt_name]["frac_of_measured_hbm"] = gro[dt_name]["hbm_gbs"] / measured_peaks()[0]
        gs.close()
        del gp
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
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--no-fuse", action="store_true")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the complex128, adjoint and trajectory measurements")
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

    n = args.n
    gates = W.random_circuit(n, LAYERS, seed=SEED + rank)
    upd = amp_updates(n, gates)
    plan = qs.Plan(n, args.dtype, gates, fuse=not args.no_fuse)
    state = qs.State(n, args.dtype)
    amp_bytes = 8 if args.dtype == "c64" else 16

    def step():
        state.init_basis(0)
        plan.execute(state)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: device events on the launching stream, plus per-launch
    # events recorded by the library around every pass
    plan.set_timing(True)
    plan.timing()
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
    kern_ms, kern_n = 0.0, 0
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    ms, nl = plan.timing()
    kern_ms += ms
    kern_n += nl
    plan.set_timing(False)
    ms_per_step, value = aggregate(ev0.elapsed_time(ev1) / args.steps, upd, world, dist)

    # roofline of the dominant kernel (the fused pass, or the pair sweep),
    # measured on its own launches with per-launch CUDA events
    peak_gbs, peak_src = measured_peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    per_launch_ms = kern_ms / max(1, kern_n)
    launches_per_step = kern_n / args.steps
    if args.no_fuse:
        # algorithmic bytes: one read and one write of every touched amplitude
        bytes_step = sum(2 * amp_bytes * (1 << (n - len(g.controls))) for g in gates)
    else:
        bytes_step = launches_per_step * 2 * (amp_bytes << n)   # one read + one write per pass
    flops_step = sum(16 * (1 << n) for g in gates if g.kind == "MATRIX")   # 8 multiply-adds per amplitude
    kern_s_step = kern_ms / args.steps / 1e3
    hbm_view = {"achieved": bytes_step / kern_s_step / 1e9, "peak": peak_gbs, "unit": "GB/s",
                "frac": bytes_step / kern_s_step / 1e9 / peak_gbs, "peak_source": peak_src}
    if args.dtype == "c64":
        alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12     # FP32 lanes x 2 flops x SM clock
        alu_src = "152 SMs x 128 FP32 lanes x 2 flops x %.0f MHz (measured SM clock)" % sm_mhz
    else:
        alu_peak = 1.25                                   # nominal FP64 rate of the part
        alu_src = "nominal FP64 1.25 TFLOP/s"
    alu_view = {"achieved": flops_step / kern_s_step / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": flops_step / kern_s_step / 1e12 / alu_peak, "peak_source": alu_src}
    t_hbm = bytes_step / (peak_gbs * 1e9)
    t_alu = flops_step / (alu_peak * 1e12)
    main = alu_view if t_alu > t_hbm else hbm_view
    # DRAM traffic of one fused-pass launch from one ncu capture of this
    # kernel at n = 26 (1013.5 MB read + write per launch), scaled to n by the
    # amplitudes processed; only valid for the complex64 fused kernel
    traffic = 1013.5e6 * (1 << (n - 26)) if (args.dtype == "c64" and not args.no_fuse) else None
    roof = {"bound": "alu" if t_alu > t_hbm else "hbm", "achieved": main["achieved"], "peak": main["peak"],
            "unit": main["unit"], "frac": main["frac"], "traffic": traffic, "traffic_unit": "bytes per launch",
            "kernel": ("k_fused_c64" if args.dtype == "c64" else "k_fused<double,4>") if not args.no_fuse else "k_pair",
            "peak_source": main["peak_source"], "launches_timed": kern_n,
            "kernel_ms_per_launch": per_launch_ms, "kernel_ms_per_step": kern_ms / args.steps,
            "hbm_view": hbm_view, "alu_view": alu_view}
    bytes_per_launch = 2 * (amp_bytes << n)

    line = {
        "metric": "amp-updates/s", "value": value, "unit": "amp-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.dtype == "c64" else "f64",
        "data": "synthetic", "config": workload_config(args, world),
        "gates_per_s": world * len(gates) / (ms_per_step / 1e3),
        "hbm_gbs_algorithmic": world * bytes_step / (ms_per_step / 1e3) / 1e9,
        "passes_per_step": plan.launches,
        "roofline": roof,
        "gpu_launches": args.steps * (plan.launches + 1),
        "clocks": clocks,
    }

    # end to end through the public API with host buffers: the gate list goes
    # in from host memory (qs_apply_circuit copies, plans and launches), the
    # final state comes back to pinned host memory (qs_copy_out)
    if not args.no_e2e:
        host = torch.empty(1 << n, dtype=torch.complex64 if args.dtype == "c64" else torch.complex128,
                           pin_memory=True)
        hbuf = host.numpy()
        import ctypes
        garr = qs.gates_to_abi(gates)
        opts = qs._opts(not args.no_fuse)

        def e2e_step():
            qs.check(qs.lib().qs_init_basis(state.handle, 0))
            qs.check(qs.lib().qs_apply_circuit(state.handle, garr, len(gates), ctypes.byref(opts)))
            qs.check(qs.lib().qs_copy_out(state.handle, hbuf.ctypes.data_as(ctypes.c_void_p), hbuf.nbytes))

        e2e_step()
        if dist:
            dist.barrier()
        k = max(1, min(args.steps, 5))
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
        # pipelined: the same steps on two states and two streams, each step's
        # copy-out overlapping the next step's passes; the serial figures stay
        # beside it
        try:
            pipe = e2e_pipelined(torch, qs, state, n, args.dtype, garr, len(gates), opts,
                                 max(4, min(args.steps, 6)), dist, local)
        except (RuntimeError, MemoryError) as exc:
            pipe = None
            line["e2e"]["pipelined_unavailable"] = str(exc).splitlines()[0][:200] if str(exc) else type(exc).__name__
        # hand the pinned host buffers back to the system (torch caches them)
        release = getattr(torch._C, "_host_emptyCache", None)
        if release is not None:
            release()
        if pipe is not None:
            serial = line["e2e"]
            line["e2e"] = {"value": world * upd / (pipe["ms_per_step"] / 1e3), "unit": "amp-updates/s",
                           "h2d_bytes_per_step": serial["h2d_bytes_per_step"],
                           "d2h_bytes_per_step": serial["d2h_bytes_per_step"], **pipe,
                           "serial": {k2: serial[k2] for k2 in ("value", "ms_per_step", "steps", "step_ms", "clocks",
                                                                "d2h_copy_ms", "d2h_gbs", "host_buffer_pinned")}}

    if not args.no_secondary and rank == 0:
        line["secondary"] = secondary(args, torch, qs, state if args.dtype == "c64" else None)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        del state
        torch.cuda.empty_cache()
        cb = cpu_baseline(args.dtype)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
