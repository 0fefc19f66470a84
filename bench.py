"""Circuit-time benchmark on one GB300 (or N replicas under torchrun).

One step = one full execution of a kernelized circuit on a 2^n complex64
state already resident in HBM (all kernels of the plan, back to back on one
stream).  The workload is the mixed-gate circuit generator at 30 qubits:
5000 gates drawn uniformly from {H, X, RX, RZ, CX, CZ, CP, SWAP}, partner
distance 1 + Geom(0.3), seed 100 -- an 8 GiB state, larger than L2, so no
L2 flush is needed between steps.

Prints one JSON line (rank 0).  `value` is milliseconds per circuit over the
whole job (max-over-ranks elapsed time / circuits executed by all ranks).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "circuit time and HBM-roofline fraction at 30 qubits, FP32 vs fused 3xTF32+learned plan"
N_QUBITS = 30
N_GATES = 5000
SEED = 100
# DRAM bytes per launch of the specialised shared-memory kernel as a fraction
# of its algorithmic bytes, from an ncu capture of that kernel form at 28
# qubits (kernel 10 of plan A, deferred factors: 2.148 GB read + 2.086 GB
# written for 4.295 GB of one pass; its generated code is the same under the
# 32-B-sector store rule, which changes 13 of the 151 kernels at 30 qubits
# and writes the same bytes; None: not measured for the current form)
QSK_TRAFFIC_RATIO = 0.986
WORKLOAD = (f"mixed circuit, {N_QUBITS} qubits, {N_GATES} gates from {{H,X,RX,RZ,CX,CZ,CP,SWAP}}, "
            f"partner distance 1+Geom(0.3), seed {SEED}; complex64 state 8 GiB")


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    replica's); x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def mem_available_gib():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) / (1 << 20)
    except Exception:
        pass
    return 0.0


def oracle_sample(gates, budget_s, n_full=N_QUBITS):
    """Times the FP64 oracle, gate by gate, on a bounded prefix of the
    circuit.  Runs at n_full qubits when host memory allows (16 GiB complex128
    at 30 qubits), else at 28 qubits scaled by the state-size ratio.
    Returns (ms per circuit estimate, sample description, threads)."""
    import numpy as np
    from oracle import sim
    n = n_full
    if mem_available_gib() < (16 << (n - 30)) * 1.0 + 8:
        n = 28
    scale = 2.0 ** (n_full - n)
    sub = gates.copy()
    ok = (sub["q0"] < n) & ((sub["q1"] < n))
    sub = sub[ok]
    psi = sim.zero_state(n)
    done, t0 = 0, time.perf_counter()
    el = 0.0
    while done < len(sub) and el < budget_s:
        psi = _apply_inplace(sim, n, sub[done:done + 1], psi)
        done += 1
        el = time.perf_counter() - t0
    per_gate_ms = el * 1e3 / max(done, 1) * scale
    desc = (f"first {done} gates of the circuit on a {n}-qubit complex128 state"
            + (f", scaled x{scale:.0f} to {n_full} qubits" if scale != 1 else "")
            + f"; per-gate time x {len(gates)} gates")
    del psi
    return per_gate_ms * len(gates), desc, sim.threads()


def _apply_inplace(sim, n, g, psi):
    import ctypes
    import numpy as np
    from synth.circuits import GATE_DTYPE
    gg = np.ascontiguousarray(g, dtype=GATE_DTYPE)
    f = psi.view(np.float64)
    rc = sim.lib().or_apply_circuit(n, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    gg.ctypes.data_as(ctypes.c_void_p), len(gg))
    if rc != 0:
        raise RuntimeError("oracle rejected a gate")
    return psi


def reference_arm(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    from synth import circuits as C
    gates = C.mixed_circuit(N_QUBITS, N_GATES, SEED)
    step_budget = 4.0
    for _ in range(args.warmup):
        oracle_sample(gates, 0.5)
    vals, desc, thr = [], "", 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc, thr = oracle_sample(gates, step_budget)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms/circuit",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall * 1e3 / max(args.steps, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_qubits": N_QUBITS, "gates": N_GATES,
                   "plan": "none (FP64 oracle applies gates one at a time)"},
        "cpu_baseline": {"value": value, "unit": "ms/circuit", "cores": thr, "kind": "oracle",
                         "sample": desc + f"; {step_budget:.0f} s per step"},
        "e2e": {"value": value, "unit": "ms/circuit", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def make_plan(Q, gates, which, shm_max=13, algo=None, n=N_QUBITS, forced_low=4, insular_x=0):
    if which.startswith("F-"):  # every kernel fused (k = 6), in the given precision
        prec = {"F-FP32": Q.QS_PREC_FP32, "F-TF32": Q.QS_PREC_TF32, "F-TF32X3": Q.QS_PREC_TF32X3}[which]
        cost = Q.default_cost_table()
        for k in range(16):
            cost.fuse_cost[k] = 1.0
        opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=prec, fuse_kmax=6, fuse_kmin=6,
                              cost=cost, insular_x=insular_x)
        return Q.Plan(n, gates, opts), f"{which}: Kernelize, every kernel a fused 2^6 unitary"
    if which == "B":  # learned-cost Kernelize, fused kernels on tensor cores in 3xTF32
        from paper_2408_09055_gb300 import costmodel as CM
        net, _ = CM.load()
        opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=Q.QS_PREC_TF32X3,
                              shm_max_active=shm_max, fuse_kmax=6, mlp=net, forced_low=forced_low,
                              insular_x=insular_x)
        if algo == "ordered":
            opts.algo = Q.QS_ALGO_ORDERED
        plan = Q.Plan(n, gates, opts)
        plan._net = net  # the model must outlive planning only, kept for reference
        return plan, ("B: learned-cost Kernelize (MLP trained on this GPU's kernel timings), "
                      "shared-memory kernels + fused 3xTF32 tensor-core kernels")
    if which == "A" and algo == "ordered":
        opts = Q.default_opts(algo=Q.QS_ALGO_ORDERED, cost_kind=Q.QS_COST_ANALYTIC,
                              precision=Q.QS_PREC_FP32, shm_max_active=shm_max, fuse_kmax=0,
                              forced_low=forced_low, insular_x=insular_x)
        label = "A': analytic-cost OrderedKernelize, shared-memory kernels, FP32"
    elif which == "A":
        opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, cost_kind=Q.QS_COST_ANALYTIC,
                              precision=Q.QS_PREC_FP32, shm_max_active=shm_max, fuse_kmax=0,
                              forced_low=forced_low, insular_x=insular_x)
        label = "A: analytic-cost Kernelize, shared-memory kernels, FP32"
    else:
        raise ValueError(which)
    return Q.Plan(n, gates, opts), label


def workload_gates(name, n=N_QUBITS):
    from synth import circuits as C
    if name == "mixed":
        return C.mixed_circuit(n, N_GATES, SEED)
    if name == "entangling":
        return C.entangling_circuit(n, 40, SEED)
    raise ValueError(name)


def entangling_desc(n):
    return (f"entangling circuit, {n} qubits, 40 layers (U3 on every qubit, CP+RXX on a random "
            f"matching, angles U[0,2pi)), seed {SEED}; complex64 state {8 << n >> 30} GiB")


def profile_run(args):
    """One untimed execution of the workload's plan at a smaller size."""
    import torch
    from paper_2408_09055_gb300 import qsim as Q
    from synth import circuits as C
    n = args.profile_run
    if args.plan.startswith("F-"):
        gates = C.entangling_circuit(n, 8, SEED) if args.workload == "entangling" else C.mixed_circuit(n, N_GATES, SEED)
        prec = {"F-FP32": Q.QS_PREC_FP32, "F-TF32": Q.QS_PREC_TF32, "F-TF32X3": Q.QS_PREC_TF32X3}[args.plan]
        cost = Q.default_cost_table()
        for k in range(16):
            cost.fuse_cost[k] = 1.0
        opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=prec, fuse_kmax=6, fuse_kmin=6, cost=cost,
                              insular_x=1 if args.insular_x else 0)
    else:
        gates = (C.entangling_circuit(n, 40, SEED) if args.workload == "entangling"
                 else C.mixed_circuit(n, N_GATES, SEED))
        opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=args.shm_max,
                              insular_x=1 if args.insular_x else 0)
        if args.algo == "ordered":
            opts.algo = Q.QS_ALGO_ORDERED
    plan = Q.Plan(n, gates, opts)
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    s = torch.cuda.current_stream().cuda_stream
    st.set_zero(s)
    st.run(plan, s)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": n, "kernels": int(plan.stats().num_kernels), "norm2": st.norm2(s)}))
    return 0


def config2_measure(args):
    """The dense entangling circuit (40 layers: U3 on every qubit, CP + RXX on
    a random matching, seed 100) on a resident n-qubit state with every
    kernel fused into a dense 2^k unitary, k = 5, 6, 7 forced in turn, in
    FP32 on CUDA cores, TF32 and 3xTF32 on the tensor cores (k = 5 widened
    to the tensor-core kernel's 6 targets; no tensor-core form for k = 7),
    beside plan A.  Per form: ms per circuit, kernels, average launch time
    and its HBM fraction; error against the FP64 oracle of the same
    generator at `err_n` qubits (rank 0)."""
    import numpy as np
    import torch
    from paper_2408_09055_gb300 import qsim as Q
    from oracle import sim
    n, err_n = args.config2, 26
    hbm, _, src = peaks()
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    eg = workload_gates("entangling", n)
    small = workload_gates("entangling", err_n)
    ref = sim.apply(err_n, small)
    ebuf = torch.empty(2 << err_n, dtype=torch.float32, device="cuda")
    est = Q.State(err_n, ebuf.data_ptr())
    names = {Q.QS_PREC_FP32: "FP32 CUDA cores", Q.QS_PREC_TF32: "TF32", Q.QS_PREC_TF32X3: "3xTF32"}

    def fused_opts(k, prec):
        cost = Q.default_cost_table()
        for j in range(16):
            cost.fuse_cost[j] = 1.0
        return Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=prec, fuse_kmax=k, fuse_kmin=k, cost=cost)

    rows = []
    forms = [("A", None, None)] + [(f"F{k}", k, p) for k in (5, 6, 7)
                                   for p in (Q.QS_PREC_FP32, Q.QS_PREC_TF32, Q.QS_PREC_TF32X3)]
    for label, k, prec in forms:
        row = {"form": label if k is None else f"fused k={k}, {names[prec]}"}
        try:
            if k is None:
                opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=args.shm_max)
            else:
                opts = fused_opts(k, prec)
            plan = Q.Plan(n, eg, opts)
        except Q.QsError as e:
            row["unsupported"] = str(e)
            rows.append(row)
            continue
        ps = plan.stats()
        st.set_zero(sp)
        ms, pk, runs = time_plan(Q, torch, st, plan, args.steps, args.warmup, stream, 1)
        types = by_kernel_type(Q, plan, pk, runs, n, hbm)
        row.update({"ms_per_circuit": ms / args.steps, "kernels": int(ps.num_kernels),
                    "fused_kernels": int(ps.num_fused), "kernel_types": types,
                    "norm2_after": st.norm2(sp)})
        eplan = Q.Plan(err_n, small, opts)
        est.set_zero(sp)
        est.run(eplan, sp)
        got = est.read(stream=sp).astype(np.complex128)
        fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
        row["error_vs_fp64"] = {"n_qubits": err_n, "one_minus_fidelity": float(1 - fid),
                                "max_abs": float(np.max(np.abs(ref - got)))}
        rows.append(row)
        del plan, eplan
    line = {"metric": "entangling circuit, every kernel fused (config 2)", "n_qubits": n,
            "workload": entangling_desc(n), "gates": int(len(eg)), "steps": args.steps, "warmup": args.warmup,
            "unit": "ms/circuit", "peak_hbm_gbs": hbm, "peak_source": src, "forms": rows}
    print(json.dumps(line), flush=True)
    return 0


def _copy_peaks(torch, host, dev, nbytes, reps=3):
    """Page-locked host <-> HBM copy bandwidth (GB/s): each direction alone,
    and both at once on two streams (their sum) -- the staged loop's bound."""
    h = host.view(torch.uint8)[:nbytes]
    d = dev.view(torch.uint8)[:nbytes]
    d2 = dev.view(torch.uint8)[nbytes:2 * nbytes]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}
    for name in ("h2d", "d2h", "both"):
        best = 0.0
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name in ("h2d", "both"):
                with torch.cuda.stream(s1):
                    d.copy_(h, non_blocking=True)
            if name in ("d2h", "both"):
                with torch.cuda.stream(s2):
                    h.copy_(d2, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = max(best, (2 if name == "both" else 1) * nbytes / dt / 1e9)
        out[name] = best
    return out


def remap_measure(args):
    """qs_remap (Alg. 1's Shard permutation) on an n-qubit resident state:
    one HBM pass per call (every amplitude read and written once); CUDA
    events over `steps` calls after `warmup`, for several bit permutations."""
    import numpy as np
    import torch
    from paper_2408_09055_gb300 import qsim as Q
    n = args.remap
    src = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    s = torch.cuda.current_stream()
    rng = np.random.default_rng(0)
    perms = {"identity": np.arange(n), "reverse": np.arange(n)[::-1], "random": rng.permutation(n),
             "low 5 <-> high 5": np.r_[np.arange(n - 5, n), np.arange(5, n - 5), np.arange(0, 5)]}
    hbm, _, src_kind = peaks()
    out = {}
    for name, perm in perms.items():
        for _ in range(args.warmup):
            Q.qs_remap(src.data_ptr(), dst.data_ptr(), n, perm, s.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            Q.qs_remap(src.data_ptr(), dst.data_ptr(), n, perm, s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        gbs = 16.0 * (1 << n) / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "GB/s": gbs, "frac": gbs / hbm}
    print(json.dumps({"metric": "qubit remap (bit permutation) bandwidth", "n_qubits": n,
                      "peak_gbs": hbm, "peak_source": src_kind, "steps": args.steps, "permutations": out}))
    return 0


def staged_measure(args):
    """Staged execution (Alg. 1's Execute over host memory): a layered
    U3 + CZ circuit (30 layers, seed 0) on an n-qubit state in page-locked
    host memory, run chunk by chunk through qs_run_plan_host with L local
    qubits.  Prints one JSON line: ms per circuit and the achieved host<->GPU
    bandwidth against the measured copy peak of both directions at once."""
    import numpy as np
    import torch
    from paper_2408_09055_gb300 import qsim as Q
    from synth import circuits as C
    n, L = args.staged, args.local_qubits or args.staged - 3
    need_gib = (8 << n) / 2 ** 30
    if mem_available_gib() < need_gib + 16:
        print(json.dumps({"staged": n, "unavailable": f"host memory: {mem_available_gib():.0f} GiB available, "
                                                      f"{need_gib:.0f} GiB state needed"}))
        return 0
    # the page-locked state first, before planning (as the resident bench's
    # end-to-end buffers)
    host = torch.empty(2 << n, dtype=torch.float32, pin_memory=True)
    gates = C.layered_u3_cz(n, 30, 0)
    opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=args.shm_max,
                          local_qubits=L)
    t0 = time.perf_counter()
    plan = Q.Plan(n, gates, opts)
    plan_s = time.perf_counter() - t0
    ps = plan.stats()
    nbuf = args.chunk_buffers
    dev = torch.empty(max(nbuf, 2) << (L + 1), dtype=torch.float32, device="cuda")
    chunk = 8 << L
    peaks_c = _copy_peaks(torch, host, dev, min(chunk, 4 << 30))  # before the state is set
    host.zero_()
    host[0] = 1.0
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    for _ in range(args.warmup):
        plan.run_host(host.data_ptr(), dev.data_ptr(), nbuf * (8 << L), stream=sp)
    torch.cuda.synchronize()
    clocks = ClockSampler(_env_int("LOCAL_RANK", 0))
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run_host(host.data_ptr(), dev.data_ptr(), nbuf * (8 << L), stream=sp)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # one more run with the per-chunk timeline: where the time goes
    tm = Q.HostTimer(plan)
    tm.run(host.data_ptr(), dev.data_ptr(), nbuf * (8 << L), stream=sp)
    torch.cuda.synchronize()
    T = tm.read()
    breakdown = {"timeline_ms": float(T[:, :, 3].max()),
                 "copy_in_ms": float((T[:, :, 1] - T[:, :, 0]).sum()),
                 "kernels_ms": float((T[:, :, 2] - T[:, :, 1]).sum()),
                 "copy_out_ms": float((T[:, :, 3] - T[:, :, 2]).sum())}
    v = host.numpy().view(np.complex64)
    norm = 0.0
    for a in range(0, v.size, 1 << 26):
        x = v[a:a + (1 << 26)].astype(np.complex128)
        norm += float(np.vdot(x, x).real)
    moved = 2.0 * ps.num_stages * (8 << n)
    achieved = moved / (ms * 1e-3) / 1e9
    line = {
        "metric": "staged circuit time (state in host memory)", "value": ms, "unit": "ms/circuit",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"layered circuit, {n} qubits, 30 layers (U3 on every qubit, CZ on a random "
                               f"perfect matching), seed 0; complex64 state {8 << n >> 30} GiB in page-locked "
                               f"host memory",
                   "n_qubits": n, "local_qubits": L, "gates": int(len(gates)), "stages": int(ps.num_stages),
                   "kernels": int(ps.num_kernels), "chunk_buffers": nbuf, "planner_s": plan_s,
                   "stager": "beam", "staging_objective": int(ps.staging_cost),
                   "plan": "analytic-cost Kernelize per stage, shared-memory kernels, FP32"},
        "roofline": {"bound": "c2c", "achieved": achieved, "peak": peaks_c["both"], "unit": "GB/s",
                     "frac": achieved / peaks_c["both"], "traffic": moved,
                     "peak_source": "measured here: concurrent H2D + D2H copies of one chunk"},
        "copy_peaks_gbs": peaks_c,
        "breakdown": breakdown,
        "gpu_launches": int(ps.num_kernels) * (1 << (n - L)) * args.steps,
        "clocks": clk, "norm2_after": norm,
        "e2e": {"value": ms, "unit": "ms/circuit", "h2d_bytes_per_step": int(ps.num_stages * (8 << n)),
                "d2h_bytes_per_step": int(ps.num_stages * (8 << n))},
    }
    print(json.dumps(line), flush=True)
    return 0


def kernel_type_name(Q, plan, d):
    ps = plan.stats()
    if d.type == Q.QS_KERNEL_SHM:
        return ("qsk<i> (plan-specialised shared-memory kernel)" if ps.num_jit else
                "shm_kernel_v2" if ps.num_phased else "shm_kernel_v1")
    return "fused_fp32_kernel" if plan.opts.precision == Q.QS_PREC_FP32 else "fused_tc_kernel"


def by_kernel_type(Q, plan, per_kernel_ms, runs, n, hbm):
    """Per kernel type: launches, total and average launch time (CUDA events
    on the launching stream) and the HBM roofline fraction of one pass
    (16 * 2^n bytes per launch) over the measured peak."""
    out = {}
    for k in range(plan.stats().num_kernels):
        nm = kernel_type_name(Q, plan, plan.kernel(k))
        t = out.setdefault(nm, {"launches": 0, "total_ms": 0.0})
        t["launches"] += runs
        t["total_ms"] += per_kernel_ms[k]
    for t in out.values():
        t["avg_launch_ms"] = t["total_ms"] / max(t["launches"], 1)
        t["hbm_frac"] = 16.0 * (1 << n) / (t["avg_launch_ms"] * 1e-3) / 1e9 / hbm
    return out


def time_plan(Q, torch, st, plan, steps, warmup, stream, world):
    """Warm-up runs, then `steps` timed runs of the plan on the resident
    state, bracketed by synchronisation (and a barrier over ranks).  Returns
    (max-over-ranks elapsed ms, per-kernel ms summed over runs, runs)."""
    import torch.distributed as dist
    sp = stream.cuda_stream
    for _ in range(warmup):
        st.run(plan, sp)
    torch.cuda.synchronize()
    timer = Q.Timer(plan, steps)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st.run_timed(plan, timer, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    per_kernel_ms, runs = timer.read()
    return elapsed, per_kernel_ms, runs


def error_vs_fp64(Q, torch, shm_max, n=26):
    """Each workload's plans A and B at n qubits against the FP64 oracle
    (the same generators and seeds as the timed 30-qubit runs): fidelity
    |<ref|psi>|^2 / (<ref|ref><psi|psi>) and max-abs error over every
    amplitude, in FP64 on the host."""
    import numpy as np
    from oracle import sim
    out = {"n_qubits": n, "reference": "FP64 (complex128) oracle, gate by gate"}
    s = torch.cuda.current_stream().cuda_stream
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    for wl in ("mixed", "entangling"):
        g = workload_gates(wl, n)
        t0 = time.perf_counter()
        ref = sim.apply(n, g)
        res = {"gates": int(len(g)), "oracle_s": time.perf_counter() - t0}
        for which in ("A", "B"):
            plan, _ = make_plan(Q, g, which, shm_max, None, n)
            st.set_zero(s)
            st.run(plan, s)
            got = st.read(stream=s).astype(np.complex128)
            fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
            res[which] = {"fidelity": float(fid), "one_minus_fidelity": float(1.0 - fid),
                          "max_abs": float(np.max(np.abs(ref - got))),
                          "fused_kernels": int(plan.stats().num_fused)}
            del got
        out[wl] = res
        del ref
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plan", default="A")
    ap.add_argument("--algo", default=None, choices=[None, "ordered", "kernelize"],
                    help="override the plan's kernelization algorithm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="with --plan A, skip timing plan B beside it")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-entangling", action="store_true",
                    help="with the default mixed workload, skip timing the entangling circuit's plans")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the 26-qubit error-against-FP64 leg (rank 0, beside the CPU baseline)")
    ap.add_argument("--shm-max", type=int, default=12)
    ap.add_argument("--insular-x", action="store_true",
                    help="plan the Pauli-frame rewrite that makes X insular (App. A.2)")
    ap.add_argument("--forced-low", type=int, default=4,
                    help="lowest qubits forced into every shared-memory kernel (2^f * 8-byte runs)")
    ap.add_argument("--workload", default="mixed", choices=["mixed", "entangling"])
    ap.add_argument("--profile-run", type=int, default=0, metavar="N",
                    help="plan the workload's circuit generator at N qubits and run the plan "
                         "once, untimed (a small case for profiler captures); with --plan F-*, "
                         "an 8-layer circuit with every kernel fused")
    ap.add_argument("--staged", type=int, default=0, metavar="N",
                    help="measure staged execution instead: an N-qubit state in page-locked host "
                         "memory, run chunk by chunk with --local-qubits L")
    ap.add_argument("--local-qubits", type=int, default=0)
    ap.add_argument("--remap", type=int, default=0, metavar="N",
                    help="measure the qubit-remap kernel on an N-qubit state instead")
    ap.add_argument("--chunk-buffers", type=int, default=4, choices=[1, 2, 3, 4])
    ap.add_argument("--config2", type=int, default=0, metavar="N",
                    help="the entangling circuit on a resident N-qubit state with every kernel fused "
                         "(k = 5, 6, 7; FP32 / TF32 / 3xTF32) beside plan A, errors against FP64 at 26 qubits")
    args = ap.parse_args()
    if args.config2:
        return config2_measure(args)
    if args.remap:
        return remap_measure(args)
    if args.staged:
        return staged_measure(args)
    if args.profile_run:
        return profile_run(args)
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local)) \
            if "device_id" in dist.init_process_group.__code__.co_varnames else dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2408_09055_gb300 import qsim as Q
    from synth import circuits as C

    n = N_QUBITS
    # the end-to-end leg's page-locked host buffers, allocated before anything
    # else: measured on the box, buffers pinned at process start move 8 GiB
    # at 210 / 193 GB/s (H2D / D2H), buffers pinned after planning as slowly
    # as 30-80 / 19-38 GB/s
    host_in = torch.zeros(2 << n, dtype=torch.float32).pin_memory()
    host_in[0] = 1.0
    host_out = torch.zeros(2 << n, dtype=torch.float32).pin_memory()
    gates = workload_gates(args.workload)
    # measured at 30 qubits: the Pauli-frame rewrite cuts the mixed circuit
    # from 151 to 142 kernels but turns free X renames into extra RZ factors
    # (28.9 -> 35.1 computing gates per kernel): 538.6 against 507 ms
    ix = 1 if args.insular_x else 0
    plan, label = make_plan(Q, gates, args.plan, args.shm_max, args.algo, forced_low=args.forced_low,
                            insular_x=ix)
    ps = plan.stats()
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    st.set_zero(sp)
    hbm, _, src = peaks()
    pass_bytes = 16.0 * (1 << n)
    clocks = ClockSampler(local)
    clocks.start()
    elapsed_ms, per_kernel_ms, runs = time_plan(Q, torch, st, plan, args.steps, args.warmup, stream, world)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    norm = st.norm2(sp)

    # roofline of the dominant kernel type (algorithmic bytes = one read and
    # one write of the state per launch)
    types = by_kernel_type(Q, plan, per_kernel_ms, runs, n, hbm)
    dom = max(types, key=lambda x: types[x]["total_ms"])
    avg_ms = types[dom]["avg_launch_ms"]
    achieved = pass_bytes / (avg_ms * 1e-3) / 1e9
    # DRAM bytes per launch measured by ncu on the same specialised kernel
    # form at 28 qubits (a 2 GiB state), as a fraction of its algorithmic
    # bytes; DRAM traffic grows with the state, so the fraction carries over
    traffic = QSK_TRAFFIC_RATIO * pass_bytes if (dom.startswith("qsk") and QSK_TRAFFIC_RATIO) else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read+write of the same kernel form at 28 qubits, "
                               "as a fraction of its algorithmic bytes" if traffic else None),
            "peak_source": src,
            "launches_timed": types[dom]["launches"], "avg_launch_ms": avg_ms,
            "share_of_step": types[dom]["total_ms"] / max(sum(v["total_ms"] for v in types.values()), 1e-12)}

    # end to end through the public API: H2D of the input state from pinned
    # memory, the circuit, D2H of the output state
    hin = host_in.numpy().view(np.complex64)
    hout = host_out.numpy().view(np.complex64)
    e2e_steps = max(1, min(args.steps, 3))
    st.write(hin, stream=sp)
    st.run(plan, sp)
    st.read(out=hout, stream=sp)
    if world > 1:
        dist.barrier()
    # events between the legs (the amplitude copies synchronise the stream):
    # where the end-to-end time goes
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(e2e_steps)]
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        ev[i][0].record(stream)
        st.write(hin, stream=sp)
        ev[i][1].record(stream)
        st.run(plan, sp)
        ev[i][2].record(stream)
        st.read(out=hout, stream=sp)
        ev[i][3].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world, "cuda")
    legs = [sum(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(e2e_steps)) / e2e_steps for j in range(3)]
    e2e_norm = float(np.sum(np.abs(hout.astype(np.complex128)) ** 2))
    del host_in, host_out, hin, hout

    value = elapsed_ms / (args.steps * world)
    launches = sum(v["launches"] for v in types.values())
    line = {
        "metric": METRIC, "value": value, "unit": "ms/circuit", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "mixed" else entangling_desc(n),
                   "n_qubits": n, "gates": int(len(gates)), "plan": label,
                   "kernels": int(ps.num_kernels), "shm_kernels": int(ps.num_shm),
                   "fused_kernels": int(ps.num_fused), "passes": int(ps.num_kernels),
                   "planner_ms": ps.planner_ms, "jit_ms": ps.jit_ms, "shm_max_active": args.shm_max,
                   "forced_low": args.forced_low,
                   "insular_x": "Pauli-frame rewrite (every X moved to the end, App. A.2)" if ix else "off",
                   "model_cost_ms": ps.cost / 1e3, "l2": "no flush: the 8 GiB state exceeds L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gates_per_s": len(gates) / (value * 1e-3),
        "hbm_roofline_frac_circuit": ps.num_kernels * pass_bytes / (value * 1e-3) / 1e9 / hbm,
        "roofline": roof,
        "kernel_types": types,
        "gpu_launches": int(launches),
        "clocks": clk,
        "norm2_after": norm,
        "e2e": {"value": e2e_ms / (e2e_steps * world) if world == 1 else e2e_ms / e2e_steps / world,
                "unit": "ms/circuit", "steps": e2e_steps,
                "h2d_bytes_per_step": int(8 << n), "d2h_bytes_per_step": int(8 << n),
                "breakdown_ms": {"h2d": legs[0], "circuit": legs[1], "d2h": legs[2]},
                "norm2_out": e2e_norm},
    }

    def arm(g, which, ref_ms=None):
        """One more plan timed the same way on the same state."""
        p, lab = make_plan(Q, g, which, args.shm_max, args.algo, forced_low=args.forced_low, insular_x=ix)
        s_ = p.stats()
        st.set_zero(sp)
        ms, pk, r = time_plan(Q, torch, st, p, args.steps, args.warmup, stream, world)
        v = ms / (args.steps * world)
        out = {"plan": lab, "value": v, "unit": "ms/circuit",
               "dtype": ("f32 shared-memory kernels, tf32x3 fused kernels"
                         if p.opts.precision == Q.QS_PREC_TF32X3 else "f32"),
               "kernels": int(s_.num_kernels), "shm_kernels": int(s_.num_shm),
               "fused_kernels": int(s_.num_fused), "model_cost_ms": s_.cost / 1e3,
               "planner_ms": s_.planner_ms, "jit_ms": s_.jit_ms,
               "kernel_types": by_kernel_type(Q, p, pk, r, n, hbm),
               "norm2_after": st.norm2(sp)}
        if ref_ms is not None:
            out["speedup_over_plan_a"] = ref_ms / v
        return out, r * s_.num_kernels  # launches in its timed region

    if args.plan == "A" and not args.no_compare:
        # the metric's second arm: the learned-cost plan with fused 3xTF32
        # kernels, timed the same way on the same state
        line["plan_b"], _ = arm(gates, "B", value)
        if args.workload == "mixed" and not args.no_entangling:
            # the dense entangling circuit (every layer U3 on every qubit and
            # CP + RXX on a matching), where fused tensor-core kernels pay
            eg = workload_gates("entangling")
            ent = {"workload": entangling_desc(n), "gates": int(len(eg))}
            ent["A"], _ = arm(eg, "A")
            ent["B"], _ = arm(eg, "B", ent["A"]["value"])
            line["entangling"] = ent
    if plan.opts.precision != Q.QS_PREC_FP32:
        line["dtype"] = {Q.QS_PREC_TF32: "tf32", Q.QS_PREC_TF32X3: "tf32x3"}[plan.opts.precision]
    del st, buf
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, thr = oracle_sample(gates, args.cpu_budget)
        line["cpu_baseline"] = {"value": v, "unit": "ms/circuit", "cores": thr, "kind": "oracle",
                                "sample": desc}
        if not args.no_error:
            # error against FP64 of every timed plan, on the same generators
            # at 26 qubits (the oracle cannot run 30 qubits in bench time)
            line["error_vs_fp64"] = error_vs_fp64(Q, torch, args.shm_max)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
