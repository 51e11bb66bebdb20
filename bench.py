"""Benchmark: one 30-qubit random grid circuit per step on the GB300 fused-gate path.

A step is one pass of the hot path over one circuit: set |0...0> and apply every fused gate
(sv_init_apply: the first gates, while they name at most 28 qubits, run on the small state of
those qubits, which is then written into the full state; the fusion places the gates of the
circuit's 28-qubit light cone first for it (--start-qubits); --start plain uses sv_init then
sv_apply_fused_gates on the circuit fused as one, and the line reports the other start's time
too), then one read pass that
yields the fp64 norm and 1024 samples (sv_sample_norm).  The circuit is the 5x6-grid random circuit (20 cycles of
sqrt(X)/sqrt(Y)/sqrt(W) plus fSim(pi/2, pi/6) on patterns ABCDCDAB, seed 2, 845 gates), fused
on the host to at most --max-k qubits; fused gates of --tc-min-k or more qubits run on the tensor
cores in --precision mode.  The complex64 state (8 GiB) is larger than L2, so no flush is needed
between steps.  The same line reports the plain path for comparison: fp32 CUDA-core kernels with
fixed greedy fusion at every max size 2..6.

Prints one JSON line (rank 0).  `value` is seconds per circuit for the whole job (time of the
slowest rank / circuits run by all ranks); `e2e` is the same metric measured through the C ABI
with host buffers (fusion on the host, sample uniforms uploaded, samples and norm read back).
`--impl reference` times the complex128 CPU oracle on a bounded sample of the same circuit.
Outside the timed step the line also reports Pauli expectation passes on the circuit's state
(`expval_pauli`), the rows beyond the hot path (`next_rows`: the controlled-gate kernel,
Grover and quantum-volume circuits, and the circuit on a complex128 state), the step's accuracy
against that complex128 state (`accuracy`: fidelity and l2 distance), and the larger workloads
(`large_configs`: the 33-qubit grid and 34-qubit QFT, learned partition vs fixed greedy fusion at
every max size, and the 256-circuit HEA batch in one persistent launch vs the per-circuit loop).
`dtype` names the arithmetic: complex64 state, 3xBF16 (or TF32) tensor-core products with fp32
accumulation for fused gates of --tc-min-k or more qubits.
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
sys.path.insert(0, ROOT)

METRIC = "circuit s & HBM GB/s (% peak), learned+TC vs plain fusion, fid≥1-1e-6, 30–34q"
UNIT = "s/circuit"
N_QUBITS = 30
N_SAMPLES = 1024
WORKLOAD = "grid30: 5x6 grid random circuit, 20 cycles, 845 gates, seed 2, |0..0>, complex64"
DTYPES = {"bf16x3": "c64 (3xbf16 products, fp32 accumulate)", "tf32": "c64 (tf32 products, fp32 accumulate)",
          "fp32": "c64 (fp32)"}
FP64_PEAK_TFLOPS = 1.20   # fp64 FMA throughput measured on this GPU (independent FMA chains, all SMs)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_traffic(kernel_key: str):
    """bytes per launch from the committed ncu summary (profiles/roofline_traffic.txt), else None."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    try:
        for line in open(path):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fields = dict(kv.split("=", 1) for kv in line.split())
            if fields.get("kernel") == kernel_key and fields.get("current") == "yes":
                return float(fields["bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region (reads only)."""

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def kernel_class(B, info):
    """Kernel path of a fused gate, with the tensor-core gates that stage through shared memory
    (three or more targets below qubit 5) as their own class: they run a different kernel."""
    name = B.PATH_NAMES[info["path"]]
    if info["path"] in (B.PATH_TC_BF16X3, B.PATH_TC_TF32) and sum(1 for t in info["targets"] if t < 5) >= 3:
        name += "_staged"
    return name


def device_state_metrics(ref_buf, buf, chunk_blocks=1 << 21):
    """Fidelity and l2 distance (fp64, on the device) between two states in the blocked layout:
    blocks of 32 real then 32 imaginary parts, fp32 or fp64 (complex64 or complex128 states)."""
    import torch
    a_all, b_all = ref_buf.view(-1, 2, 32), buf.view(-1, 2, 32)
    ov = torch.zeros((), dtype=torch.complex128, device=ref_buf.device)
    d2 = torch.zeros((), dtype=torch.float64, device=ref_buf.device)
    na = torch.zeros_like(d2)
    nb = torch.zeros_like(d2)
    for lo in range(0, a_all.shape[0], chunk_blocks):
        a = a_all[lo:lo + chunk_blocks].double()
        b = b_all[lo:lo + chunk_blocks].double()
        ca, cb = torch.complex(a[:, 0], a[:, 1]), torch.complex(b[:, 0], b[:, 1])
        ov += (ca.conj() * cb).sum()
        d2 += ((cb - ca).abs() ** 2).sum()
        na += (ca.abs() ** 2).sum()
        nb += (cb.abs() ** 2).sum()
    return float(ov.abs() ** 2 / (na * nb)), float(d2.sqrt())


def large_configs(B, wl, model, stream):
    """The 30-qubit QFT of a seeded basis state (8 GiB state), the 33-qubit grid circuit (6x6 minus
    3 sites, 24 cycles, seed 4; 64 GiB) and the 34-qubit QFT (128 GiB): learned partition vs fixed
    greedy fusion at every max size (3xBF16 tensor cores for 4+ qubit gates), the plain fp32
    CUDA-core K = 4 and post-phase fusion, device time of one circuit each (apply only; the state is
    set before each timing).  Then the 256-circuit HEA batch: one persistent graph launch
    (autotuned) vs the per-circuit launch loop."""
    import torch
    from paper_2602_09604_gb300.state import DeviceState
    out = {}
    for name, n, gates, x in (("qft30", 30, wl.qft_circuit(30), wl.qft_basis_index(30, seed=30)),
                              ("grid33_24c", wl.GRID_33.n, wl.random_grid_circuit(wl.GRID_33, 24, seed=4), 0),
                              ("qft34", 34, wl.qft_circuit(34), wl.qft_basis_index(34, seed=34))):
        st = DeviceState(n, stream=stream)
        res = {}
        variants = [("learned_bf16x3", dict(max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4, model=model)),
                    ("plain_fp32_k4", dict(max_k=4))]
        variants += [(f"greedy_k{k}_bf16x3", dict(max_k=k, precision=B.PREC_BF16X3, tc_min_k=4)) for k in range(2, 7)]
        variants += [("phases_bf16x3", dict(max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3, tc_min_k=4))]
        for label, kw in variants:
            if kw.get("model", 1) is None:
                continue
            f = B.sv_fuse_circuit(gates, n, **kw)
            B.sv_init(st.h, x)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sv_apply_fused_gates(st.h, f)
            e1.record(stream)
            torch.cuda.synchronize()
            res[label] = {"s": e0.elapsed_time(e1) / 1e3, "fused_gates": B.sv_fused_count(f)}
            B.sv_fused_free(f)
        B.sv_device_status()
        st.free()
        del st
        torch.cuda.empty_cache()
        best = min((v["s"], k) for k, v in res.items() if k.startswith("greedy"))
        out[name] = {"n_qubits": n, "gates": len(gates), "variants": res, "best_fixed": best[1],
                     "learned_over_best_fixed": res["learned_bf16x3"]["s"] / best[0] if "learned_bf16x3" in res else None}
    from paper_2602_09604_gb300 import batch as bt
    rep = bt.report()
    out["hea256_batch"] = {k: rep[k] for k in ("workload", "batched_ms", "loop_ms", "speedup", "batched_per_gate_tiles_k4_ms",
                                               "traffic_gb", "fused_gates", "state_mb")}
    out["hea256_batch"]["autotuned"] = {k: rep["autotuned"][k] for k in ("max_k", "stage_log2", "stage_k", "stage_layers", "threads",
                                                                        "ctas_per_sm", "ctas", "wave_mb", "split_min_n")}
    out["hea256_batch"]["list"] = {k: rep["list"][k] for k in ("stages", "stage_gates", "staged", "items")}
    return out


# ------------------------------------------------------------------------------------- oracle arm
def oracle_strata(gates):
    """The circuit's gates grouped by kind (number of targets, number of controls): the oracle's
    time per gate depends on the kind, so samples are drawn per kind and weighted by its count."""
    strata = {}
    for g in gates:
        strata.setdefault((len(g.targets), len(tuple(g.controls))), []).append(g)
    return strata


def run_oracle_steps(n, gates, steps, per_kind):
    """Times the oracle on the n-qubit complex128 state: per step, `per_kind` gates of every kind
    (evenly spaced within the kind).  One untimed gate first touches every page of the state.
    Returns (seconds per circuit = sum over kinds of mean s/gate x the kind's count, threads,
    per-kind detail)."""
    import numpy as np
    import oracle
    oracle.build()
    th = host_cores()
    psi = oracle.basis_state(n, 0)
    strata = oracle_strata(gates)
    oracle.apply_gate(psi, n, gates[0], th)          # page faults of the fresh state, untimed
    detail = {}
    for kind, gl in sorted(strata.items()):
        idx = np.linspace(0, len(gl) - 1, per_kind).round().astype(int)
        t = 0.0
        for _ in range(steps):
            for i in idx:
                t0 = time.perf_counter()
                oracle.apply_gate(psi, n, gl[i], th)
                t += time.perf_counter() - t0
        detail[kind] = {"count": len(gl), "timed": steps * len(idx), "s_per_gate": t / (steps * len(idx))}
    value = sum(d["s_per_gate"] * d["count"] for d in detail.values())
    return value, th, detail


def oracle_sample_text(detail, steps):
    kinds = ", ".join(f"{d['timed']} of the {d['count']} {k[0]}-qubit{' controlled' if k[1] else ''} gates "
                      f"({d['s_per_gate']:.3f} s/gate)" for k, d in sorted(detail.items()))
    return (f"stratified by gate kind over {steps} step(s): {kinds}, applied to the 2^30 complex128 state "
            f"after one untimed gate; s/circuit = sum of mean s/gate x the kind's count")


def bench_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2602_09604_gb300 import workloads as wl
    n, gates = wl.circuit_30q_grid()
    value, th, detail = run_oracle_steps(n, gates, args.steps, args.ref_gates_per_kind)
    timed = sum(d["timed"] for d in detail.values())
    sample = oracle_sample_text(detail, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sum(d["s_per_gate"] * d["timed"] for d in detail.values()) / args.steps * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_qubits": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample,
                             "gates_timed": timed},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------- GPU arm
def bench_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if local == 0:
        import __graft_entry__
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_2602_09604_gb300 import binding as B
    from paper_2602_09604_gb300 import costs
    from paper_2602_09604_gb300 import workloads as wl
    from paper_2602_09604_gb300.state import DeviceState

    n, gates = wl.circuit_30q_grid()
    prec = {"fp32": B.PREC_FP32, "tf32": B.PREC_TF32, "bf16x3": B.PREC_BF16X3}[args.precision]
    model = None
    fusion = args.fusion
    model_path = os.path.join(ROOT, "paper_2602_09604_gb300", "cost_model_gb300.bin")
    if fusion == "learned":
        if os.path.exists(model_path):
            model = B.sv_mlp_load(model_path)
        else:
            fusion = "greedy"
    mode = B.FUSE_LEARNED if fusion == "learned" else B.FUSE_GREEDY
    fuse_kw = dict(max_k=args.max_k, precision=prec, tc_min_k=args.tc_min_k, mode=mode, model=model)
    # a start from |0...0> through sv_init_apply: the light cone on start_qubits qubits fused apart
    start_kw = {"lazy": dict(start_qubits=args.start_qubits), "plain": {}}
    fused_by_start = {m: B.sv_fuse_circuit(gates, n, **fuse_kw, **start_kw[m]) for m in ("lazy", "plain")}
    fused = fused_by_start[args.start]
    n_fused = B.sv_fused_count(fused)
    infos = [B.sv_fused_get_info(fused, i) for i in range(n_fused)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st = DeviceState(n, stream=stream)
    rng = np.random.default_rng(1234 + rank)
    uniforms = rng.random(N_SAMPLES)

    def step(record, start=None):
        start = start or args.start
        fc = fused_by_start[start]
        if start == "lazy":   # gates run on the small state of the qubits named so far, then expand
            rec = B.sv_init_apply(st.h, 0, fc, timings=record)
        else:
            B.sv_init(st.h, 0)
            rec = B.sv_apply_fused_gates(st.h, fc, timings=record)
        smp, nrm = B.sv_sample_norm(st.h, uniforms)   # norm and samples from one read pass
        return rec, nrm, smp

    for _ in range(args.warmup):
        step(False)
    # ---- device-timed region (events on the launching stream)
    kernel_us = {}
    small_source_us = []
    lazy_gates = 0
    # per step: fused gates + chunk sums + scan + search, plus the basis set (plain start) or the
    # small state's basis set, and the expansion unless the first full-state gate read the small
    # state itself (lazy start; counted after the timed steps from the timing records)
    norms = []
    with ClockSampler(dev) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            rec, nrm, _ = step(True)
            norms.append(nrm)
            for info, r in zip(infos, rec):
                if r["path"] == B.PATH_AUTO:   # ran on the small start state, not a full pass
                    lazy_gates += 1
                    continue
                if r["flags"] & B.TIMING_SMALL_SOURCE:   # read only the small state: its own class
                    key = (kernel_class(B, info) + "_small_source", info["k"])
                    small_source_us.append(r["us"])
                    continue
                key = (kernel_class(B, info), info["k"])
                kernel_us.setdefault(key, []).append(r["us"])
        ev1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    elapsed_s = ev0.elapsed_time(ev1) / 1e3
    reads_small = len(small_source_us) >= args.steps
    launches_per_step = n_fused + 3 + (1 + (0 if reads_small else 1) if args.start == "lazy" else 1)
    from paper_2602_09604_gb300.dist import max_over_ranks
    elapsed_s = max_over_ranks(elapsed_s, device="cuda")   # the slowest rank defines the job time
    value = elapsed_s / (args.steps * ws)
    # the other start, device-timed the same way, for comparison
    other = "plain" if args.start == "lazy" else "lazy"
    torch.cuda.synchronize()
    e0o, e1o = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0o.record(stream)
    for _ in range(3):
        step(False, other)
    e1o.record(stream)
    torch.cuda.synchronize()
    other_s = e0o.elapsed_time(e1o) / 3e3

    # ---- end to end through the C ABI with host buffers (host fusion included)
    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f2 = B.sv_fuse_circuit(gates, n, **fuse_kw, **start_kw[args.start])
        if args.start == "lazy":
            B.sv_init_apply(st.h, 0, f2)
        else:
            B.sv_init(st.h, 0)
            B.sv_apply_fused_gates(st.h, f2)
        smp, nrm = B.sv_sample_norm(st.h, uniforms)
        B.sv_fused_free(f2)
        e2e_times.append(time.perf_counter() - t0)
    mat_bytes = sum(2 * 4 * (1 << (2 * i["k"])) for i in infos)

    # ---- the plain path: fp32 CUDA cores, fixed greedy fusion, every max size (device-timed)
    plain = {}
    if not args.no_plain_sweep:
        for mk in range(2, 7):
            fp = B.sv_fuse_circuit(gates, n, max_k=mk, precision=B.PREC_FP32)
            B.sv_init(st.h, 0)
            B.sv_apply_fused_gates(st.h, fp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                B.sv_init(st.h, 0)
                B.sv_apply_fused_gates(st.h, fp)
            e1.record(stream)
            torch.cuda.synchronize()
            plain[str(mk)] = {"s_per_circuit": e0.elapsed_time(e1) / 2e3, "fused_gates": B.sv_fused_count(fp)}
            B.sv_fused_free(fp)
    h2d = 8 * N_SAMPLES + mat_bytes
    d2h = 8 * N_SAMPLES + 8

    # ---- Pauli expectation values on the circuit's state (read-only passes of 8 * 2^n bytes)
    expval = {}
    if not args.no_expval:
        B.sv_init(st.h, 0)
        B.sv_apply_fused_gates(st.h, fused)
        xr = (1 << 3) | (1 << 8) | (1 << 17) | (1 << 29)
        groups = {"z_string_x0": ([0], [(1 << 2) | (1 << 20)]),
                  "xy_string": ([xr], [(1 << 5) | (1 << 3)]),
                  "z_strings_x0": ([0] * 8, [(1 << q) | (1 << (q + 6)) for q in range(8)]),
                  "xy_strings_shared_x": ([xr] * 8, [(1 << q) | (xr if q % 2 else 0) for q in range(8)])}
        for name, (xs, zs) in groups.items():
            B.sv_expval_pauli(st.h, xs, zs)
            ts = []
            for _ in range(5):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.sv_expval_pauli(st.h, xs, zs)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3)
            us = statistics.median(ts)
            expval[name] = {"strings": len(xs), "passes": 1, "us": us,
                            "gbs": (8 << n) / (us * 1e-6) / 1e9}

    # ---- NEXT rows on the same state buffer: controlled-gate kernel, Grover and quantum volume
    next_rows = {}
    accuracy = None
    if not args.no_next_rows:
        rng2 = np.random.default_rng(77)
        ctrl = {}
        for k, c in ((1, 1), (1, 3), (2, 2), (3, 3)):
            qs = [int(q) for q in rng2.permutation(n)]
            g = wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng2), tuple(qs[k:k + c]))
            fc = B.sv_fuse_circuit([g] * 4, n, max_k=1)          # k + c > 1: kept controlled
            recs = B.sv_apply_fused_gates(st.h, fc, timings=True)
            B.sv_fused_free(fc)
            us = statistics.median(r["us"] for r in recs[1:])
            ctrl[f"k{k}_c{c}"] = {"us": us, "gbs": 16 * (1 << (n - c)) / (us * 1e-6) / 1e9,
                                  "bytes": 16 * (1 << (n - c))}
        next_rows["controlled_gate"] = ctrl
        # complex128 states: the benchmark circuit in fp64 (bound by fp64 arithmetic, not HBM)
        c128 = {}
        st128 = DeviceState(n, stream=stream, c128=True)
        for mk in (2, 3):
            fc = B.sv_fuse_circuit(gates, n, max_k=mk)
            ks = [B.sv_fused_get_info(fc, i)["k"] for i in range(B.sv_fused_count(fc))]
            B.sv_init(st128.h, 0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sv_init(st128.h, 0)
            B.sv_apply_fused_gates(st128.h, fc)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            flops = sum((8 * (1 << k) - 2) * (1 << n) for k in ks)
            c128[f"greedy_k{mk}"] = {"s_per_circuit": sec, "fused_gates": len(ks), "tflops": flops / sec / 1e12,
                                     "frac_of_fp64_peak": flops / sec / 1e12 / FP64_PEAK_TFLOPS}
            B.sv_fused_free(fc)
        # the timed step's state (same fused circuit, same start) against the complex128 state
        step(False)
        torch.cuda.synchronize()
        fid, l2 = device_state_metrics(st128.buf, st.buf)
        accuracy = {"fidelity": fid, "one_minus_fidelity": 1.0 - fid, "l2_error": l2,
                    "reference": "complex128 GPU state of the same circuit (fp64, greedy K = 3)",
                    "bar": "F >= 1 - 1e-6 and l2 <= 1e-4"}
        st128.free()
        next_rows["c128_grid30"] = c128
        circ = {"grover30_r3": wl.grover_circuit(n, 0x2C0FFEE1, 3), "qv30": wl.qv_circuit(n, seed=1)}
        for name, gl in circ.items():
            fcirc = B.sv_fuse_circuit(gl, n, **fuse_kw)
            cinfo = [B.sv_fused_get_info(fcirc, i) for i in range(B.sv_fused_count(fcirc))]
            B.sv_init(st.h, 0)
            B.sv_apply_fused_gates(st.h, fcirc)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sv_init(st.h, 0)
            B.sv_apply_fused_gates(st.h, fcirc)
            e1.record(stream)
            torch.cuda.synchronize()
            next_rows[name] = {"gates": len(gl), "fused_gates": len(cinfo),
                               "controlled": sum(1 for i in cinfo if i["path"] == B.PATH_CONTROLLED),
                               "s_per_circuit": e0.elapsed_time(e1) / 1e3}
            B.sv_fused_free(fcirc)

    # ---- roofline of the dominant kernel class
    totals = {k: sum(v) for k, v in kernel_us.items()}
    dom = max(totals, key=totals.get)
    avg_us = statistics.mean(kernel_us[dom])
    bytes_per_launch = costs.bytes_per_pass(n)
    achieved = bytes_per_launch / (avg_us * 1e-6) / 1e9
    peak, src = peaks()
    kernel_key = f"apply_{dom[0]}_k{dom[1]}_n{n}"
    traffic = read_traffic(kernel_key)
    all_us = sum(totals.values())
    # full passes: gates that ran on the full state, less the one that read the small state
    full_passes = n_fused - (lazy_gates + len(small_source_us)) // max(1, args.steps)
    passes_gbs = full_passes * bytes_per_launch / (sum(totals.values()) / args.steps * 1e-6) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_s / args.steps * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_qubits": n, "max_k": args.max_k, "precision": args.precision,
                   "tc_min_k": args.tc_min_k, "fusion": fusion, "fused_gates": n_fused,
                   "fused_k_histogram": {str(k): sum(1 for i in infos if i["k"] == k) for k in range(1, 7)}, "samples_per_step": N_SAMPLES,
                   "l2": "state 8 GiB > 129 MB L2, no flush", "parallelism": f"replicas x{ws}",
                   "start": args.start, "start_qubits": args.start_qubits if args.start == "lazy" else 0,
                   "lazy_start_gates_per_step": lazy_gates // max(1, args.steps)},
        f"s_per_circuit_{other}_start": other_s,
        "e2e": {"value": statistics.mean(e2e_times), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kernel_key,
                     "launches": len(kernel_us[dom]), "avg_us": avg_us, "peak_source": src,
                     "all_apply_kernels_gbs": passes_gbs,
                     "share_of_apply_time": totals[dom] / all_us},
        "per_kernel_class": {f"{p}_k{k}": {"launches": len(v), "avg_us": statistics.mean(v),
                                           "gbs": bytes_per_launch / (statistics.mean(v) * 1e-6) / 1e9}
                             for (p, k), v in sorted(kernel_us.items())},
        "small_source_gate_us": statistics.mean(small_source_us) if small_source_us else None,
        "plain_fusion_fp32": plain,
        "plain_best_s": min((v["s_per_circuit"] for v in plain.values()), default=None),
        "speedup_vs_best_plain": (min(v["s_per_circuit"] for v in plain.values()) / value) if plain else None,
        "norm": norms[-1] if norms else None,
        "expval_pauli": expval or None,
        "next_rows": next_rows or None,
        "accuracy": accuracy,
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, th, detail = run_oracle_steps(n, gates, 1, args.cpu_gates_per_kind)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                                "sample": oracle_sample_text(detail, 1)}
    for fc in fused_by_start.values():
        B.sv_fused_free(fc)
    st.free()
    del st
    torch.cuda.empty_cache()
    if not args.no_large and ws == 1:
        line["large_configs"] = large_configs(B, wl, model, stream)
    if model is not None:
        line["cost_model"] = {k: v for k, v in B.sv_mlp_get_stats(model).items() if k in ("val_mape", "steps")}
        B.sv_mlp_free(model)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--max-k", type=int, default=6)
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--tc-min-k", type=int, default=4)
    ap.add_argument("--fusion", default="learned", choices=["learned", "greedy"])
    ap.add_argument("--no-plain-sweep", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-gates-per-kind", type=int, default=6,
                    help="oracle gates timed per gate kind for cpu_baseline (one step)")
    ap.add_argument("--ref-gates-per-kind", type=int, default=2,
                    help="--impl reference: oracle gates timed per gate kind and step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-expval", action="store_true")
    ap.add_argument("--no-next-rows", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 33-qubit grid, 34-qubit QFT and HEA batch comparisons (run after the timed step)")
    ap.add_argument("--start-qubits", type=int, default=28,
                    help="light cone fused apart for the lazy start (0 = fuse the circuit as one)")
    ap.add_argument("--start", choices=["lazy", "plain"], default="lazy",
                    help="lazy: sv_init_apply (first gates on the small state of the qubits they name); "
                         "plain: sv_init then sv_apply_fused_gates")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
