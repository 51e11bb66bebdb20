"""Run one library operation on a synthetic state and print its device time (CUDA events).

For timing and profiling single kernels outside the full circuit step:

    python -m paper_2602_09604_gb300.opbench expval --n 26 --strings 8
    python -m paper_2602_09604_gb300.opbench controlled --n 26 --k 1 --controls 7,12
    python -m paper_2602_09604_gb300.opbench batch --count 64
    python -m paper_2602_09604_gb300.opbench qft --n 27 --mode phases

Every run does --warm untimed repetitions, then --repeats timed ones, and prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np
import torch

from . import binding as B
from . import workloads as wl
from .state import DeviceState


def _time(fn, stream, warm, repeats):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3)
    return statistics.median(ts)


def run_expval(a):
    st = DeviceState(a.n)
    st.init(0)
    x = int(a.x, 0)
    xs = [x] * a.strings
    zs = [((1 << (s % a.n)) | (1 << ((3 * s + 7) % a.n))) for s in range(a.strings)]
    us = _time(lambda: B.sv_expval_pauli(st.h, xs, zs), st.stream, a.warm, a.repeats)
    st.free()
    return {"op": "expval", "n": a.n, "strings": a.strings, "x": x, "us": us,
            "gbs": (8 << a.n) / (us * 1e-6) / 1e9}


def run_controlled(a):
    rng = np.random.default_rng(a.seed)
    controls = tuple(int(q) for q in a.controls.split(","))
    targets = tuple(int(q) for q in a.targets.split(","))
    g = wl.Gate(targets, wl.random_unitary(1 << len(targets), rng), controls)
    f = B.sv_fuse_circuit([g], a.n, max_k=1)   # k + controls > 1: kept controlled
    st = DeviceState(a.n)
    st.init(0)
    us = _time(lambda: st.apply(f), st.stream, a.warm, a.repeats)
    st.free()
    B.sv_fused_free(f)
    c = len(controls)
    return {"op": "controlled", "n": a.n, "targets": targets, "controls": controls, "us": us,
            "gbs": 16 * (1 << (a.n - c)) / (us * 1e-6) / 1e9}


def run_batch(a):
    from .batch import Batch
    circuits = wl.hea_batch(count=a.count, seed=a.seed)
    b = Batch(circuits, a.max_k)
    ctas = a.ctas or 2 * torch.cuda.get_device_properties(0).multi_processor_count
    b.set(a.threads, a.smem_max_n, ctas, True, a.split_min_n, a.tile_log2, a.wave_mb, a.stage_log2, a.stage_k,
          a.stage_layers, a.ctas_per_sm)
    us = _time(b.run, b.stream, a.warm, a.repeats)
    B.sv_device_status()
    info = B.sv_batch_get_info(b.h)
    b.free()
    return {"op": "batch", "count": a.count, "us": us, "list": info,
            "traffic_gbs": info["traffic_bytes"] / (us * 1e-6) / 1e9}


def run_qft(a):
    """The n-qubit QFT of a seeded basis state, fused in the given mode (3xBF16 tensor cores for
    4+ qubit gates), applied whole: the circuit's device time and each fused gate's."""
    gates = wl.qft_circuit(a.n)
    x = wl.qft_basis_index(a.n, seed=a.n)
    kw = dict(max_k=6, precision=B.PREC_BF16X3, tc_min_k=4)
    model = None
    if a.mode == "phases":
        kw["mode"] = B.FUSE_PHASES
    elif a.mode == "learned":
        import os
        model = B.sv_mlp_load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cost_model_gb300.bin"))
        kw.update(mode=B.FUSE_LEARNED, model=model)
    f = B.sv_fuse_circuit(gates, a.n, **kw)
    st = DeviceState(a.n)
    ts = []
    for r in range(a.warm + a.repeats):   # the state is set before each run, outside the timing
        st.init(x)
        ts.append(_time(lambda: st.apply(f), st.stream, 0, 1))
    us = statistics.median(ts[a.warm:])
    st.init(x)
    rec = st.apply(f, timings=True)
    B.sv_device_status()
    out = {"op": "qft", "n": a.n, "mode": a.mode, "fused": B.sv_fused_count(f), "us": us,
           "gates": [(r["k"], B.PATH_NAMES[r["path"]], round(r["us"], 1)) for r in rec], "norm": st.norm()}
    st.free()
    B.sv_fused_free(f)
    if model is not None:
        B.sv_mlp_free(model)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["expval", "controlled", "batch", "qft"])
    ap.add_argument("--mode", default="phases", choices=["phases", "learned", "greedy"], help="qft: fusion mode")
    ap.add_argument("--n", type=int, default=26)
    ap.add_argument("--strings", type=int, default=1)
    ap.add_argument("--x", default="0x20108", help="x mask of the Pauli strings")
    ap.add_argument("--targets", default="9")
    ap.add_argument("--controls", default="7")
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--max-k", type=int, default=4)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--smem-max-n", type=int, default=0)
    ap.add_argument("--split-min-n", type=int, default=17)
    ap.add_argument("--tile-log2", type=int, default=12)
    ap.add_argument("--wave-mb", type=int, default=0)
    ap.add_argument("--stage-log2", type=int, default=0)
    ap.add_argument("--stage-k", type=int, default=0)
    ap.add_argument("--stage-layers", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=1)
    ap.add_argument("--ctas", type=int, default=0, help="persistent CTAs (0: twice the SM count)")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--warm", type=int, default=1)
    ap.add_argument("--repeats", type=int, default=3)
    a = ap.parse_args(argv)
    out = {"expval": run_expval, "controlled": run_controlled, "batch": run_batch, "qft": run_qft}[a.op](a)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
