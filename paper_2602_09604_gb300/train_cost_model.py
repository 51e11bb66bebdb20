"""Collect self-recorded fused-gate timings and train the learned fusion cost model on the GPU.

    python -m paper_2602_09604_gb300.train_cost_model --out cost_model_gb300.bin --data timings.csv

Timings: random fused gates (k = 1..6; targets all below qubit 5, all at or above it, mixed, or
anywhere) on n = 24..32-qubit states, on every kernel path that can run them (CUDA-core class
path, tensor cores in 3xBF16 and TF32 for k >= 4), median of repeats after a warm-up launch
(timing_sweep.time_specs); and six-qubit tensor-core gates that carry post-phases
(timing_sweep.time_post_specs, feature post_phases = 1).  Training: sv_mlp_train (the library's
forward / backward / Adam kernels), 10% held out to measure the prediction error.
"""
from __future__ import annotations

import argparse
import csv
import json
import time

import numpy as np

from . import binding as B
from .timing_sweep import random_post_targets, random_targets, time_post_specs, time_specs

# specs per qubit count: more where a pass is cheap
DEFAULT_COUNTS = {24: 1400, 25: 900, 26: 900, 27: 700, 28: 700, 29: 450, 30: 350, 31: 220, 32: 160}
POST_FRACTION = 0.06   # gates with post-phases, per qubit count, relative to the counts above


def make_specs(counts, seed):
    rng = np.random.default_rng(seed)
    specs = []
    for n, cnt in counts.items():
        for _ in range(cnt):
            k = int(rng.integers(1, 7))
            cls = ["low", "high", "mixed", "any"][int(rng.integers(0, 4))]
            t = random_targets(n, k, rng, cls)
            specs.append((n, t, B.PATH_AUTO, B.PREC_FP32))
            if k >= 4 and n >= k + 5:
                specs.append((n, t, B.PATH_TC_BF16X3, B.PREC_BF16X3))
                if rng.random() < 0.5:
                    specs.append((n, t, B.PATH_TC_TF32, B.PREC_TF32))
    return specs


def make_post_specs(counts, seed):
    rng = np.random.default_rng(seed + 1)
    specs = {B.PREC_BF16X3: [], B.PREC_TF32: []}
    for n, cnt in counts.items():
        for _ in range(max(1, int(round(POST_FRACTION * cnt)))):
            prec = B.PREC_BF16X3 if rng.random() < 0.7 else B.PREC_TF32
            specs[prec].append((n, random_post_targets(n, rng)))
    return specs


def collect(counts=None, seed=7, repeats=3):
    counts = counts or DEFAULT_COUNTS
    specs = make_specs(counts, seed)
    rows = []
    for prec in (B.PREC_FP32, B.PREC_BF16X3, B.PREC_TF32):
        sp = [(n, t, p) for n, t, p, pr in specs if pr == prec]
        if sp:
            rows += time_specs(sp, repeats=repeats, precision=prec, seed=seed)
    for prec, sp in make_post_specs(counts, seed).items():
        if sp:
            rows += time_post_specs(sp, repeats=repeats, precision=prec, seed=seed)
    return rows


def featurize(rows):
    X = np.stack([B.sv_mlp_features(r["k"], r["targets"], r["path"], r["n"], r.get("post", False))
                  for r in rows]).astype(np.float32)
    us = np.array([r["us"] for r in rows], dtype=np.float32)
    return X, us


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--data", default=None, help="write the timing records here (csv)")
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--scale", type=float, default=1.0, help="multiply the per-n spec counts")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--fallback-k", type=int, default=4)
    args = ap.parse_args(argv)
    counts = {n: max(1, int(c * args.scale)) for n, c in DEFAULT_COUNTS.items()}
    t0 = time.time()
    rows = collect(counts, seed=args.seed)
    t1 = time.time()
    if args.data:
        with open(args.data, "w", newline="") as fh:
            w = csv.writer(fh)
            w.writerow(["n", "k", "targets", "path", "post", "us"])
            for r in rows:
                w.writerow([r["n"], r["k"], " ".join(map(str, r["targets"])), B.PATH_NAMES[r["path"]],
                            int(r.get("post", False)), f"{r['us']:.3f}"])
    X, us = featurize(rows)
    m = B.sv_mlp_create(seed=args.seed)
    stats = B.sv_mlp_train(m, X, us, epochs=args.epochs, seed=args.seed, fallback_k=args.fallback_k)
    t2 = time.time()
    B.sv_mlp_save(m, args.out)
    B.sv_mlp_free(m)
    print(json.dumps({"records": len(rows), "collect_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
                      "stats": stats, "model": args.out}))


if __name__ == "__main__":
    main()
