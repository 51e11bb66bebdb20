"""Self-recorded fused-gate timings (the training data of the learned cost model).

The simulator times its own kernels: single random fused gates of chosen size k, target set and
kernel path are applied to an n-qubit state through ``sv_apply_fused_gates`` with CUDA-event
timing records, and the median over repeats is kept.  Gates are built without fusion
(``FUSE_NONE``) so each record is exactly one kernel launch.
"""
from __future__ import annotations

import statistics
from collections import defaultdict

import numpy as np

from . import binding as B
from . import workloads as wl


def path_ok(path: int, targets) -> bool:
    if path == B.PATH_HIGH:
        return all(t >= 5 for t in targets)
    return True


def random_targets(n: int, k: int, rng: np.random.Generator, cls: str):
    """k distinct targets of class 'low' (all < 5), 'high' (all >= 5), 'mixed' or 'any'."""
    if cls == "low" and k <= 5:
        return tuple(sorted(int(t) for t in rng.choice(5, size=k, replace=False)))
    if cls == "high" and n - 5 >= k:
        return tuple(sorted(int(t) for t in 5 + rng.choice(n - 5, size=k, replace=False)))
    if cls == "mixed" and k >= 2 and n - 5 >= 1:
        nl = int(rng.integers(1, min(k - 1, 5) + 1))
        nh = k - nl
        if nh <= n - 5:
            lo = rng.choice(5, size=nl, replace=False)
            hi = 5 + rng.choice(n - 5, size=nh, replace=False)
            return tuple(sorted(int(t) for t in np.concatenate([lo, hi])))
    return tuple(sorted(int(t) for t in rng.choice(n, size=k, replace=False)))


def time_specs(specs, repeats: int = 5, seed: int = 0, precision: int = B.PREC_FP32, warm: int = 1):
    """specs: iterable of (n, targets, path).  Returns a list of dicts with the median microseconds."""
    from .state import DeviceState
    rng = np.random.default_rng(seed)
    by_n = defaultdict(list)
    for i, (n, targets, path) in enumerate(specs):
        by_n[n].append((i, tuple(targets), path))
    out = [None] * sum(len(v) for v in by_n.values())
    for n, items in sorted(by_n.items()):
        st = DeviceState(n)
        st.init(0)
        by_path = defaultdict(list)
        for i, targets, path in items:
            by_path[path].append((i, targets))
        for path, lst in by_path.items():
            gates = []
            for _, targets in lst:
                g = wl.random_gate(n, len(targets), rng, targets=targets)
                gates += [g] * (repeats + warm)
            f = B.sv_fuse_circuit(gates, n, mode=B.FUSE_NONE, precision=precision, force_path=path,
                                  max_k=6)
            try:
                rec = st.apply(f, timings=True)
            finally:
                B.sv_fused_free(f)
            for s, (i, targets) in enumerate(lst):
                r = rec[s * (repeats + warm) + warm:(s + 1) * (repeats + warm)]
                out[i] = {"n": n, "k": len(targets), "targets": targets, "path": r[0]["path"],
                          "us": statistics.median(x["us"] for x in r)}
        st.free()
    return out


def random_post_targets(n: int, rng: np.random.Generator):
    """Six targets a post-phase gate can have: at most two below qubit 5, not both 0 and 1."""
    while True:
        nl = int(rng.integers(0, 3))
        lo = [int(t) for t in rng.choice(5, size=nl, replace=False)]
        if {0, 1} <= set(lo):
            continue
        hi = [int(t) for t in 5 + rng.choice(n - 5, size=6 - nl, replace=False)]
        return tuple(sorted(lo + hi))


def fuse_post_gates(n: int, target_sets, per: int, rng: np.random.Generator, precision: int = B.PREC_BF16X3):
    """Fused circuit (``FUSE_PHASES``) of `per` gates with post-phases for each target set, in order:
    a random 6-qubit unitary on the targets followed by two to four controlled phases from a
    target to a qubit outside them.  Raises if the gates do not fuse one to one."""
    gates = []
    for targets in target_sets:
        outside = [q for q in range(n) if q not in targets]
        for _ in range(per):
            gates.append(wl.random_gate(n, 6, rng, targets=targets))
            for _ in range(int(rng.integers(2, 5))):
                a = int(rng.choice(targets))
                b = int(rng.choice(outside))
                th = float(rng.uniform(-np.pi, np.pi))
                gates.append(wl.Gate((a, b), np.diag([1, 1, 1, np.exp(1j * th)]).astype(np.complex128)))
    f = B.sv_fuse_circuit(gates, n, mode=B.FUSE_PHASES, precision=precision, max_k=6, tc_min_k=4)
    ok = B.sv_fused_count(f) == len(target_sets) * per
    for g in range(B.sv_fused_count(f) if ok else 0):
        ok = ok and B.sv_fused_get_post_phases(f, g) and B.sv_fused_get_info(f, g)["k"] == 6
    if not ok:
        B.sv_fused_free(f)
        raise RuntimeError("fuse_post_gates: the gates did not fuse one to one into gates with post-phases")
    return f


def time_post_specs(specs, repeats: int = 5, seed: int = 0, precision: int = B.PREC_BF16X3, warm: int = 1):
    """Gates that carry post-phases (made by fuse_post_gates), specs: iterable of (n, targets) with
    six targets.  Returns dicts like time_specs, with "post": True."""
    from .state import DeviceState
    rng = np.random.default_rng(seed)
    by_n = defaultdict(list)
    for i, (n, targets) in enumerate(specs):
        by_n[n].append((i, tuple(targets)))
    out = [None] * sum(len(v) for v in by_n.values())
    per = repeats + warm
    for n, items in sorted(by_n.items()):
        st = DeviceState(n)
        st.init(0)
        f = fuse_post_gates(n, [t for _, t in items], per, rng, precision)
        try:
            rec = st.apply(f, timings=True)
        finally:
            B.sv_fused_free(f)
        for s, (i, targets) in enumerate(items):
            r = rec[s * per + warm:(s + 1) * per]
            out[i] = {"n": n, "k": 6, "targets": targets, "path": r[0]["path"], "post": True,
                      "us": statistics.median(x["us"] for x in r)}
        st.free()
    return out


def main(argv=None):
    """Time single fused gates: python -m paper_2602_09604_gb300.timing_sweep --n 26 --targets 0,1,2,4,10,24 ..."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--targets", required=True, help="comma-separated target qubits")
    ap.add_argument("--path", default="auto", choices=list(B.PATH_NAMES.values()))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--warm", type=int, default=1)
    args = ap.parse_args(argv)
    path = {v: k for k, v in B.PATH_NAMES.items()}[args.path]
    prec = {"fp32": B.PREC_FP32, "tf32": B.PREC_TF32, "bf16x3": B.PREC_BF16X3}[args.precision]
    targets = tuple(int(t) for t in args.targets.split(","))
    rec = time_specs([(args.n, targets, path)], repeats=args.repeats, precision=prec, warm=args.warm)[0]
    rec["gbs"] = 16 * (1 << args.n) / (rec["us"] * 1e-6) / 1e9
    rec["path"] = B.PATH_NAMES[rec["path"]]
    B.sv_device_status()
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
