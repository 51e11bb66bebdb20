"""Batched uneven circuits in one persistent launch, with a project-written autotuner.

The autotuner times the real batch on the GPU for candidate settings -- the circuits' fusion size
(2..4, or none: then staged circuits are fused per stage and their diagonal +-1 gates become sign
runs), the stage tile size (or one pass per fused gate) and the stage re-fusion size, CTA size, the largest
circuit kept in shared memory, the smallest circuit split across CTAs, the per-gate tile size, the
wave size (MB of split-circuit state per wave), and the persistent grid -- by coordinate descent
from a default, each candidate replayed from its captured CUDA graph and timed with CUDA events
(median of repeats).  The winner is cached in a JSON file keyed by GPU name and a digest of the
batch's circuit sizes and gate counts.

    python -m paper_2602_09604_gb300.batch --report     # HEA batch: 256 circuits, n ~ U{10..20}

Several GPUs (one process each, launched by torchrun) split the batch by circuit with no data
exchange: each rank autotunes and runs its balanced share in one persistent launch, and the job
time is the slowest rank's (``dist.sharded_batch_time``):

    python -m torch.distributed.run --nproc-per-node N -m paper_2602_09604_gb300.batch --shard
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics

import numpy as np
import torch

from . import binding as B
from . import workloads as wl

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batch_autotune.json")


class Batch:
    """Device arena + fused circuits + sv_batch handle for one fusion size (max_k = 0: every gate
    kept as it is, so staged circuits are fused per stage, with their diagonal +-1 gates -- CZ, Z --
    applied as sign runs instead of dense matrices)."""

    def __init__(self, circuits, max_k: int, stream: torch.cuda.Stream | None = None):
        self.circuits = circuits
        self.max_k = max_k
        self.ns = [n for n, _ in circuits]
        self.stream = stream or torch.cuda.current_stream()
        self.nbytes = B.sv_batch_arena_bytes(self.ns)
        self.arena = torch.empty(self.nbytes // 4, dtype=torch.float32, device="cuda")
        self.fused = [B.sv_fuse_circuit(g, n, max_k=max_k) if max_k > 0 else
                      B.sv_fuse_circuit(g, n, max_k=4, mode=B.FUSE_NONE) for n, g in circuits]
        self.h = B.sv_batch_create(self.fused, self.arena.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def set(self, threads, smem_max_n, ctas, use_graph=True, split_min_n=15, tile_log2=12, wave_mb=0, stage_log2=0,
            stage_k=0, stage_layers=0, ctas_per_sm=1):
        B.sv_batch_set_opts(self.h, threads, smem_max_n, ctas, use_graph, split_min_n, tile_log2, wave_mb, stage_log2,
                            stage_k, stage_layers, ctas_per_sm)

    def run(self):
        B.sv_batch_run(self.h)

    def run_loop(self):
        B.sv_batch_run_loop(self.h)

    def time(self, fn, repeats=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def state(self, i: int) -> np.ndarray:
        """Circuit i's state as interleaved complex64 (host)."""
        n = self.ns[i]
        off = B.sv_batch_state_offset(self.h, i) // 4
        nf = max(2 << n, 64)
        blk = self.arena[off:off + nf].cpu().numpy().reshape(-1, 2, 32)
        amp = (blk[:, 0, :] + 1j * blk[:, 1, :]).reshape(-1)[: 1 << n]
        return amp.astype(np.complex64)

    def free(self):
        if self.h is not None:
            B.sv_batch_free(self.h)
            for f in self.fused:
                B.sv_fused_free(f)
            self.h = None


def digest(circuits) -> str:
    h = hashlib.sha256()
    for n, g in circuits:
        h.update(f"{n}:{len(g)};".encode())
    return h.hexdigest()[:16]


FIELDS = ("threads", "smem_max_n", "ctas", "split_min_n", "tile_log2", "wave_mb", "stage_log2", "stage_k",
          "stage_layers", "ctas_per_sm")


def apply(b: "Batch", cfg: dict, use_graph: bool = True) -> None:
    b.set(*(cfg[f] for f in FIELDS[:3]), use_graph, *(cfg[f] for f in FIELDS[3:]))


def autotune(circuits, repeats=5, cache=CACHE, use_cache=True, k_range=(0, 2, 3, 4), rounds=2):
    """Returns (best settings dict, trial log).  Coordinate descent over the fusion size and every
    batch option, up to `rounds` sweeps (stopping early when a sweep changes nothing)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = f"v7|{torch.cuda.get_device_name(0)}|{digest(circuits)}"
    if use_cache and os.path.exists(cache):
        try:
            got = json.load(open(cache)).get(key)
            if got:
                return got, []
        except Exception:
            pass
    log = []
    best = {"max_k": 0, "threads": 512, "smem_max_n": 0, "ctas": sms, "split_min_n": 8, "tile_log2": 12,
            "wave_mb": 48, "stage_log2": 14, "stage_k": 2, "stage_layers": 1, "ctas_per_sm": 1}
    batches = {}

    def measure(cfg):
        if cfg["max_k"] not in batches:
            batches[cfg["max_k"]] = Batch(circuits, cfg["max_k"])
        b = batches[cfg["max_k"]]
        apply(b, cfg)
        ms = b.time(b.run, repeats)
        log.append(dict(cfg, ms=ms))
        return ms

    # "form": threads per CTA and CTAs per SM together (two per SM take at most 256 threads and
    # shared memory for two, so stage tiles of at most 13 qubits and at least 2 x SMs CTAs)
    forms = ((512, 1), (256, 1), (128, 1), (256, 2), (128, 2))

    def variant(cfg, field, v):
        if field != "form":
            return dict(cfg, **{field: v})
        c = dict(cfg, threads=v[0], ctas_per_sm=v[1])
        if v[1] == 2:
            c["stage_log2"] = min(c["stage_log2"], 13)
            c["smem_max_n"] = min(c["smem_max_n"], 13)
            c["ctas"] = max(c["ctas"], 2 * sms)
        return c

    space = (("max_k", k_range), ("stage_log2", (0, 11, 12, 13, 14)), ("stage_k", (0, 2, 3, 4)), ("stage_layers", (0, 1)),
             ("form", forms), ("smem_max_n", (0, 11, 12, 13, 14)),
             ("split_min_n", (0, 8, 10, 11, 13, 14, 15, 16, 17)), ("tile_log2", (10, 11, 12, 13, 14)),
             ("wave_mb", (0, 24, 48, 96)), ("ctas", (sms, 2 * sms, 3 * sms, 4 * sms)))
    try:
        best_ms = measure(best)
        for _ in range(rounds):
            changed = False
            for field, values in space:
                if field == "tile_log2" and best["stage_log2"] > 0:
                    continue   # per-gate tiles only
                if field in ("stage_k", "stage_layers") and best["stage_log2"] == 0:
                    continue
                for v in values:
                    if v == (best[field] if field != "form" else (best["threads"], best["ctas_per_sm"])):
                        continue
                    cfg = variant(best, field, v)
                    try:
                        ms = measure(cfg)
                    except B.SvError:
                        continue
                    if ms < best_ms:
                        best, best_ms, changed = cfg, ms, True
            if not changed:
                break
    finally:
        for b in batches.values():
            b.free()
    best = dict(best, ms=best_ms)
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[key] = best
        json.dump(data, open(cache, "w"), indent=1)
    except Exception:
        pass
    return best, log


def report(count=256, seed=5):
    circuits = wl.hea_batch(count=count, seed=seed)
    best, log = autotune(circuits, use_cache=False)
    b = Batch(circuits, best["max_k"])
    apply(b, best)
    info = B.sv_batch_get_info(b.h)
    t_batch = b.time(b.run)
    apply(b, dict(best, stage_log2=0))
    info_gate = B.sv_batch_get_info(b.h)
    t_per_gate = b.time(b.run)
    apply(b, dict(best, stage_log2=0, split_min_n=0))
    t_nosplit = b.time(b.run)
    t_loop_same_k = b.time(b.run_loop, repeats=3)
    # the comparisons at their own best fusion size (k = 4 for one launch or one pass per gate)
    b4 = Batch(circuits, 4)
    apply(b4, dict(best, max_k=4, threads=256, smem_max_n=12, split_min_n=15, tile_log2=13, wave_mb=0, stage_log2=0,
                   stage_k=0, stage_layers=0, ctas_per_sm=1))
    t_per_gate_k4 = b4.time(b4.run)
    t_loop = b4.time(b4.run_loop, repeats=3)
    b4.free()
    out = {"workload": f"{count} HEA circuits, n ~ U{{10..20}}, 8 layers RZ RY + CZ ladder, seed {seed}",
           "batched_ms": t_batch, "batched_per_gate_tiles_ms": t_per_gate, "batched_no_split_ms": t_nosplit,
           "batched_per_gate_tiles_k4_ms": t_per_gate_k4, "loop_ms": t_loop, "loop_same_k_ms": t_loop_same_k,
           "speedup": t_loop / t_batch, "autotuned": best, "trials": len(log),
           "fused_gates": sum(B.sv_fused_count(f) for f in b.fused), "state_mb": b.nbytes / 1e6,
           "list": info, "traffic_gb": info["traffic_bytes"] / 1e9,
           "traffic_gbs": info["traffic_bytes"] / (t_batch * 1e-3) / 1e9,
           "per_gate_traffic_gb": info_gate["traffic_bytes"] / 1e9}
    b.free()
    return out


def run_sharded(count=256, seed=5, repeats=5):
    """This process's rank (RANK / LOCAL_RANK / WORLD_SIZE from torchrun; one GPU each) runs its
    share of the HEA batch; rank 0 returns the job line, the others None."""
    import torch.distributed as tdist
    from . import dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl")
    circuits = wl.hea_batch(count=count, seed=seed)
    tuned = {}

    def time_share(share):
        best, _ = autotune(share)
        b = Batch(share, best["max_k"])
        try:
            apply(b, best)
            ms = b.time(b.run, repeats)
            B.sv_device_status()
        finally:
            b.free()
        tuned.update(best)
        return ms

    idx, job_ms = dist.sharded_batch_time(circuits, rank, world, time_share, device="cuda")
    if world > 1:
        tdist.destroy_process_group()
    if rank != 0:
        return None
    return {"workload": f"{count} HEA circuits, n ~ U{{10..20}}, seed {seed}", "ranks": world,
            "job_ms": job_ms, "rank0_circuits": len(idx), "rank0_autotuned": tuned}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--report", action="store_true")
    ap.add_argument("--shard", action="store_true", help="one rank per GPU under torchrun, batch split by circuit")
    ap.add_argument("--count", type=int, default=256)
    a = ap.parse_args()
    import __graft_entry__  # noqa: F401  (build)
    if a.shard:
        line = run_sharded(a.count)
        if line is not None:
            print(json.dumps(line))
    else:
        print(json.dumps(report(a.count)))
