"""Host-side multi-process helpers (one process per GPU).

A single circuit is not sharded across GPUs here: ranks run independent replicas, so the only
cross-rank steps are agreeing on the timing (the slowest rank defines the job time) and, for a
batch of independent circuits, splitting the circuits among ranks without any data exchange.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` (every item to exactly one rank, sizes differ by <= 1)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    return [x for i, x in enumerate(items) if i % world == rank]


def shard_balanced(sizes, rank: int, world: int):
    """Indices of the items for `rank` when item i costs sizes[i]: greedy longest-first onto the
    least-loaded rank (deterministic, identical on every rank)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    load = [0.0] * world
    owner = {}
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(value: float, device=None) -> float:
    """All-reduce MAX of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_circuits(circuits, rank: int, world: int):
    """`rank`'s share of a batch of (n_qubits, gates) circuits: every circuit goes to exactly one
    rank, balanced by the work of one pass per gate (2^n amplitudes x gate count).  Returns
    (indices into `circuits`, the circuits)."""
    cost = [float(1 << int(n)) * max(1, len(g)) for n, g in circuits]
    idx = shard_balanced(cost, rank, world)
    return idx, [circuits[i] for i in idx]


def sharded_batch_time(circuits, rank: int, world: int, time_share, device=None):
    """Runs this rank's share through `time_share(share) -> milliseconds` and returns
    (indices of the share, job milliseconds = the slowest rank's).  No circuit data crosses
    ranks: only the one float of the timing reduction."""
    idx, share = shard_circuits(circuits, rank, world)
    ms = time_share(share) if share else 0.0
    return idx, max_over_ranks(ms, device=device)
