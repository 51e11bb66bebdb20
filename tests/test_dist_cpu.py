"""Multi-process host logic on CPU with the gloo backend (world size 2): circuit sharding for the
batch (no data exchange), the sharded batch driver's job time (the path `batch.py --shard` runs
on GPUs, here with a stand-in timer) and the max-over-ranks job time used by the benchmark."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2602_09604_gb300 import dist as D


def test_shard_partitions_items():
    items = list(range(11))
    parts = [D.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        D.shard(items, 3, 3)


def test_shard_balanced_is_a_partition_and_balances():
    sizes = [2 ** n for n in (20, 10, 19, 12, 20, 15, 11, 18)]
    parts = [D.shard_balanced(sizes, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) <= sum(sizes) / 3 + max(sizes)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = D.shard_balanced([2 ** n for n in range(10, 21)], rank, world)
        t = D.max_over_ranks(1.0 + rank)          # the slowest rank defines the job time
        q.put((rank, mine, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_agree_on_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    assert sorted(got[0][1] + got[1][1]) == list(range(11))
    assert not set(got[0][1]) & set(got[1][1])
    assert got[0][2] == got[1][2] == 2.0


def _sharded_worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2602_09604_gb300 import workloads as wl
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        circuits = wl.hea_batch(count=64, seed=5)
        # stand-in timer: the share's work in units of 2^20 amplitude-gates
        idx, job = D.sharded_batch_time(circuits, rank, world,
                                        lambda share: sum((1 << n) * len(g) for n, g in share) / 2.0 ** 20)
        q.put((rank, idx, job, sum((1 << circuits[i][0]) * len(circuits[i][1]) for i in idx) / 2.0 ** 20))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_driver_two_gloo_ranks():
    """The HEA batch split across two ranks: the shares are disjoint and cover every circuit, each
    rank times only its own share, and both ranks report the slower rank's time as the job time."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, i0, j0, w0), (_, i1, j1, w1) = got
    assert not set(i0) & set(i1)
    assert sorted(i0 + i1) == list(range(64))
    assert j0 == j1 == max(w0, w1)
    assert max(w0, w1) <= 1.1 * min(w0, w1)     # balanced to within 10%
