"""Multi-process host logic on CPU with the gloo backend (world size 2): circuit sharding for the
batch (no data exchange) and the max-over-ranks job time used by the benchmark."""
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
