"""Batched uneven circuits in one persistent (graph-captured) launch: every circuit's state equals
the circuit run alone (and the oracle for the smaller ones), in every shared-memory tier; graph
replays are deterministic; the per-circuit launch loop gives the same states."""
import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import batch
    from paper_2602_09604_gb300 import binding
    return binding, batch


def test_batch_matches_oracle_every_tier(env):
    B, batch = env
    rng = np.random.default_rng(9)
    circuits = [(int(n), wl.hea_circuit(int(n), 3, rng)) for n in [5, 16, 9, 3, 14, 12, 7, 15, 10, 13, 1, 11]]
    refs = [oracle.run_circuit(n, g, 0) for n, g in circuits]
    for max_k in (2, 3, 4):
        b = batch.Batch(circuits, max_k)
        for smem_n in (0, 12, 14):
            for threads in (128, 512):
                b.set(threads, smem_n, 7)
                b.arena.fill_(float("nan"))
                b.run()
                for i, ref in enumerate(refs):
                    got = b.state(i)
                    assert oracle.fidelity(ref, got) >= 1 - 1e-6, (max_k, smem_n, i)
                    assert oracle.l2_error(ref, got) <= 1e-4
        b.free()


def test_graph_replay_is_deterministic_and_loop_agrees(env):
    B, batch = env
    circuits = wl.hea_batch(count=40, n_lo=8, n_hi=17, layers=4, seed=3)
    b = batch.Batch(circuits, 4)
    b.set(256, 13, 64, use_graph=True)
    b.run()
    first = b.arena.clone()
    b.arena.zero_()
    b.run()
    assert bool((first == b.arena).all())
    b.arena.fill_(float("nan"))
    b.run_loop()
    for i in range(len(circuits)):
        g = b.state(i)
        ref = first[B.sv_batch_state_offset(b.h, i) // 4:].cpu().numpy()
        nf = max(2 << circuits[i][0], 64)
        blk = ref[:nf].reshape(-1, 2, 32)
        r = (blk[:, 0, :] + 1j * blk[:, 1, :]).reshape(-1)[: 1 << circuits[i][0]]
        assert np.max(np.abs(g - r)) <= 1e-5
    b.free()


def test_batch_rejects_bad_input(env):
    B, batch = env
    import torch
    n = 10
    f6 = B.sv_fuse_circuit([wl.Gate(tuple(range(6)), wl.random_unitary(64, np.random.default_rng(0)))], n, max_k=6)
    buf = torch.empty(B.sv_batch_arena_bytes([n]) // 4, dtype=torch.float32, device="cuda")
    with pytest.raises(B.SvError):
        B.sv_batch_create([f6], buf.data_ptr(), buf.numel() * 4)      # k > 4 is not batched
    f2 = B.sv_fuse_circuit(wl.hea_circuit(n, 1, np.random.default_rng(1)), n, max_k=2)
    with pytest.raises(B.SvError) as e:
        B.sv_batch_create([f2], buf.data_ptr(), 64)                   # arena too small
    assert e.value.code == B.SV_ENOMEM
    B.sv_fused_free(f6)
    B.sv_fused_free(f2)


def test_autotuner_picks_a_measured_best(env, tmp_path):
    B, batch = env
    circuits = wl.hea_batch(count=24, n_lo=8, n_hi=16, layers=3, seed=4)
    best, log = batch.autotune(circuits, repeats=2, cache=str(tmp_path / "c.json"), use_cache=False, k_range=(2, 4))
    assert log and best["ms"] <= min(t["ms"] for t in log) + 1e-9
    again, log2 = batch.autotune(circuits, cache=str(tmp_path / "c.json"))
    assert again == best and log2 == []
