"""Batched uneven circuits in one persistent (graph-captured) launch: every circuit's state equals
the oracle in every item kind (shared-memory circuits, single-CTA global circuits, circuits split
into tiles that all CTAs share, with tiles from 32 to 4096 groups and from 1 to many CTAs,
circuits run in stages of shared-memory tiles of 2^8 to 2^14 amplitudes); graph
replays are deterministic; the per-circuit launch loop gives the same states; a wait that cannot
be satisfied gives up and is reported without a fault."""
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
    # (threads, smem_max_n, ctas, split_min_n, tile_log2, wave_mb)
    configs = [(128, 0, 7, 0, 12, 0), (512, 12, 7, 0, 12, 0), (256, 14, 7, 0, 12, 0),
               (256, 9, 7, 6, 5, 0), (128, 0, 1, 1, 7, 1), (512, 12, 300, 13, 12, 0), (256, 10, 19, 11, 8, 1),
               (256, 0, 40, 8, 6, 1)]
    for max_k in (2, 3, 4):
        b = batch.Batch(circuits, max_k)
        for threads, smem_n, ctas, split_n, tl, wave in configs:
            b.set(threads, smem_n, ctas, True, split_n, tl, wave)
            b.arena.fill_(float("nan"))
            b.run()
            B.sv_device_status()
            for i, ref in enumerate(refs):
                got = b.state(i)
                cfg = (max_k, threads, smem_n, ctas, split_n, tl, wave, i)
                assert oracle.fidelity(ref, got) >= 1 - 1e-6, cfg
                assert oracle.l2_error(ref, got) <= 1e-4, cfg
        b.free()


def _random_circuit(n, count, rng):
    """Gates of 1-3 qubits on random qubits (any position, low and high), random unitaries."""
    gates = []
    for _ in range(count):
        k = int(rng.integers(1, min(3, n) + 1))
        t = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        gates.append(wl.Gate(t, wl.random_unitary(1 << k, rng)))
    return gates


def test_staged_batch_matches_oracle(env):
    """Circuits run in stages of shared-memory tiles: every tile size, re-fusion size and CTA size
    gives the oracle's states, for HEA circuits and for gates on random qubits (stages of up to
    200 gates, loaded into shared memory in several chunks)."""
    B, batch = env
    rng = np.random.default_rng(21)
    circuits = [(int(n), wl.hea_circuit(int(n), 3, rng)) for n in [16, 9, 8, 14, 12, 5, 15, 10]]
    # 200 gates: a stage of the small ones holds more gates than one shared-memory chunk
    circuits += [(int(n), _random_circuit(int(n), c, rng)) for n, c in [(13, 200), (16, 60), (11, 60), (8, 200)]]
    circuits += [(12, [])]                                   # no gate: the first stage only
    refs = [oracle.run_circuit(n, g, 0) for n, g in circuits]
    # (threads, smem_max_n, ctas, split_min_n, stage_log2, stage_k)
    configs = [(256, 0, 7, 1, 8, 0), (512, 0, 152, 8, 14, 4), (256, 9, 19, 9, 11, 2), (64, 0, 3, 10, 9, 1),
               (128, 12, 40, 13, 10, 3), (256, 0, 304, 1, 13, 4), (512, 0, 1, 8, 12, 2)]
    for max_k in (2, 4):
        b = batch.Batch(circuits, max_k)
        for threads, smem_n, ctas, split_n, sl, sk in configs:
            b.set(threads, smem_n, ctas, True, split_n, 12, 0, sl, sk)
            info = B.sv_batch_get_info(b.h)
            want = sum(1 for n, _ in circuits if n > smem_n and n >= max(split_n, 8))
            assert info["staged"] == want and info["stages"] >= want, (info, sl)
            b.arena.fill_(float("nan"))
            b.run()
            B.sv_device_status()
            for i, ref in enumerate(refs):
                got = b.state(i)
                cfg = (max_k, threads, smem_n, ctas, split_n, sl, sk, i)
                assert oracle.fidelity(ref, got) >= 1 - 1e-6, cfg
                assert oracle.l2_error(ref, got) <= 1e-4, cfg
        b.free()


_SIGN_DIAGS = [np.diag([1, 1, 1, -1]), np.diag([1, -1, -1, 1]), np.diag([-1, 1, 1, 1]), np.diag([1, -1, 1, 1]),
               np.diag([1, -1]), np.diag([-1, 1]), np.diag([-1, -1])]


def _sign_circuit(n, count, rng):
    """Dense one- and two-qubit gates mixed with +-1 diagonals on one or two qubits at every
    distance (CZ, ZZ, -|00><00|-style, Z, -Z, -I), so stages carry sign runs with pair terms of up
    to several distances, linear terms, global signs, and runs with no gate after them."""
    gates = []
    for _ in range(count):
        r = rng.random()
        if r < 0.45:
            d = _SIGN_DIAGS[int(rng.integers(0, len(_SIGN_DIAGS)))].astype(np.complex128)
            k = 1 if d.shape[0] == 2 else 2
            t = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
            gates.append(wl.Gate(t, d))
        else:
            k = int(rng.integers(1, 3))
            t = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
            gates.append(wl.Gate(t, wl.random_unitary(1 << k, rng)))
    gates += [wl.Gate((q, (q + 3) % n), np.diag([1, 1, 1, -1]).astype(np.complex128)) for q in range(n)]
    return gates


def _layer_circuit(n, layers, rng):
    """Layers of one-qubit gates and sign gates between them: a third of the layers only on qubits
    0-4 (phases of one window that outgrow one phase's record limit), the others on random subsets
    (every window, the qubits two windows share); sign gates at distances 1-5 and single-qubit
    signs."""
    gates = []
    for _ in range(layers):
        qs = range(5) if rng.random() < 0.34 else [q for q in range(n) if rng.random() < 0.7]
        for q in qs:
            gates.append(wl.Gate((int(q),), wl.random_unitary(2, rng)))
            if rng.random() < 0.3:
                gates.append(wl.Gate((int(q),), wl.random_unitary(2, rng)))
        for _ in range(int(rng.integers(1, n))):
            d = int(rng.integers(1, 6))
            a = int(rng.integers(0, n - d))
            if rng.random() < 0.8:
                gates.append(wl.Gate((a, a + d), np.diag([1, 1, 1, -1]).astype(np.complex128)))
            else:
                gates.append(wl.Gate((a,), np.diag([1, -1]).astype(np.complex128)))
    return gates


@pytest.mark.parametrize("layers", [0, 1])
def test_sign_runs_match_oracle(env, layers):
    """Circuits kept unfused (fusion size 0), so each stage re-fuses its dense gates and applies
    its +-1 diagonals as sign runs on the inputs of the next gate (or as a sweep of their own):
    HEA circuits (CZ ladders), circuits dense in sign gates and layered circuits, at every stage
    tile size, re-fusion size and CTA size, against the oracle.  With layers, runs of one-qubit
    gates and the sign runs between them go through register phases (tiles of 10 or more qubits:
    windows of five qubits in registers, sign runs formed per thread)."""
    B, batch = env
    rng = np.random.default_rng(31)
    circuits = [(int(n), wl.hea_circuit(int(n), 3, rng)) for n in [16, 9, 14, 12, 11]]
    circuits += [(int(n), _sign_circuit(int(n), c, rng)) for n, c in [(13, 150), (16, 80), (10, 200), (8, 60)]]
    circuits += [(int(n), _layer_circuit(int(n), c, rng)) for n, c in [(14, 40), (11, 30), (15, 12)]]
    circuits += [(17, wl.hea_circuit(17, 8, rng))]
    refs = [oracle.run_circuit(n, g, 0) for n, g in circuits]
    # (threads, smem_max_n, ctas, split_min_n, stage_log2, stage_k, CTAs per SM)
    configs = [(256, 0, 7, 1, 8, 0, 1), (512, 0, 152, 8, 14, 4, 1), (256, 0, 19, 8, 11, 2, 1), (128, 0, 40, 8, 10, 3, 1),
               (512, 0, 304, 1, 13, 3, 1), (256, 0, 1, 8, 12, 1, 1), (256, 0, 304, 8, 13, 2, 2), (128, 0, 60, 1, 12, 3, 2)]
    b = batch.Batch(circuits, 0)
    for threads, smem_n, ctas, split_n, sl, sk, per_sm in configs:
        b.set(threads, smem_n, ctas, True, split_n, 12, 0, sl, sk, layers, per_sm)
        info = B.sv_batch_get_info(b.h)
        assert info["staged"] == len(circuits), info
        b.arena.fill_(float("nan"))
        b.run()
        B.sv_device_status()
        for i, ref in enumerate(refs):
            got = b.state(i)
            cfg = (threads, ctas, sl, sk, layers, per_sm, i)
            assert oracle.fidelity(ref, got) >= 1 - 1e-6, cfg
            assert oracle.l2_error(ref, got) <= 1e-4, cfg
    b.free()


@pytest.mark.parametrize("layers", [0, 1])
def test_stages_relabel_qubits(env, layers):
    """The state is relabelled between stages (a tile is stored in the next stage's qubit
    layout), so no stage has to hold qubits 0-2: an 8-layer CZ-ladder circuit on 20 qubits takes
    two stages of gates on 14 local qubits and one pass that only relabels (with qubits 0-2 in
    every stage it took six); the states still equal the oracle's."""
    B, batch = env
    rng = np.random.default_rng(41)
    circuits = [(20, wl.hea_circuit(20, 8, rng)), (17, wl.hea_circuit(17, 5, rng)), (19, _layer_circuit(19, 10, rng))]
    refs = [oracle.run_circuit(n, g, 0) for n, g in circuits]
    b = batch.Batch(circuits, 0)
    b.set(512, 0, 152, True, 8, 12, 0, 14, 2, layers)
    info = B.sv_batch_get_info(b.h)
    assert info["staged"] == 3
    one = batch.Batch(circuits[:1], 0)
    one.set(512, 0, 152, True, 8, 12, 0, 14, 2, layers)
    assert B.sv_batch_get_info(one.h)["stages"] == 3
    one.free()
    for sl in (14, 12, 10):
        b.set(512, 0, 152, True, 8, 12, 0, sl, 2, layers)
        b.arena.fill_(float("nan"))
        b.run()
        B.sv_device_status()
        for i, ref in enumerate(refs):
            got = b.state(i)
            assert oracle.fidelity(ref, got) >= 1 - 1e-6, (sl, i)
            assert oracle.l2_error(ref, got) <= 1e-4, (sl, i)
    b.free()


def test_staging_cuts_traffic_and_waves_keep_results(env):
    """Stages move fewer bytes than one pass per fused gate; waves and a direct launch give the
    same states as the graph replay."""
    B, batch = env
    circuits = wl.hea_batch(count=24, n_lo=14, n_hi=18, layers=4, seed=8)
    b = batch.Batch(circuits, 2)
    b.set(256, 0, 152, True, 14, 12, 0)
    per_gate = B.sv_batch_get_info(b.h)
    b.set(256, 0, 152, True, 14, 12, 0, 14, 4)
    staged = B.sv_batch_get_info(b.h)
    assert per_gate["split"] == len(circuits) and staged["staged"] == len(circuits)
    assert staged["traffic_bytes"] < per_gate["traffic_bytes"] / 3, (staged, per_gate)
    b.run()
    first = b.arena.clone()
    b.set(512, 0, 152, False, 14, 12, 16, 13, 3)   # waves of 16 MB, no graph, other tiles
    b.arena.fill_(float("nan"))
    b.run()
    B.sv_device_status()
    for i in range(len(circuits)):
        off = B.sv_batch_state_offset(b.h, i) // 4
        nf = 2 << circuits[i][0]
        d = (first[off:off + nf] - b.arena[off:off + nf]).abs().max().item()
        assert d <= 1e-5, (i, d)
    for i in (0, 11, 23):
        n, g = circuits[i]
        assert oracle.fidelity(oracle.run_circuit(n, g, 0), b.state(i)) >= 1 - 1e-6
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


def test_split_tiles_without_graph_and_reuse(env):
    """Many split circuits interleaved step by step, launched directly (no graph), twice."""
    B, batch = env
    circuits = wl.hea_batch(count=30, n_lo=12, n_hi=18, layers=3, seed=11)
    b = batch.Batch(circuits, 3)
    b.set(256, 0, 152, False, 12, 10)
    b.run()
    first = b.arena.clone()
    b.set(512, 0, 40, False, 0, 10)       # same circuits, no split: one CTA per circuit
    b.arena.fill_(float("nan"))
    b.run()
    B.sv_device_status()
    for i in range(len(circuits)):
        off = B.sv_batch_state_offset(b.h, i) // 4
        nf = max(2 << circuits[i][0], 64)
        d = (first[off:off + nf] - b.arena[off:off + nf]).abs().max().item()
        assert d <= 1e-5, (i, d)
    for i in (0, 7, 29):
        n, g = circuits[i]
        assert oracle.fidelity(oracle.run_circuit(n, g, 0), b.state(i)) >= 1 - 1e-6
    b.free()


def test_stalled_wait_gives_up_and_is_reported(env):
    """A step counter that can never fill: every wait on it gives up after its bound, the launch
    ends without a fault, sv_device_status reports SV_ETIMEOUT, and the batch runs correctly next."""
    B, batch = env
    import torch
    rng = np.random.default_rng(2)
    circuits = [(16, wl.hea_circuit(16, 2, rng)), (10, wl.hea_circuit(10, 2, rng))]
    b = batch.Batch(circuits, 3)
    for stage_log2 in (0, 10):            # per-gate tiles, then stages
        b.set(256, 12, 8, True, 15, 10, 0, stage_log2, 2)
        if stage_log2:
            assert B.sv_batch_get_info(b.h)["stages"] >= 2
        B.sv_batch_inject_stall(b.h, True)
        b.run()
        torch.cuda.synchronize()
        with pytest.raises(B.SvError) as e:
            B.sv_device_status()
        assert e.value.code == B.SV_ETIMEOUT, stage_log2
        B.sv_device_status()              # the error word was cleared by the read
        B.sv_batch_inject_stall(b.h, False)
        b.arena.fill_(float("nan"))
        b.run()
        B.sv_device_status()
        for i, (n, g) in enumerate(circuits):
            assert oracle.fidelity(oracle.run_circuit(n, g, 0), b.state(i)) >= 1 - 1e-6
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
    h = B.sv_batch_create([f2], buf.data_ptr(), buf.numel() * 4)
    for bad in (dict(threads=1024), dict(split_min_n=25), dict(tile_log2=4), dict(tile_log2=17), dict(smem_max_n=15),
                dict(wave_mb=-1), dict(stage_log2=7), dict(stage_log2=15), dict(stage_k=5), dict(stage_k=-1),
                dict(ctas_per_sm=3), dict(ctas_per_sm=-1), dict(ctas_per_sm=2, threads=512),
                dict(ctas_per_sm=2, stage_log2=14)):
        kw = dict(threads=256, smem_max_n=12, ctas=8, use_graph=True, split_min_n=15, tile_log2=12, wave_mb=0)
        kw.update(bad)
        with pytest.raises(B.SvError) as e:
            B.sv_batch_set_opts(h, **kw)
        assert e.value.code == B.SV_EINVAL, bad
    B.sv_batch_free(h)
    B.sv_fused_free(f6)
    B.sv_fused_free(f2)


def test_autotuner_picks_a_measured_best(env, tmp_path):
    B, batch = env
    circuits = wl.hea_batch(count=24, n_lo=8, n_hi=16, layers=3, seed=4)
    best, log = batch.autotune(circuits, repeats=2, cache=str(tmp_path / "c.json"), use_cache=False, k_range=(2, 4))
    assert log and best["ms"] <= min(t["ms"] for t in log) + 1e-9
    again, log2 = batch.autotune(circuits, cache=str(tmp_path / "c.json"))
    assert again == best and log2 == []
