"""CPU-only checks of the batch stage planner (sv_batch_plan_stages, host code, no kernel): the
stages apply every gate once, in an order that moves gates only past gates on other qubits (the
oracle gives the same state), each stage's gates lie on its local qubits, the layouts chain (a
stage loads in the layout the stage before stored in, the last stores in the circuit's order),
physical qubits 0-2 are local at every load and store (tiles move in 32-byte runs), and the
relabelling cuts a 20-qubit CZ-ladder circuit into two stages of gates and one relabelling pass."""
import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    from paper_2602_09604_gb300 import binding
    return binding


def _random_circuit(n, count, rng):
    gates = []
    for _ in range(count):
        k = int(rng.integers(1, 4))
        t = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        gates.append(wl.Gate(t, wl.random_unitary(1 << k, rng)))
    return gates


def _check_plan(B, gates, n, L):
    f = B.sv_fuse_circuit(gates, n, mode=B.FUSE_NONE)
    try:
        plan = B.sv_batch_plan_stages(f, L)
    finally:
        B.sv_fused_free(f)
    Lq = min(n, L)
    order = [i for st in plan for i in st["gates"]]
    assert sorted(order) == list(range(len(gates)))
    pos = {g: i for i, g in enumerate(order)}
    masks = [sum(1 << q for q in g.targets) for g in gates]
    for i in range(len(gates)):
        for j in range(i + 1, len(gates)):
            if masks[i] & masks[j]:
                assert pos[i] < pos[j], (i, j)
    full = (1 << n) - 1
    for s, st in enumerate(plan):
        lam = st["lam"]
        assert bin(lam).count("1") == Lq and lam & ~full == 0
        for i in st["gates"]:
            assert masks[i] & ~lam == 0
        lp, sp = st["load_pos"][:n], st["store_pos"][:n]
        assert sorted(lp) == list(range(n)) and sorted(sp) == list(range(n))
        local_load = {lp[q] for q in range(n) if lam >> q & 1}
        local_store = {sp[q] for q in range(n) if lam >> q & 1}
        assert {0, 1, 2} <= local_load and {0, 1, 2} <= local_store, s
        want = plan[s + 1]["load_pos"][:n] if s + 1 < len(plan) else list(range(n))
        assert sp == want, s
    # the reordered circuit is the circuit
    rng = np.random.default_rng(n * 100 + L)
    init = int(rng.integers(0, 1 << n))
    a = oracle.run_circuit(n, gates, init)
    b = oracle.run_circuit(n, [gates[i] for i in order], init)
    assert np.max(np.abs(a - b)) <= 1e-12
    return plan


@pytest.mark.parametrize("n,L", [(9, 8), (11, 8), (12, 10), (13, 9), (14, 10), (12, 12), (10, 14)])
def test_plan_random_circuits(B, n, L):
    rng = np.random.default_rng(n + 31 * L)
    for count in (1, 30, 120):
        _check_plan(B, _random_circuit(n, count, rng), n, L)


@pytest.mark.parametrize("n,L", [(12, 8), (13, 10), (14, 9)])
def test_plan_hea_and_sign_heavy_circuits(B, n, L):
    rng = np.random.default_rng(7 * n + L)
    _check_plan(B, wl.hea_circuit(n, 6, rng), n, L)
    cz = np.diag([1, 1, 1, -1]).astype(np.complex128)
    gates = []
    for _ in range(60):
        a, b = (int(q) for q in rng.choice(n, size=2, replace=False))
        gates.append(wl.Gate((a, b), cz) if rng.random() < 0.5 else wl.Gate((a,), wl.random_unitary(2, rng)))
    _check_plan(B, gates, n, L)


def test_plan_relabels_a_20_qubit_ladder_into_three_passes(B):
    rng = np.random.default_rng(41)
    n = 20
    gates = wl.hea_circuit(n, 8, rng)
    f = B.sv_fuse_circuit(gates, n, mode=B.FUSE_NONE)
    plan = B.sv_batch_plan_stages(f, 14)
    B.sv_fused_free(f)
    # the left light cone (qubits 0-13), the rest (qubits 6-19), then a pass back to the
    # circuit's qubit order
    assert [len(st["gates"]) for st in plan] == [244, 228, 0]
    assert plan[0]["lam"] == (1 << 14) - 1
    used = 0
    for i in plan[1]["gates"]:
        used |= sum(1 << q for q in gates[i].targets)
    assert used == ((1 << 20) - 1) & ~((1 << 6) - 1)
    assert plan[2]["store_pos"][:n] == list(range(n))
    order = [i for st in plan for i in st["gates"]]
    masks = [sum(1 << q for q in g.targets) for g in gates]
    pos = {g: i for i, g in enumerate(order)}
    for i in range(len(gates)):
        for j in range(i + 1, len(gates)):
            if masks[i] & masks[j]:
                assert pos[i] < pos[j]


def test_plan_rejects_bad_input(B):
    f = B.sv_fuse_circuit([], 6, mode=B.FUSE_NONE)
    with pytest.raises(B.SvError):
        B.sv_batch_plan_stages(f, 10)          # fewer than 8 qubits are never staged
    B.sv_fused_free(f)
    f = B.sv_fuse_circuit([], 12, mode=B.FUSE_NONE)
    for bad in (7, 15):
        with pytest.raises(B.SvError):
            B.sv_batch_plan_stages(f, bad)
    assert len(B.sv_batch_plan_stages(f, 10)) == 1   # no gates: one stage that builds |0...0>
    B.sv_fused_free(f)


def test_plan_refuses_post_phases_and_swap_networks(B):
    """Gates with post-phases and swap networks (SV_FUSE_PHASES) are for single states: the stage
    planner (like the batch) refuses a circuit holding them."""
    n = 12
    f = B.sv_fuse_circuit(wl.qft_circuit(n), n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
    kinds = {B.sv_fused_get_info(f, i)["path"] for i in range(B.sv_fused_count(f))}
    assert B.PATH_SWAPS in kinds
    with pytest.raises(B.SvError):
        B.sv_batch_plan_stages(f, 10)
    B.sv_fused_free(f)
