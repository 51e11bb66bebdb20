"""CPU-only checks of post-phase fusion (SV_FUSE_PHASES, host code): the fused gates followed by
their post-phases (applied here with numpy: amplitude i times exp(i theta) for each term whose two
bits are set in i) give the oracle's state for the QFT and for circuits dense in diagonal gates;
the QFT's controlled-phase ladders collapse into six-qubit gates; each input gate is counted once;
bad options are refused; the learned search scores the post-phase partition (with the post-phase
feature and cost flag) and takes it only when it is predicted cheaper."""
import math

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


SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def apply_fused_with_phases(B, f, n, psi):
    idx = np.arange(1 << n)
    for i in range(B.sv_fused_count(f)):
        info = B.sv_fused_get_info(f, i)
        if info["path"] == B.PATH_SWAPS:   # a swap network: its swaps, one by one
            assert info["k"] == 0 and not B.sv_fused_get_post_phases(f, i)
            for a, b in B.sv_fused_get_swaps(f, i):
                oracle.apply_gate(psi, n, wl.Gate((a, b), SWAP))
            continue
        assert not B.sv_fused_get_swaps(f, i)
        oracle.apply_gate(psi, n, wl.Gate(info["targets"], B.sv_fused_get_matrix(f, i)))
        post = B.sv_fused_get_post_phases(f, i)
        if post:
            ph = np.zeros(1 << n)
            for j, q, th in post:
                assert q not in info["targets"]
                ph += th * (((idx >> info["targets"][j]) & 1) & ((idx >> q) & 1))
            psi *= np.exp(1j * ph)
    return psi


def _diag_circuit(n, count, rng):
    gates = []
    for _ in range(count):
        r = rng.random()
        a, b = (int(q) for q in rng.choice(n, size=2, replace=False))
        if r < 0.3:
            gates.append(wl.Gate((a, b), np.diag(np.exp(1j * rng.uniform(0, 2 * math.pi, 4)))))   # any diagonal
        elif r < 0.45:
            gates.append(wl.Gate((a, b), wl.cphase(rng.uniform(0, 2 * math.pi))))
        elif r < 0.55:
            gates.append(wl.Gate((a,), np.diag(np.exp(1j * rng.uniform(0, 2 * math.pi, 2)))))
        elif r < 0.85:
            gates.append(wl.Gate((a,), wl.random_unitary(2, rng)))
        else:
            gates.append(wl.Gate((a, b), wl.random_unitary(4, rng)))
    return gates


@pytest.mark.parametrize("n", [12, 14, 16])
def test_qft_phase_fusion_is_exact_and_short(B, n):
    gates = wl.qft_circuit(n)
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
    init = (0x5a5a5 * n) % (1 << n)
    psi = np.zeros(1 << n, complex)
    psi[init] = 1.0
    got = apply_fused_with_phases(B, f, n, psi)
    ref = oracle.run_circuit(n, gates, init)
    assert np.max(np.abs(got - ref)) <= 1e-12
    # one pass per six qubits of H + phase ladders, then the swap network
    count = B.sv_fused_count(f)
    assert count <= math.ceil(n / 6) + math.ceil(n / 2 / 3) + 1, count
    assert sum(len(B.sv_fused_get_post_phases(f, i)) for i in range(count)) > 0
    # every input gate is counted once (split-off factors and leftover phases count nowhere)
    assert sum(B.sv_fused_get_info(f, i)["n_source_gates"] for i in range(count)) == len(gates)
    B.sv_fused_free(f)


@pytest.mark.parametrize("n,seed", [(11, 1), (13, 2), (15, 3)])
def test_diagonal_heavy_phase_fusion_is_exact(B, n, seed):
    rng = np.random.default_rng(seed)
    gates = _diag_circuit(n, 160, rng)
    for prec in (B.PREC_BF16X3, B.PREC_TF32):
        f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=prec)
        init = int(rng.integers(0, 1 << n))
        psi = np.zeros(1 << n, complex)
        psi[init] = 1.0
        got = apply_fused_with_phases(B, f, n, psi)
        ref = oracle.run_circuit(n, gates, init)
        assert np.max(np.abs(got - ref)) <= 1e-11
        assert sum(B.sv_fused_get_info(f, i)["n_source_gates"] for i in range(B.sv_fused_count(f))) == len(gates)
        for i in range(B.sv_fused_count(f)):   # only tensor-core six-qubit gates carry phases
            if B.sv_fused_get_post_phases(f, i):
                info = B.sv_fused_get_info(f, i)
                assert info["k"] == 6 and info["path"] in (B.PATH_TC_TF32, B.PATH_TC_BF16X3)
                assert sum(t < 5 for t in info["targets"]) <= 2
        B.sv_fused_free(f)


def test_phase_mode_refuses_bad_options(B):
    gates = wl.qft_circuit(10)
    for kw in (dict(precision=B.PREC_FP32), dict(precision=B.PREC_BF16X3, start_qubits=6)):
        with pytest.raises(B.SvError):
            B.sv_fuse_circuit(gates, 10, max_k=6, mode=B.FUSE_PHASES, **kw)


def test_post_phases_feature_and_flag(B):
    t = (3, 7, 9, 12, 15, 20)
    plain = B.sv_mlp_features(6, t, B.PATH_TC_BF16X3, 24)
    post = B.sv_mlp_features(6, t, B.PATH_TC_BF16X3, 24, post_phases=True)
    assert plain[15] == 0.0 and post[15] == 1.0
    assert np.array_equal(plain[:15], post[:15])
    assert B.sv_mlp_features(6, (0, 1, 2, 3, 4, 9), B.PATH_TC_BF16X3, 24)[13] == 1.0   # five low targets


def test_post_gate_timing_circuit_fuses_one_to_one(B):
    from paper_2602_09604_gb300.timing_sweep import fuse_post_gates, random_post_targets
    rng = np.random.default_rng(4)
    for n in (24, 28, 32):
        sets = [random_post_targets(n, rng) for _ in range(5)]
        for t in sets:
            assert len(t) == 6 and sum(q < 5 for q in t) <= 2 and not {0, 1} <= set(t)
        f = fuse_post_gates(n, sets, 3, rng)
        assert B.sv_fused_count(f) == 15
        assert [B.sv_fused_get_info(f, i)["targets"] for i in range(15)] == [t for t in sets for _ in range(3)]
        B.sv_fused_free(f)


def _learned(B, gates, n, post_factor, seen=None):
    def cost(k, targets, path, nq):
        if seen is not None:
            seen.append(path)
        c = 2.0 ** nq * (1.0 if (path & ~B.PATH_POST_PHASES) in (B.PATH_TC_TF32, B.PATH_TC_BF16X3) else 3.0)
        return c * (post_factor if path & B.PATH_POST_PHASES else 1.0)
    return B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4,
                             cost_fn=cost)


@pytest.mark.parametrize("n", [12, 15])
def test_learned_search_scores_the_phase_partition(B, n):
    """The learned search takes the post-phase partition when the cost says it is cheaper (the
    QFT: a few six-qubit passes against many), and not when gates with post-phases cost too much;
    either way the fused circuit is the circuit."""
    gates = wl.qft_circuit(n)
    fp = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3, tc_min_k=4)
    n_phase = B.sv_fused_count(fp)
    B.sv_fused_free(fp)
    init = (0x3c3c3 * n) % (1 << n)
    ref = oracle.run_circuit(n, gates, init)
    seen = []
    for factor, expect_post in ((1.2, True), (1e4, False)):
        f = _learned(B, gates, n, factor, seen)
        count = B.sv_fused_count(f)
        n_post = sum(len(B.sv_fused_get_post_phases(f, i)) for i in range(count))
        assert (n_post > 0) == expect_post, (factor, n_post)
        if expect_post:
            assert count == n_phase
        psi = np.zeros(1 << n, complex)
        psi[init] = 1.0
        got = apply_fused_with_phases(B, f, n, psi)
        assert np.max(np.abs(got - ref)) <= 1e-12
        B.sv_fused_free(f)
    # gates with post-phases reach the cost function with the flag, on a tensor-core path
    flagged = [p for p in seen if p & B.PATH_POST_PHASES]
    assert flagged and all(p & ~B.PATH_POST_PHASES == B.PATH_TC_BF16X3 for p in flagged)


def test_learned_search_without_diagonal_pairs_has_no_post_phases(B):
    rng = np.random.default_rng(9)
    n = 12
    gates = [wl.Gate(tuple(int(q) for q in rng.choice(n, size=2, replace=False)), wl.random_unitary(4, rng))
             for _ in range(60)]
    f = _learned(B, gates, n, 0.5)   # post-phases made cheap: still none to make
    assert all(not B.sv_fused_get_post_phases(f, i) for i in range(B.sv_fused_count(f)))
    B.sv_fused_free(f)


def test_qft_swap_network_is_one_gate(B):
    for n in (12, 15):
        f = B.sv_fuse_circuit(wl.qft_circuit(n), n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
        nets = [i for i in range(B.sv_fused_count(f)) if B.sv_fused_get_info(f, i)["path"] == B.PATH_SWAPS]
        assert nets == [B.sv_fused_count(f) - 1]
        assert sorted(B.sv_fused_get_swaps(f, nets[0])) == [(q, n - 1 - q) for q in range(n // 2)]
        assert B.sv_fused_get_info(f, nets[0])["n_source_gates"] == n // 2
        with pytest.raises(B.SvError):
            B.sv_fused_get_matrix(f, nets[0])
        B.sv_fused_free(f)


def test_short_or_overlapping_swap_runs_stay_ordinary_gates(B):
    n = 12
    for pairs in ([(0, 7), (3, 9)], [(0, 1), (1, 2), (2, 3)], [(4, 5), (6, 7), (5, 8)]):
        gates = [wl.Gate(p, SWAP) for p in pairs]
        f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
        assert all(B.sv_fused_get_info(f, i)["path"] != B.PATH_SWAPS for i in range(B.sv_fused_count(f)))
        B.sv_fused_free(f)
    # fewer than 10 qubits: no swap networks at all
    f = B.sv_fuse_circuit([wl.Gate((q, 8 - q), SWAP) for q in range(4)], 9, max_k=6, mode=B.FUSE_PHASES,
                          precision=B.PREC_BF16X3)
    assert all(B.sv_fused_get_info(f, i)["path"] != B.PATH_SWAPS for i in range(B.sv_fused_count(f)))
    B.sv_fused_free(f)


@pytest.mark.parametrize("n,seed", [(10, 4), (12, 5), (14, 6)])
def test_swap_runs_among_other_gates_are_exact(B, n, seed):
    """Runs of disjoint swaps between dense, diagonal and controlled-phase gates: the swap network
    is placed after everything before it on its qubits and before everything after it there."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(8):
        gates += _diag_circuit(n, 25, rng)
        qs = [int(q) for q in rng.permutation(n)]
        gates += [wl.Gate((qs[2 * i], qs[2 * i + 1]), SWAP) for i in range(int(rng.integers(3, n // 2 + 1)))]
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
    count = B.sv_fused_count(f)
    assert sum(B.sv_fused_get_info(f, i)["path"] == B.PATH_SWAPS for i in range(count)) >= 4
    assert sum(B.sv_fused_get_info(f, i)["n_source_gates"] for i in range(count)) == len(gates)
    init = int(rng.integers(0, 1 << n))
    psi = np.zeros(1 << n, complex)
    psi[init] = 1.0
    got = apply_fused_with_phases(B, f, n, psi)
    assert np.max(np.abs(got - oracle.run_circuit(n, gates, init))) <= 1e-11
    B.sv_fused_free(f)


@pytest.mark.parametrize("seed", [11, 12])
def test_phase_partition_with_kept_controls_and_swaps_is_exact(B, seed):
    """Kept controlled gates (more controls than the fusion size allows folding), diagonal pairs,
    dense gates and swap runs in one circuit: the post-phase partition, and the learned search
    with it among its candidates, give the oracle's state."""
    rng = np.random.default_rng(seed)
    n = 10
    gates = []
    for _ in range(4):
        gates += _diag_circuit(n, 20, rng)
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(wl.Gate((qs[0],), wl.random_unitary(2, rng), tuple(qs[1:8])))   # 7 controls: kept
        qs = [int(q) for q in rng.permutation(n)]
        gates += [wl.Gate((qs[2 * i], qs[2 * i + 1]), SWAP) for i in range(4)]
    init = int(rng.integers(0, 1 << n))
    ref = oracle.run_circuit(n, gates, init)
    for f in (B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3),
              _learned(B, gates, n, 1.1)):
        count = B.sv_fused_count(f)
        infos = [B.sv_fused_get_info(f, i) for i in range(count)]
        assert sum(i["path"] == B.PATH_CONTROLLED for i in infos) == 4
        assert sum(i["n_source_gates"] for i in infos) == len(gates)
        psi = np.zeros(1 << n, complex)
        psi[init] = 1.0
        # apply gate by gate: controlled gates through the oracle with their controls
        idx = np.arange(1 << n)
        for i, info in enumerate(infos):
            if info["path"] == B.PATH_SWAPS:
                for a, b in B.sv_fused_get_swaps(f, i):
                    oracle.apply_gate(psi, n, wl.Gate((a, b), SWAP))
                continue
            oracle.apply_gate(psi, n, wl.Gate(info["targets"], B.sv_fused_get_matrix(f, i), info["controls"]))
            post = B.sv_fused_get_post_phases(f, i)
            if post:
                ph = np.zeros(1 << n)
                for j, q, th in post:
                    ph += th * (((idx >> info["targets"][j]) & 1) & ((idx >> q) & 1))
                psi *= np.exp(1j * ph)
        got = psi
        assert np.max(np.abs(got - ref)) <= 1e-11
        B.sv_fused_free(f)


def test_phase_mode_below_six_qubits_has_swaps_but_no_post_terms(B):
    """With max_k below 6 no fused gate can carry post terms (their kernel is the six-qubit one),
    but swap runs still become swap networks; the circuit stays exact."""
    n = 11
    gates = wl.qft_circuit(n)
    f = B.sv_fuse_circuit(gates, n, max_k=4, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
    count = B.sv_fused_count(f)
    assert all(not B.sv_fused_get_post_phases(f, i) for i in range(count))
    assert sum(B.sv_fused_get_info(f, i)["path"] == B.PATH_SWAPS for i in range(count)) == 1
    psi = np.zeros(1 << n, complex)
    psi[77] = 1.0
    got = apply_fused_with_phases(B, f, n, psi)
    assert np.max(np.abs(got - oracle.run_circuit(n, gates, 77))) <= 1e-12
    B.sv_fused_free(f)


def test_phase_partition_exact_on_random_circuits_property(B):
    """Property check over many random circuits (hypothesis draws the seed, the size and the gate
    mix): the post-phase partition with post terms and swap networks is the circuit."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2**31 - 1), n=st.integers(10, 11), count=st.integers(1, 90),
               swap_every=st.integers(0, 4))
    def check(seed, n, count, swap_every):
        rng = np.random.default_rng(seed)
        gates = []
        for r in range(count):
            gates += _diag_circuit(n, 1, rng)
            if swap_every and r % (swap_every * 7) == 0:
                qs = [int(q) for q in rng.permutation(n)]
                gates += [wl.Gate((qs[2 * i], qs[2 * i + 1]), SWAP) for i in range(int(rng.integers(1, n // 2 + 1)))]
        f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3)
        try:
            infos = [B.sv_fused_get_info(f, i) for i in range(B.sv_fused_count(f))]
            assert sum(i["n_source_gates"] for i in infos) == len(gates)
            init = int(rng.integers(0, 1 << n))
            psi = np.zeros(1 << n, complex)
            psi[init] = 1.0
            got = apply_fused_with_phases(B, f, n, psi)
            assert np.max(np.abs(got - oracle.run_circuit(n, gates, init))) <= 1e-11
        finally:
            B.sv_fused_free(f)

    check()


def test_learned_search_exact_under_random_costs_property(B):
    """Whatever the cost function says (hypothesis draws the circuit and a random cost table), the
    partition the learned search returns, post-phase candidate included, is the circuit."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=25, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2**31 - 1), post_factor=st.floats(0.2, 3.0))
    def check(seed, post_factor):
        rng = np.random.default_rng(seed)
        n = 10
        gates = wl.qft_circuit(n) if rng.random() < 0.3 else _diag_circuit(n, 60, rng)
        salt = int(rng.integers(1, 1 << 30))

        def cost(k, targets, path, nq):
            h = (hash((k, tuple(targets), path & ~B.PATH_POST_PHASES, nq, salt)) % 1000) / 1000.0
            c = 2.0 ** nq * (0.5 + h)
            return c * (post_factor if path & B.PATH_POST_PHASES else 1.0)
        f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4,
                              cost_fn=cost)
        try:
            init = int(rng.integers(0, 1 << n))
            psi = np.zeros(1 << n, complex)
            psi[init] = 1.0
            got = apply_fused_with_phases(B, f, n, psi)
            assert np.max(np.abs(got - oracle.run_circuit(n, gates, init))) <= 1e-11
        finally:
            B.sv_fused_free(f)

    check()
