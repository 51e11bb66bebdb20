"""CPU-only checks of the C ABI library: it loads, exports every declared symbol, and its host-side
fuser is exact algebra (fused gates applied by the oracle == unfused circuit applied by the oracle).
No kernel is launched here."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    from paper_2602_09604_gb300 import binding
    return binding


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^SV_API\s+[\w\s\*]+?\b(sv_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(B):
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(B.lib, name), name


def test_required_bytes_c128_is_sixteen_per_amplitude(B):
    for n in range(5, 35):
        assert B.sv_required_bytes_c128(n) == 2 ** (n + 4)
    assert B.sv_required_bytes_c128(3) == 512 and B.sv_required_bytes_c128(0) == 0


def test_required_bytes_is_eight_per_amplitude(B):
    # the artifact appendix: an N-qubit run needs 2^(N+3) bytes
    for n in range(5, 36):
        assert B.sv_required_bytes(n) == 2 ** (n + 3)
    for n in range(1, 5):
        assert B.sv_required_bytes(n) == 256       # one whole 32-amplitude block
    assert B.sv_required_bytes(0) == 0 and B.sv_required_bytes(36) == 0


class _G:
    def __init__(self, targets, matrix, controls=()):
        self.targets, self.matrix, self.controls = targets, matrix, tuple(controls)


def fused_as_gates(B, f):
    """The fused circuit as plain gates: each fused gate, then its post-phases (a learned partition
    may be the post-phase one) as controlled phases on (target, outside qubit)."""
    out = []
    swap = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
    for i in range(B.sv_fused_count(f)):
        info = B.sv_fused_get_info(f, i)
        if info["path"] == B.PATH_SWAPS:   # a swap network (the post-phase partition makes them)
            out += [_G((a, b), swap) for a, b in B.sv_fused_get_swaps(f, i)]
            continue
        out.append(_G(info["targets"], B.sv_fused_get_matrix(f, i), info["controls"]))
        for j, q, th in B.sv_fused_get_post_phases(f, i):
            out.append(_G((info["targets"][j], q), np.diag([1, 1, 1, np.exp(1j * th)])))
    return out


def check_fusion(B, n, gates, max_k, init=0, **kw):
    f = B.sv_fuse_circuit(gates, n, max_k=max_k, **kw)
    try:
        infos = [B.sv_fused_get_info(f, i) for i in range(B.sv_fused_count(f))]
        biggest = max(len(g.targets) + len(g.controls) for g in gates)
        assert all(1 <= x["k"] <= max(max_k, biggest) or (x["k"] == 0 and x["path"] == B.PATH_SWAPS) for x in infos)
        assert sum(x["n_source_gates"] for x in infos) == len(gates)
        assert all(list(x["targets"]) == sorted(x["targets"]) for x in infos)
        ref = oracle.run_circuit(n, gates, init)
        got = oracle.run_circuit(n, fused_as_gates(B, f), init)
        assert np.max(np.abs(ref - got)) < 1e-12
        return infos
    finally:
        B.sv_fused_free(f)


@pytest.mark.parametrize("max_k", [1, 2, 3, 4, 5, 6])
def test_fusion_is_exact_on_grid_circuit(B, max_k):
    n, gates = wl.GRID_16.n, wl.random_grid_circuit(wl.Grid(3, 4), 6, seed=3)
    n = 12
    infos = check_fusion(B, n, gates, max_k)
    if max_k >= 2:
        assert len(infos) < len(gates)


@pytest.mark.parametrize("max_k,m", [(2, 4), (4, 6), (6, 8), (3, 24), (5, 28)])
def test_light_cone_split_is_exact_and_first(B, max_k, m):
    """start_qubits = m: the fused circuit is still exact, and its first fused gates name at most
    min(m, n - 1) qubits together and commute past every later gate they overtake (so a start
    from a basis state can run them on a small state)."""
    rng = np.random.default_rng(40 + m)
    n = 10
    gates = []
    for _ in range(60):
        k = int(rng.integers(1, 3))
        qs = [int(q) for q in rng.permutation(n)]
        nc = 1 if rng.random() < 0.15 else 0
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    infos = check_fusion(B, n, gates, max_k, init=5, start_qubits=m)
    lim = min(m, n - 1)
    plain = check_fusion(B, n, gates, max_k, init=5)
    # the light-cone part of the input gates (the fuser's rule), fused alone
    S, closed, part = 0, 0, []
    for g in gates:
        q = sum(1 << t for t in tuple(g.targets) + tuple(g.controls))
        if not (q & closed) and bin(S | q).count("1") <= lim:
            S |= q
            part.append(g)
        else:
            closed |= q
    fp = B.sv_fuse_circuit(part, n, max_k=max_k)
    head = [B.sv_fused_get_info(fp, i) for i in range(B.sv_fused_count(fp))]
    B.sv_fused_free(fp)
    assert [x["targets"] for x in infos[:len(head)]] == [x["targets"] for x in head]
    named = 0
    for x in head:
        for q in tuple(x["targets"]) + tuple(x["controls"]):
            named |= 1 << q
    assert named & ~S == 0 and bin(named).count("1") <= lim
    assert sum(x["n_source_gates"] for x in infos) == sum(x["n_source_gates"] for x in plain) == len(gates)


def test_light_cone_option_validated(B):
    U = wl.random_unitary(2, np.random.default_rng(1))
    for bad in (-1, 29):
        with pytest.raises(B.SvError) as e:
            B.sv_fuse_circuit([wl.Gate((0,), U)], 4, start_qubits=bad)
        assert e.value.code == B.SV_EINVAL


@pytest.mark.parametrize("max_k", [2, 4, 6])
def test_fusion_with_controls_and_random_gates(B, max_k):
    rng = np.random.default_rng(5)
    n = 9
    gates = []
    for _ in range(40):
        k = int(rng.integers(1, 4))
        qs = [int(q) for q in rng.permutation(n)]
        nc = int(rng.integers(0, 3)) if k + 2 <= max(max_k, 3) else 0
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    check_fusion(B, n, gates, max_k, init=77)


@pytest.mark.parametrize("max_k", [1, 2, 4, 6])
def test_fusion_with_many_controls(B, max_k):
    # gates with up to 7 controls: folded where k + controls fits max_k, kept controlled (a fusion
    # barrier on every qubit they name) otherwise; the result is exact either way
    rng = np.random.default_rng(11 + max_k)
    n = 10
    gates = []
    for _ in range(60):
        k = int(rng.integers(1, 4))
        nc = int(rng.integers(0, 8)) if rng.random() < 0.6 else 0
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    infos = check_fusion(B, n, gates, max_k, init=333)
    kept = [g for g in gates if g.controls and len(g.targets) + len(g.controls) > max_k]
    ctrl = [x for x in infos if x["path"] == B.PATH_CONTROLLED]
    assert len(ctrl) == len(kept)
    assert all(x["n_source_gates"] == 1 and x["controls"] for x in ctrl)
    assert all(not x["controls"] for x in infos if x["path"] != B.PATH_CONTROLLED)


def test_controlled_gate_limits(B):
    rng = np.random.default_rng(4)
    n = 9
    big = wl.Gate((0, 1, 2, 3), wl.random_unitary(16, rng), (5, 6, 7))     # 4 targets + 3 controls
    with pytest.raises(B.SvError) as e:
        B.sv_fuse_circuit([big], n, max_k=4)
    assert e.value.code == B.SV_EINVAL
    fold = wl.Gate((0, 1, 2, 3), wl.random_unitary(16, rng), (5, 6))     # folds into 6 qubits
    f = B.sv_fuse_circuit([fold], n, max_k=4)
    try:
        info = B.sv_fused_get_info(f, 0)
        assert info["k"] == 6 and info["path"] != B.PATH_CONTROLLED
    finally:
        B.sv_fused_free(f)


@pytest.mark.parametrize("max_k", [2, 4, 6])
def test_grover_and_qv_fuse_exactly(B, max_k):
    n = 9
    infos = check_fusion(B, n, wl.grover_circuit(n, 300, 3), max_k, init=0)
    mcz = [x for x in infos if x["path"] == B.PATH_CONTROLLED]
    assert len(mcz) == 6 and all(x["targets"] == (8,) and x["controls"] == tuple(range(8)) for x in mcz)
    check_fusion(B, 8, wl.qv_circuit(8, seed=1), max_k, init=5)


def test_fusion_of_textbook_circuits(B):
    check_fusion(B, 10, wl.qft_circuit(10), 4, init=345)
    check_fusion(B, 11, wl.ghz_circuit(11, controlled=True), 3)
    rng = np.random.default_rng(1)
    check_fusion(B, 8, wl.hea_circuit(8, 3, rng), 5)


def test_vertical_fusion_collapses_same_qubit_gates(B):
    gates = [wl.Gate((2,), wl.H), wl.Gate((2,), wl.SQRT_X), wl.Gate((2,), wl.H)]
    f = B.sv_fuse_circuit(gates, 4, max_k=1)
    try:
        assert B.sv_fused_count(f) == 1
        assert np.allclose(B.sv_fused_get_matrix(f, 0), wl.H @ wl.SQRT_X @ wl.H, atol=1e-15)
    finally:
        B.sv_fused_free(f)


def test_horizontal_fusion_is_tensor_product(B):
    # Eq. 4: gates on disjoint qubits fuse to U1 (x) U2; local bit 0 <-> lower qubit
    rng = np.random.default_rng(8)
    U1, U2 = wl.random_unitary(2, rng), wl.random_unitary(2, rng)
    f = B.sv_fuse_circuit([wl.Gate((1,), U1), wl.Gate((4,), U2)], 6, max_k=2)
    try:
        assert B.sv_fused_count(f) == 1
        assert B.sv_fused_get_info(f, 0)["targets"] == (1, 4)
        assert np.allclose(B.sv_fused_get_matrix(f, 0), np.kron(U2, U1), atol=1e-15)
    finally:
        B.sv_fused_free(f)


def test_path_classification(B):
    rng = np.random.default_rng(2)
    cases = {(0, 3): B.PATH_LOW, (5, 9): B.PATH_HIGH, (2, 7): B.PATH_MIXED, (4,): B.PATH_LOW, (5,): B.PATH_HIGH}
    for t, path in cases.items():
        f = B.sv_fuse_circuit([wl.Gate(t, wl.random_unitary(1 << len(t), rng))], 12, max_k=2)
        try:
            assert B.sv_fused_get_info(f, 0)["path"] == path
        finally:
            B.sv_fused_free(f)


def test_fuser_rejects_bad_input(B):
    rng = np.random.default_rng(4)
    U = wl.random_unitary(2, rng)
    bad = [
        ([wl.Gate((7,), U)], 5, B.SV_EINVAL),                       # qubit out of range
        ([wl.Gate((1, 1), np.eye(4))], 5, B.SV_EINVAL),             # repeated qubit
        ([wl.Gate((0,), U, (0,))], 5, B.SV_EINVAL),                  # control == target
        ([wl.Gate((0,), 1.1 * U)], 5, B.SV_EUNITARY),               # not unitary
        ([wl.Gate(tuple(range(7)), np.eye(128))], 8, B.SV_EINVAL),  # k > 6
        ([wl.Gate((0, 1, 2, 3, 4), np.eye(32), (5, 6))], 8, B.SV_EINVAL),  # k + controls > 6
    ]
    for gates, n, code in bad:
        with pytest.raises(B.SvError) as e:
            B.sv_fuse_circuit(gates, n, max_k=4)
        assert e.value.code == code
    with pytest.raises(B.SvError):
        B.sv_fuse_circuit([wl.Gate((0,), U)], 0)
    with pytest.raises(B.SvError):
        B.sv_fuse_circuit([wl.Gate((0,), U)], 4, max_k=7)


def test_empty_circuit_fuses_to_nothing(B):
    f = B.sv_fuse_circuit([], 5)
    try:
        assert B.sv_fused_count(f) == 0
    finally:
        B.sv_fused_free(f)


def test_no_fusion_mode_keeps_every_gate(B):
    rng = np.random.default_rng(6)
    n = 7
    gates = [wl.Gate((3, 1), wl.random_unitary(4, rng)), wl.Gate((3, 1), wl.random_unitary(4, rng)),
             wl.Gate((0,), wl.X, (5,))]
    f = B.sv_fuse_circuit(gates, n, mode=B.FUSE_NONE)
    try:
        assert B.sv_fused_count(f) == 3
        assert [B.sv_fused_get_info(f, i)["targets"] for i in range(3)] == [(1, 3), (1, 3), (0, 5)]
        got = oracle.run_circuit(n, fused_as_gates(B, f), 9)
        assert np.max(np.abs(got - oracle.run_circuit(n, gates, 9))) < 1e-13
    finally:
        B.sv_fused_free(f)


# ---------------------------------------------------------------------- learned partition search
def _random_cost(seed):
    """A deterministic but arbitrary cost per (k, targets, path): whatever candidate or merge the
    search then prefers, the fused circuit must stay exact."""
    def cost(k, targets, path, n):
        h = hash((k, tuple(targets), path, n, seed)) & 0xFFFF
        return 1.0 + h / 65536.0 * (1 + k)
    return cost


def _pass_cost(B):
    """One unit per pass over the state; CUDA-core gates of 4+ qubits are arithmetic-bound (slower)."""
    def cost(k, targets, path, n):
        if path in (B.PATH_TC_BF16X3, B.PATH_TC_TF32):
            return 1.0 + 0.4 * (sum(1 for t in targets if t < 5) >= 3)
        return max(1.0, (8 * 2 ** k - 2) / 60.0)
    return cost


def _random_controlled_circuit(n, count, rng):
    gates = []
    for _ in range(count):
        k = int(rng.integers(1, 3))
        qs = [int(q) for q in rng.permutation(n)]
        nc = 1 if rng.random() < 0.1 else 0
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    return gates


@pytest.mark.parametrize("max_k,seed,start", [(3, 1, 0), (4, 2, 0), (5, 3, 6), (6, 4, 0), (6, 5, 8), (4, 6, 5)])
def test_learned_search_is_exact(B, max_k, seed, start):
    """The learned search (greedy candidates under every closing rule, then cost-guided merging)
    with a caller's cost function: exact algebra whatever the costs prefer, with kept controlled
    gates and with the light-cone split."""
    rng = np.random.default_rng(seed)
    n = 10
    gates = _random_controlled_circuit(n, 70, rng)
    for cost in (_random_cost(seed), _pass_cost(B)):
        check_fusion(B, n, gates, max_k, init=3, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4,
                     cost_fn=cost, start_qubits=start)


def _fused_cost(B, f, n, cost):
    tot = 0.0
    for i in range(B.sv_fused_count(f)):
        info = B.sv_fused_get_info(f, i)
        if info["controls"]:
            continue
        tot += cost(info["k"], info["targets"], info["path"], n)
    return tot


@pytest.mark.parametrize("name", ["grid", "qft", "qv", "random"])
def test_learned_search_is_never_worse_than_greedy(B, name):
    """Scored by the same cost function, the learned partition costs no more than greedy fusion at
    any max size (greedy partitions are among its candidates), and its kernel paths are the
    cheapest the cost function allows."""
    rng = np.random.default_rng(11)
    n, gates = {"grid": (12, wl.random_grid_circuit(wl.Grid(3, 4), 8, seed=3)), "qft": (12, wl.qft_circuit(12)),
                "qv": (12, wl.qv_circuit(12, seed=2)), "random": (12, _random_controlled_circuit(12, 120, rng))}[name]
    cost = _pass_cost(B)
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4, cost_fn=cost)
    learned = _fused_cost(B, f, n, cost)
    for i in range(B.sv_fused_count(f)):
        info = B.sv_fused_get_info(f, i)
        if info["controls"]:
            continue
        alt = [B.PATH_TC_BF16X3] if info["k"] >= 4 else []
        assert cost(info["k"], info["targets"], info["path"], n) <= min(
            [cost(info["k"], info["targets"], p, n) for p in alt] + [cost(info["k"], info["targets"], info["path"], n)])
    B.sv_fused_free(f)
    for k in range(2, 7):
        g = B.sv_fuse_circuit(gates, n, max_k=k, precision=B.PREC_BF16X3, tc_min_k=4)
        greedy = _fused_cost(B, g, n, lambda kk, t, p, nn: min(cost(kk, t, p, nn), cost(kk, t, B.PATH_TC_BF16X3, nn))
                             if kk >= 4 else cost(kk, t, p, nn))
        B.sv_fused_free(g)
        assert learned <= greedy + 1e-9, (k, learned, greedy)


def test_learned_search_rejects_a_bad_cost(B):
    n, gates = 8, wl.qft_circuit(8)
    with pytest.raises(B.SvError):
        B.sv_fuse_circuit(gates, n, max_k=4, mode=B.FUSE_LEARNED, cost_fn=lambda k, t, p, nn: -1.0)


def test_learned_search_scores_smaller_light_cones(B):
    """With a light-cone split the learned search also scores smaller light cones (their gates costed
    on the smaller start state).  A cost that makes small-state gates dear drives it to the smallest
    one tried, a cost that makes them cheap keeps the largest; both stay exact."""
    rng = np.random.default_rng(23)
    n = 10
    gates = _random_controlled_circuit(n, 80, rng)
    dear = lambda k, t, p, nn: 1.0 if nn == n else 1e3       # small-state gates dear
    cheap = lambda k, t, p, nn: 2.0 ** nn                      # proportional to the state size
    counts = {}
    for name, cost in (("dear", dear), ("cheap", cheap)):
        infos = check_fusion(B, n, gates, 4, init=5, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4,
                             cost_fn=cost, start_qubits=8)
        counts[name] = infos
    # the light-cone part comes first: count the leading fused gates whose qubits stay within a set
    # of at most m qubits, m = 8 (cheap) or 4 (dear: the smallest of 8 - 1 .. 8 - 4)
    def lead(infos, m):
        S, c = 0, 0
        for x in infos:
            q = sum(1 << t for t in x["targets"]) | sum(1 << t for t in x["controls"])
            if bin(S | q).count("1") > m:
                break
            S |= q
            c += 1
        return c
    assert lead(counts["dear"], 4) >= 1
    assert lead(counts["cheap"], 8) >= lead(counts["dear"], 8)


def _diagonal_mix(n, count, rng):
    """Dense gates mixed with diagonal ones (RZ, CZ, controlled phases, a phase on three qubits,
    and some kept as controlled gates), so diagonal gates move past each other."""
    gates = []
    for _ in range(count):
        r = rng.random()
        qs = [int(q) for q in rng.permutation(n)]
        if r < 0.2:
            gates.append(wl.Gate((qs[0],), wl.rz(float(rng.uniform(0, 6.3)))))
        elif r < 0.35:
            gates.append(wl.Gate((qs[0], qs[1]), wl.CZ))
        elif r < 0.5:
            gates.append(wl.Gate((qs[0], qs[1]), wl.cphase(float(rng.uniform(0, 6.3)))))
        elif r < 0.55:
            gates.append(wl.Gate((qs[0], qs[1], qs[2]), np.diag(np.exp(1j * rng.uniform(0, 6.3, 8)))))
        elif r < 0.6:
            gates.append(wl.Gate((qs[0],), wl.Z, (qs[1], qs[2])))      # controlled: kept or folded
        else:
            k = int(rng.integers(1, 3))
            gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng)))
    return gates


@pytest.mark.parametrize("name,max_k,start", [("qft", 6, 0), ("qft", 4, 7), ("mix", 6, 0), ("mix", 3, 0), ("mix", 5, 8)])
def test_learned_search_defers_diagonals_exactly(B, name, max_k, start):
    """Learned mode also tries the equivalent order with diagonal gates moved later (to just before
    the next non-diagonal gate on one of their qubits): the fused circuit stays exact, and scored by
    the same cost it has no more passes than greedy fusion at max_k."""
    n = 10
    gates = wl.qft_circuit(n) if name == "qft" else _diagonal_mix(n, 90, np.random.default_rng(max_k + start))
    cost = lambda k, t, p, nn: 2.0 ** nn
    infos = check_fusion(B, n, gates, max_k, init=37, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, tc_min_k=4,
                         cost_fn=cost, start_qubits=start)
    if start == 0:
        g = B.sv_fuse_circuit(gates, n, max_k=max_k, precision=B.PREC_BF16X3, tc_min_k=4)
        assert len(infos) <= B.sv_fused_count(g)
        B.sv_fused_free(g)
