"""sv_init_apply (gates run on the small state of the qubits named so far, then one expansion)
gives the oracle's state: random circuits with kept controls at several sizes and fusion sizes,
prefixes that cover the whole circuit, the 3xBF16 tensor-core path, Grover, nonzero basis states,
timing records for every gate; and at 30 qubits it matches sv_init + sv_apply_fused_gates."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    return binding


def run(B, n, gates, x, timings=False, **kw):
    from paper_2602_09604_gb300.state import DeviceState
    f = B.sv_fuse_circuit(gates, n, **kw)
    st = DeviceState(n)
    rec = B.sv_init_apply(st.h, x, f, timings)
    B.sv_device_status()
    got = st.store()
    cnt = B.sv_fused_count(f)
    B.sv_fused_free(f)
    st.free()
    return got, rec, cnt


@pytest.mark.parametrize("n,max_k,prec", [(6, 2, 0), (12, 4, 0), (20, 3, 0), (26, 6, 2), (27, 5, 2)])
def test_random_circuits(B, n, max_k, prec):
    rng = np.random.default_rng(n + max_k)
    gates = []
    for _ in range(90):
        k = int(rng.integers(1, 4))
        nc = int(rng.integers(0, 4)) if rng.random() < 0.3 else 0
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    x = int(rng.integers(0, 1 << n))
    got, rec, cnt = run(B, n, gates, x, timings=True, max_k=max_k, precision=prec, tc_min_k=4)
    assert len(rec) == cnt and all(r["us"] >= 0 for r in rec)
    ref = oracle.run_circuit(n, gates, x, threads=oracle.default_threads())
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    assert oracle.l2_error(ref, got) <= 1e-4


def test_prefix_covers_the_circuit(B):
    n = 16
    rng = np.random.default_rng(3)
    gates = [wl.random_gate(n, 2, rng, targets=(1 + i % 5, 9 + i % 4)) for i in range(40)]   # 9 qubits named
    x = 0b1010011100101101
    got, _, _ = run(B, n, gates, x, max_k=4)
    ref = oracle.run_circuit(n, gates, x)
    assert np.max(np.abs(got - ref)) <= 2e-6


def test_grover_from_basis(B):
    n, marked, r = 18, 0x2B3C1, 4
    got, _, _ = run(B, n, wl.grover_circuit(n, marked, r), 0, max_k=4)
    a, b = closed_forms.grover_amplitudes(n, r)
    assert abs(got[marked] - a) <= 2e-5
    assert np.max(np.abs(np.delete(got, marked) - b)) <= 2e-6


@pytest.mark.parametrize("n,m,max_k,prec", [(12, 8, 4, 0), (20, 14, 3, 0), (26, 24, 6, 2), (27, 26, 5, 2), (28, 27, 6, 2)])
def test_light_cone_fusion(B, n, m, max_k, prec):
    """Fusion with the light cone on m qubits fused apart: sv_init_apply runs at least that part on
    its small state, and the state is the oracle's."""
    rng = np.random.default_rng(7 * n + m)
    gates = []
    for _ in range(120):
        k = int(rng.integers(1, 3))
        nc = int(rng.integers(0, 3)) if rng.random() < 0.2 else 0
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    x = int(rng.integers(0, 1 << n))
    got, rec, cnt = run(B, n, gates, x, timings=True, max_k=max_k, precision=prec, tc_min_k=4, start_qubits=m)
    small = sum(1 for r in rec if r["path"] == B.PATH_AUTO)
    # the light-cone part alone, fused the same way, is what the small state must cover
    S, closed, part = 0, 0, []
    for g in gates:
        q = sum(1 << t for t in tuple(g.targets) + tuple(g.controls))
        if not (q & closed) and bin(S | q).count("1") <= min(m, n - 1):
            S |= q
            part.append(g)
        else:
            closed |= q
    fp = B.sv_fuse_circuit(part, n, max_k=max_k, precision=prec, tc_min_k=4)
    assert small >= B.sv_fused_count(fp) > 0
    B.sv_fused_free(fp)
    ref = oracle.run_circuit(n, gates, x, threads=oracle.default_threads())
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    assert oracle.l2_error(ref, got) <= 1e-4


@pytest.mark.parametrize("prec", [1, 2])   # TF32, 3xBF16
@pytest.mark.parametrize("tg", [(3, 7, 12, 24, 25, 20), (0, 9, 14, 24, 25, 17), (8, 11, 24, 25, 19),
                                (1, 2, 24, 25), (5, 6, 7, 24, 25, 16)])
def test_first_full_gate_reads_the_small_state(B, tg, prec):
    """After a light cone on qubits 0-23 the first full-state gate is a direct tensor-core gate
    (warp-specialised k = 6 with no, one or two targets below qubit 5, k = 5, k = 4 with two low
    targets): it reads the small state in place of the zeroed full state, and its timing record
    says so.  Basis bits above the light cone are set.  The state is the oracle's."""
    n = 26
    rng = np.random.default_rng(sum(tg))
    gates = [wl.random_gate(n, 1, rng, targets=(q,)) for q in range(24)]
    gates += [wl.random_gate(n, 2, rng, targets=(q, q + 1)) for q in range(0, 23, 2)]
    gates += [wl.random_gate(n, len(tg), rng, targets=tuple(tg))]
    gates += [wl.random_gate(n, 2, rng, targets=(24, 25)), wl.random_gate(n, 2, rng, targets=(2, 13))]
    x = (1 << 24) | (1 << 25) | 0b1011
    got, rec, cnt = run(B, n, gates, x, timings=True, max_k=6, precision=prec, tc_min_k=4, start_qubits=24)
    small = sum(1 for r in rec if r["path"] == B.PATH_AUTO)
    assert 0 < small < cnt
    # the records are in fused order; the small-state gates come first there, then the gate that
    # read the small state: a tensor-core gate holding the tested gate's targets
    first_full = next(r for r in rec if r["path"] != B.PATH_AUTO)
    assert first_full["flags"] == B.TIMING_SMALL_SOURCE
    assert sum(1 for r in rec if r["flags"]) == 1
    assert first_full["path"] == (B.PATH_TC_TF32 if prec == 1 else B.PATH_TC_BF16X3)
    mask = sum(1 << q for q in tg)
    assert first_full["target_mask"] & mask == mask and first_full["k"] >= len(tg)
    ref = oracle.run_circuit(n, gates, x, threads=oracle.default_threads())
    if prec == 2:
        assert oracle.fidelity(ref, got) >= 1 - 1e-6
        assert oracle.l2_error(ref, got) <= 1e-4
    else:   # TF32: ~3e-4 relative per tensor-core gate (10-bit mantissa inputs)
        assert oracle.fidelity(ref, got) >= 1 - 1e-5
        assert oracle.l2_error(ref, got) <= 2e-3


def test_bench_circuit_matches_plain_route(B):
    """The bench's lazy route (light cone fused apart, sv_init_apply) against the plain route
    (the circuit fused as one, sv_init then sv_apply_fused_gates)."""
    import torch
    from paper_2602_09604_gb300.state import DeviceState
    n, gates = wl.circuit_30q_grid()
    f = B.sv_fuse_circuit(gates, n, max_k=6, precision=B.PREC_BF16X3, tc_min_k=4, start_qubits=28)
    st = DeviceState(n)
    B.sv_init_apply(st.h, 0, f, False)
    lazy = st.buf.clone()
    B.sv_fused_free(f)
    f = B.sv_fuse_circuit(gates, n, max_k=6, precision=B.PREC_BF16X3, tc_min_k=4)
    st.init(0)
    st.apply(f)
    B.sv_fused_free(f)
    d = torch.zeros((), dtype=torch.float64, device="cuda")
    ov = torch.zeros((), dtype=torch.float64, device="cuda")
    step = 1 << 26
    for lo in range(0, lazy.numel(), step):
        a = lazy[lo:lo + step].double()
        b = st.buf[lo:lo + step].double()
        d += ((a - b) ** 2).sum()
    assert float(d.sqrt()) <= 1e-4, float(d.sqrt())
    assert abs(st.norm() - 1.0) <= 1e-4
    st.free()
