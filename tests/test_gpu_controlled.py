"""Controlled gates kept whole (SV_PATH_CONTROLLED: only amplitudes whose control bits are 1 are
touched) against the oracle: single gates with every placement of targets and controls (inside
and outside the 32-amplitude block), random circuits mixing many-control gates with fused and
tensor-core gates, Grover at 20 qubits against its closed form and with learned fusion, Grover at
30 qubits (full size) against the closed form, and quantum volume against the oracle."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2602_09604_gb300",
                     "cost_model_gb300.bin")


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    return binding


def run_gpu(B, n, gates, init=0, **kw):
    from paper_2602_09604_gb300.state import DeviceState
    f = B.sv_fuse_circuit(gates, n, **kw)
    paths = [B.sv_fused_get_info(f, i)["path"] for i in range(B.sv_fused_count(f))]
    st = DeviceState(n)
    st.init(init)
    st.apply(f)
    B.sv_device_status()
    psi = st.store()
    st.free()
    B.sv_fused_free(f)
    return psi, paths


def test_single_controlled_gates_every_placement(B):
    n = 14
    rng = np.random.default_rng(21)
    cases = [((3,), (0,)), ((0,), (13,)), ((9,), (2, 4)), ((1, 6), (0, 12, 3)), ((2, 3, 4), (0, 1)),
             ((7, 11, 13), (5, 6, 8, 9, 10)), ((4,), tuple(q for q in range(n) if q != 4)),
             ((0, 1), tuple(range(2, 14)))]
    psi0 = wl.random_state(n, rng)
    for targets, controls in cases:
        g = wl.Gate(targets, wl.random_unitary(1 << len(targets), rng), controls)
        from paper_2602_09604_gb300.state import DeviceState
        f = B.sv_fuse_circuit([g], n, mode=B.FUSE_NONE)
        info = B.sv_fused_get_info(f, 0)
        assert info["path"] == B.PATH_CONTROLLED or len(targets) + len(controls) <= 6
        st = DeviceState(n)
        st.load(psi0)
        st.apply(f)
        got = st.store()
        st.free()
        B.sv_fused_free(f)
        ref = psi0.astype(np.complex128)
        oracle.apply_gate(ref, n, g)
        assert np.max(np.abs(got - ref)) <= 2e-6, (targets, controls)


@pytest.mark.parametrize("n,max_k,prec", [(12, 2, 0), (17, 4, 0), (21, 6, 2), (21, 3, 0)])
def test_random_circuits_with_many_controls(B, n, max_k, prec):
    rng = np.random.default_rng(n * 10 + max_k)
    gates = []
    for _ in range(120):
        k = int(rng.integers(1, 4))
        nc = int(rng.integers(0, 9)) if rng.random() < 0.4 else 0
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    got, paths = run_gpu(B, n, gates, max_k=max_k, precision=prec, tc_min_k=4)
    assert B.PATH_CONTROLLED in paths
    ref = oracle.run_circuit(n, gates, 0, threads=oracle.default_threads())
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    assert oracle.l2_error(ref, got) <= 1e-4


def test_grover_20_closed_form_greedy_and_learned(B):
    n, marked, r = 20, 0xB5A3C, 6
    a, b = closed_forms.grover_amplitudes(n, r)
    kws = [dict(max_k=4), dict(max_k=6, precision=2, tc_min_k=4)]
    if os.path.exists(MODEL):
        kws.append(dict(max_k=6, precision=2, tc_min_k=4, mode=B.FUSE_LEARNED, model=B.sv_mlp_load(MODEL)))
    for kw in kws:
        got, paths = run_gpu(B, n, wl.grover_circuit(n, marked, r), **kw)
        assert paths.count(B.PATH_CONTROLLED) == 2 * r
        assert abs(got[marked] - a) <= 2e-5
        assert np.max(np.abs(np.delete(got, marked) - b)) <= 2e-6
        if kw.get("model") is not None:
            B.sv_mlp_free(kw["model"])


def test_grover_30_full_size(B):
    n, marked, r = 30, 0x2C0FFEE1, 3
    a, b = closed_forms.grover_amplitudes(n, r)
    got, paths = run_gpu(B, n, wl.grover_circuit(n, marked, r), max_k=6, precision=2, tc_min_k=4)
    assert paths.count(B.PATH_CONTROLLED) == 2 * r
    assert abs(got[marked] - a) <= 1e-5
    assert abs(float(np.sum(np.abs(got) ** 2, dtype=np.float64)) - 1.0) <= 1e-4
    got[marked] = b
    assert float(np.max(np.abs(got - np.complex64(b)))) <= 1e-6


def test_quantum_volume_matches_oracle(B):
    n = 18
    gates = wl.qv_circuit(n, seed=9)
    ref = oracle.run_circuit(n, gates, 0, threads=oracle.default_threads())
    for kw in (dict(max_k=2), dict(max_k=6, precision=2, tc_min_k=4)):
        got, _ = run_gpu(B, n, gates, **kw)
        assert oracle.fidelity(ref, got) >= 1 - 1e-6
        assert oracle.l2_error(ref, got) <= 1e-4
