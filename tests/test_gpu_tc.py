"""GPU parity of the tensor-core (tcgen05) path against the complex128 oracle.

Error model (stated, then checked): TF32 rounds both operands to 11 significant bits, so one
fused gate carries a relative error of about 2^-11 per product; BF16X3 keeps hi*hi + hi*lo +
lo*hi of bf16 splits, leaving about 3 * 2^-17 per product.  Over the 2^(k+1)-term real dot
products of a unit-norm state that bounds ||delta||_2 per gate by ~1e-3 (TF32) and ~3e-5 (BF16X3).
"""
import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GATE_L2 = {"tf32": 2e-3, "bf16x3": 5e-5}


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def DS(B):
    from paper_2602_09604_gb300.state import DeviceState
    return DeviceState


def prec(B, name):
    return {"tf32": B.PREC_TF32, "bf16x3": B.PREC_BF16X3}[name]


def run(B, DS, n, gates, max_k, precision, psi0=None, init=0, tc_min_k=4):
    st = DS(n)
    if psi0 is None:
        st.init(init)
    else:
        st.load(psi0)
    f = B.sv_fuse_circuit(gates, n, max_k=max_k, precision=precision, tc_min_k=tc_min_k)
    try:
        paths = [B.sv_fused_get_info(f, i)["path"] for i in range(B.sv_fused_count(f))]
        st.apply(f)
        out = st.store()
    finally:
        B.sv_fused_free(f)
        st.free()
    return out, paths


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
@pytest.mark.parametrize("n", [6, 10, 11, 13, 20])
def test_single_tc_gate(B, DS, mode, n):
    """Tensor cores take fused gates of k = 4..6 qubits once the state has 2^k blocks of 32
    amplitudes (n >= k + 5); smaller states fall back to the fp32 CUDA-core kernels."""
    rng = np.random.default_rng(300 + n)
    psi0 = wl.random_state(n, rng).astype(np.complex64)
    for k in (4, 5, 6):
        if k > n:
            continue
        cands = [tuple(sorted(int(t) for t in rng.choice(n, size=k, replace=False)))]
        if n - 5 >= k:
            cands.append(tuple(int(t) for t in 5 + np.sort(rng.choice(n - 5, size=k, replace=False))))
        if k <= 5:
            cands.append(tuple(range(k)))
        for tg in cands:
            g = wl.random_gate(n, k, rng, targets=tg)
            ref = psi0.astype(np.complex128)
            oracle.apply_gate(ref, n, g)
            got, paths = run(B, DS, n, [g], k, prec(B, mode), psi0=psi0)
            tc_path = B.PATH_TC_TF32 if mode == "tf32" else B.PATH_TC_BF16X3
            if n >= k + 5:
                assert paths == [tc_path]
            else:
                assert paths[0] in (B.PATH_LOW, B.PATH_HIGH, B.PATH_MIXED)
            err = oracle.l2_error(ref, got)
            assert err <= GATE_L2[mode], (k, tg, err)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_k6_every_kernel_variant(B, DS, mode):
    """k = 6 gates reach every tensor-core kernel form by their low targets (below qubit 5): up to
    two -- none, one at qubits 0-4, two, or exactly qubits 0 and 1 (16-byte loaders) -- run on the
    warp-specialised kernel, three or more are staged through shared memory.  Each matches the
    oracle."""
    n = 13
    rng = np.random.default_rng(606)
    psi0 = wl.random_state(n, rng).astype(np.complex64)
    for tg in [(5, 6, 7, 8, 9, 12), (3, 6, 7, 9, 10, 12), (4, 5, 8, 9, 11, 12), (1, 6, 7, 9, 10, 12),
               (3, 4, 7, 9, 10, 12), (0, 1, 7, 9, 10, 12), (0, 1, 5, 6, 7, 8), (0, 5, 6, 7, 8, 9),
               (0, 2, 4, 8, 9, 12), (0, 1, 2, 3, 4, 12)]:
        g = wl.random_gate(n, 6, rng, targets=tg)
        ref = psi0.astype(np.complex128)
        oracle.apply_gate(ref, n, g)
        got, paths = run(B, DS, n, [g], 6, prec(B, mode), psi0=psi0)
        assert paths == [B.PATH_TC_TF32 if mode == "tf32" else B.PATH_TC_BF16X3]
        err = oracle.l2_error(ref, got)
        assert err <= GATE_L2[mode], (tg, err)


@pytest.mark.parametrize("max_k", [4, 5, 6])
def test_tc_circuit_bf16x3_meets_fidelity_bar(B, DS, max_k):
    n, gates = wl.circuit_16q()
    ref = oracle.run_circuit(n, gates, 0, threads=oracle.default_threads())
    got, paths = run(B, DS, n, gates, max_k, B.PREC_BF16X3)
    assert any(p == B.PATH_TC_BF16X3 for p in paths)
    F = oracle.fidelity(ref, got)
    err = oracle.l2_error(ref, got)
    assert F >= 1 - 1e-6 and err <= 1e-4, (F, err)


def test_tc_grid_22q_both_modes_reported(B, DS):
    grid = wl.Grid(4, 6, dropped=((3, 4), (3, 5)))
    n = grid.n
    gates = wl.random_grid_circuit(grid, 12, seed=4)
    ref = oracle.run_circuit(n, gates, 0, threads=oracle.default_threads())
    got, _ = run(B, DS, n, gates, 6, B.PREC_BF16X3)
    F = oracle.fidelity(ref, got)
    assert F >= 1 - 1e-6 and oracle.l2_error(ref, got) <= 1e-4
    got_tf, _ = run(B, DS, n, gates, 6, B.PREC_TF32)
    F_tf = oracle.fidelity(ref, got_tf)
    assert F_tf >= 1 - 1e-3          # tf32 is the fast, lower-precision mode
    B.sv_device_status()
