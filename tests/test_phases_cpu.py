"""CPU-only checks of post-phase fusion (SV_FUSE_PHASES, host code): the fused gates followed by
their post-phases (applied here with numpy: amplitude i times exp(i theta) for each term whose two
bits are set in i) give the oracle's state for the QFT and for circuits dense in diagonal gates;
the QFT's controlled-phase ladders collapse into six-qubit gates; bad options are refused."""
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


def apply_fused_with_phases(B, f, n, psi):
    idx = np.arange(1 << n)
    for i in range(B.sv_fused_count(f)):
        info = B.sv_fused_get_info(f, i)
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
