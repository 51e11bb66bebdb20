"""Post-phase fusion (SV_FUSE_PHASES) on the GPU: the warp-specialised tensor-core kernel applies a
fused gate and, in the same pass, its post-phases (controlled-phase terms between its targets and
other qubits) -- the QFT and circuits dense in diagonal gates against the oracle, element by
element, in 3xBF16 and TF32, started from basis states through sv_init and sv_init_apply; swap
networks (runs of disjoint SWAP gates in one pass) bit for bit against the oracle."""
import math

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
    from paper_2602_09604_gb300 import binding
    from paper_2602_09604_gb300.state import DeviceState
    return binding, DeviceState


def _diag_circuit(n, count, rng):
    gates = []
    for _ in range(count):
        r = rng.random()
        a, b = (int(q) for q in rng.choice(n, size=2, replace=False))
        if r < 0.35:
            gates.append(wl.Gate((a, b), np.diag(np.exp(1j * rng.uniform(0, 2 * math.pi, 4)))))
        elif r < 0.5:
            gates.append(wl.Gate((a, b), wl.cphase(rng.uniform(0, 2 * math.pi))))
        elif r < 0.85:
            gates.append(wl.Gate((a,), wl.random_unitary(2, rng)))
        else:
            gates.append(wl.Gate((a, b), wl.random_unitary(4, rng)))
    return gates


def _run(B, DS, n, gates, prec, init, lazy):
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=prec, tc_min_k=4)
    carried = sum(1 for i in range(B.sv_fused_count(f)) if B.sv_fused_get_post_phases(f, i))
    st = DS(n)
    if lazy:
        B.sv_init_apply(st.h, init, f)
    else:
        st.init(init)
        st.apply(f)
    B.sv_device_status()
    got = st.store().astype(np.complex128)
    st.free()
    B.sv_fused_free(f)
    return got, carried


@pytest.mark.parametrize("n", [14, 18, 22])
def test_qft_phases_match_oracle(env, n):
    B, DS = env
    gates = wl.qft_circuit(n)
    x = wl.qft_basis_index(n, seed=n)
    ref = oracle.run_circuit(n, gates, x)
    for prec, tol in ((B.PREC_BF16X3, 2e-4), (B.PREC_TF32, 2e-3)):
        for lazy in (False, True):
            got, carried = _run(B, DS, n, gates, prec, x, lazy)
            assert carried >= 1
            # every QFT amplitude has size 2^(-n/2): relative error per element
            assert np.max(np.abs(got - ref)) * 2.0 ** (n / 2) <= tol, (prec, lazy)
            assert oracle.fidelity(ref, got) >= 1 - (1e-6 if prec == B.PREC_BF16X3 else 1e-4)


@pytest.mark.parametrize("n,seed", [(13, 1), (16, 2), (19, 3)])
def test_diagonal_heavy_phases_match_oracle(env, n, seed):
    B, DS = env
    rng = np.random.default_rng(seed)
    gates = _diag_circuit(n, 300, rng)
    x = int(rng.integers(0, 1 << n))
    ref = oracle.run_circuit(n, gates, x)
    got, carried = _run(B, DS, n, gates, B.PREC_BF16X3, x, False)
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    assert oracle.l2_error(ref, got) <= 1e-4


SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def _swap_network(n, rng, n_ll, n_lh, n_hh):
    """Disjoint swaps: n_ll with both qubits below 5, n_lh with one below and one at or above 5,
    n_hh with both at or above 5, in random order."""
    low = [int(q) for q in rng.permutation(5)]
    high = [int(q) for q in 5 + rng.permutation(n - 5)]
    pairs = [(low.pop(), low.pop()) for _ in range(n_ll)]
    pairs += [(low.pop(), high.pop()) for _ in range(n_lh)]
    pairs += [(high.pop(), high.pop()) for _ in range(n_hh)]
    rng.shuffle(pairs)
    return [wl.Gate(p, SWAP) for p in pairs]


@pytest.mark.parametrize("n,n_ll,n_lh,n_hh", [(10, 0, 5, 0), (10, 2, 1, 1), (12, 0, 0, 3), (13, 1, 3, 2),
                                              (17, 2, 1, 5), (20, 0, 5, 5), (21, 1, 2, 0), (23, 0, 4, 7)])
def test_swap_network_is_one_exact_pass(env, n, n_ll, n_lh, n_hh):
    """A run of disjoint SWAP gates fuses into one swap network (SV_PATH_SWAPS) whose pass moves
    every amplitude bit for bit to where the oracle's swaps put it (a random state, so every
    amplitude is distinct)."""
    B, DS = env
    rng = np.random.default_rng(n * 100 + n_lh)
    gates = _swap_network(n, rng, n_ll, n_lh, n_hh)
    assert len(gates) >= 3
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3, tc_min_k=4)
    assert B.sv_fused_count(f) == 1 and B.sv_fused_get_info(f, 0)["path"] == B.PATH_SWAPS
    assert len(B.sv_fused_get_swaps(f, 0)) == len(gates)
    psi = wl.random_state(n, rng).astype(np.complex64)
    st = DS(n)
    st.load(psi)
    recs = st.apply(f, timings=True)
    B.sv_device_status()
    got = st.store()
    st.free()
    B.sv_fused_free(f)
    ref = psi.astype(np.complex128)
    for g in gates:
        oracle.apply_gate(ref, n, g)
    assert np.array_equal(got, ref.astype(np.complex64))
    assert len(recs) == 1 and recs[0]["path"] == B.PATH_SWAPS and recs[0]["k"] == 0


@pytest.mark.parametrize("n", [14, 22])
def test_swap_network_refused_on_complex128(env, n):
    B, DS = env
    gates = _swap_network(n, np.random.default_rng(n), 0, 2, 2)
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3, tc_min_k=4)
    st = DS(n, c128=True)
    try:
        with pytest.raises(B.SvError):
            B.sv_apply_fused_gates(st.h, f)
    finally:
        st.free()
        B.sv_fused_free(f)
